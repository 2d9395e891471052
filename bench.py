#!/usr/bin/env python
"""Benchmark of the local findpts hot path: located + evaluated points/s.

Workload (one step): find + interpolate 10^6 points on the 32^3 hex mesh of
order 4 (smooth deformation, amplitude 0.3; points uniform in
[-0.0034, 1.0034]^3), scalar field, all inputs resident on the GPU.  The
mesh setup (boxes, Psi_L) happens once before timing.  L2 is flushed (a
256 MB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision f64|mixed]
  python bench.py --impl reference ...   # the FP64 CPU oracle on a sample

Under torchrun each rank runs an independent replica on its own GPU with its
own point set (weak scaling, no collective on the data path); rank 0 prints
one JSON line with the whole-job throughput (points of all ranks / slowest
rank's time).
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "located+evaluated points/s (3D hex p=4)"
WORKLOAD = "hex3d_32^3_p4_kershaw0.3_1e6pts"


# DRAM bytes (read + write) per launch of a kernel on this workload (32^3
# p=4 mesh, 10^6 points), from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), with the SHA-256 of the kernel's source files at
# the time of the capture: the figure is reported only while the sources
# are unchanged, and as null once they differ.
PKG_SRC = ROOT / "paper_2501_12349_b300" / "csrc"
KERNEL_SOURCES = {
    "k_find_f64": ["find_f64.cuh", "find_common.cuh", "fp_basis.cuh", "beta_warp.cuh", "fp_common.cuh",
                   "find.cu", "order.cu", "setup.cu"],
    "k_find_mixed": ["find_mixed.cu", "find_mixed.cuh", "find_f64.cuh", "find_common.cuh", "fp_basis.cuh",
                     "beta_warp.cuh", "fp_common.cuh", "find.cu", "order.cu", "setup.cu"],
}
TRAFFIC = {
    # ncu -k regex:k_find_f64 -s 3 -c 1 (sections SpeedOfLight, MemoryWorkloadAnalysis, ...) on
    # bench.py --steps 2 --warmup 3 --skip-mixed --skip-batch --skip-serve --no-cpu-baseline
    "k_find_f64": {"sha": "2c6e87d7009350f2", "bytes": 729277952 + 74185984},
    # the same with --precision mixed and -k regex:k_find_mixed
    "k_find_mixed": {"sha": "1880c1ff13ae6897", "bytes": 653234176 + 74882304},
}


def source_sha(kernel: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        h.update(name.encode())
        h.update((PKG_SRC / name).read_bytes())
    return h.hexdigest()[:16]


def traffic_of(kernel: str):
    """(bytes per launch, note): the captured figure while the kernel's
    sources hash to the value it was captured with, else (None, why)."""
    rec = TRAFFIC.get(kernel)
    sha = source_sha(kernel)
    if rec is None:
        return None, f"no capture for sources {sha}"
    if rec["sha"] != sha:
        return None, f"captured for sources {rec['sha']}, now {sha}"
    return rec["bytes"], f"ncu capture, sources {sha}"


def iteration_model_flops(C, I, N, d):
    """The per-candidate and per-iteration flop model of a 3D find: per
    candidate the box tests (~30) and the closest-node start over all
    n_e = N^3 nodes (3 d n_e), per Newton iteration x and G by sum
    factorisation (2 (6 N^3 + 9 N^2 + 12 N)), the bases (~30 N) and the step
    algebra (~60); candidate and iteration counts are the kernel's own
    counters (they equal the oracle's: same candidates, iterations within
    1%)."""
    return float(C * (30 + 3 * d * N ** 3) + I * (2 * (6 * N ** 3 + 9 * N ** 2 + 12 * N) + 30 * N + 60))


def boxes_flops(NE, N, M, d, dr):
    """FP64 flops of k_boxes' function bounds (Secs. 3.1.1-3.1.2): for every
    bounding piece (6 faces of a hex, 4 edges of a quad, the element of a
    surface quad or line), coordinate and box kind (AABB, OBB frame), a
    lower and an upper bound over the M^dp Chebyshev grid points (dp the
    piece's dimension), each an N^dp-term sum of FMAs (Eq. 2D_function_bound
    with the min/max of the products precomputed)."""
    if dr == 3:
        pieces, dp = 6, 2
    elif d == 2 and dr == 2:
        pieces, dp = 4, 1
    else:
        pieces, dp = 1, dr
    return float(NE * pieces * d * 2 * 2 * 2 * (N ** dp) * (M ** dp))


def flop_terms(N, d, dr):
    """Flops (FMA = 2) of the per-point building blocks: x and G by sum
    factorisation (eval_g), the beta term restricted to the face (edge in
    2D) the iterate is held on (hess), one interpolated component
    (eval_x), the box tests, the closest-node search, the Newton step
    algebra."""
    ne = N ** dr
    if dr == 3:
        eval_g = d * 2 * (N * N * (2 * N + 3) + 4 * N) + dr * 8 * N
        hess = d * 2 * (3 * N * N + 3 * N) + 2 * 12 * N + 6 * d
        eval_x = 2 * (N ** 3 + N ** 2 + N) + dr * 4 * N
    else:
        eval_g = d * 2 * (N * (2 * N + 3)) + dr * 8 * N
        hess = d * 2 * N + 12 * N + 2 * d
        eval_x = 2 * (N ** 2 + N) + dr * 4 * N
    return {"eval_g": eval_g, "hess": hess, "eval_x": eval_x, "box": 2 * d * d + d,
            "node": 3 * d * ne, "newton": 60, "basis": dr * 4 * N,
            "node_start": 2 * d * dr * N + 3 * d, "linear_start": 2 * d * dr}


def find_flops(stats, N, d, dr, start="node"):
    """Algorithmic flops of a find from its counters: candidates C, Newton
    steps I, steps with the beta term B, full evaluations EV of x and G (re-
    evaluations after rejected steps are not counted).  start: "node" (the
    FP64 kernel: x at the closest node is the node, G one N-term sum per
    direction; the search itself runs on the FP32 pipe and is not counted;
    EV = one per trial step) or "linear" (the mixed kernel's FP32 phase:
    r0 from the linearised map, then a full evaluation; EV counts it)."""
    t = flop_terms(N, d, dr)
    C, I, B, EV = int(stats[0]), int(stats[1]), int(stats[3]), int(stats[7])
    return C * (t["box"] + t[start + "_start"]) + EV * t["eval_g"] + I * t["newton"] + B * t["hess"]


def flop_model(stats, N, d, dr, n_found, nc):
    """Algorithmic FP64 flops of one find launch and one eval launch."""
    t = flop_terms(N, d, dr)
    ev = n_found * (nc * (t["eval_x"] - t["basis"]) + t["basis"])
    return float(find_flops(stats, N, d, dr, "node")), float(ev)


def mixed_flop_model(stats, N, d, dr):
    """(FP32, FP64) algorithmic flops of one mixed-precision find: the FP32
    kernel's candidates, steps and evaluations (linearised initial guess
    instead of the node search), its refinements (x(r) in d components and
    the residual in FP64; the normal equations and their solve in FP32 for
    volumes, in FP64 with the FP64 Jacobian for surfaces and lines), and the
    FP64 kernel on the handed-over points (counters [8]-[15])."""
    f32, f64_main, f64_follow = mixed_flop_parts(stats, N, d, dr)
    return f32, f64_main + f64_follow


def mixed_flop_parts(stats, N, d, dr):
    """(FP32 flops of k_find_mixed, FP64 flops of k_find_mixed (its
    refinements), FP64 flops of the FP64 kernel on the handed-over points)."""
    t = flop_terms(N, d, dr)
    R = int(stats[4])
    f32 = find_flops(stats[0:8], N, d, dr, "linear")
    refine = d * (t["eval_x"] - t["basis"]) + t["basis"] + 2 * d
    solve = 2 * d * dr * (dr + 1) + 30
    if dr == d:
        f32 += R * solve
    else:
        refine += solve
    return float(f32), float(R * refine), float(find_flops(stats[8:16], N, d, dr, "node"))


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 20 ms; the sampler
    starts before the warm-up (nvidia-smi takes a while to start) and only the
    samples whose timestamps fall inside the timed region are kept."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark(self, begin: bool):
        """Marks the start (begin) or the end of the timed region."""
        if begin:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = [l.split(",") for l in Path(self.f.name).read_text().splitlines() if l.strip()]
        os.unlink(self.f.name)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        parsed = []
        for r in rows:
            try:
                ts = datetime.datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
                parsed.append((ts, float(r[2]), float(r[3]),
                               [nm for nm, v in zip(names, r[6:10]) if v.strip().lower() == "active"]))
            except (ValueError, IndexError):
                continue
        if not parsed:
            return None
        window = "timed region"
        sel = [p for p in parsed if self.t0 is not None and self.t1 is not None and self.t0 <= p[0] <= self.t1]
        if not sel:  # the region was shorter than the sampling interval
            window = "nearest sample"
            mid = 0.5 * ((self.t0 or 0) + (self.t1 or 0))
            sel = [min(parsed, key=lambda p: abs(p[0] - mid))]
        reasons = sorted({nm for p in sel for nm in p[3]})
        return {"sm_mhz": statistics.median(p[1] for p in sel), "sm_max_mhz": max(p[2] for p in sel),
                "reasons": reasons, "samples": len(sel), "window": window,
                "samples_total": len(parsed)}


def cpu_baseline(w, nc_field, target_s=10.0):
    """The FP64 oracle as it stands (brute-force candidates, direct sums,
    OpenMP over points) on a bounded sample of the same workload."""
    import oracle
    om = oracle.OracleMesh(w.coords, w.d, w.dr, w.N)
    t = time.perf_counter()
    probe = w.pts[:1000]
    c, e, r, d2 = om.findpts(probe)
    om.eval(w.field, c, e, r)
    dt = time.perf_counter() - t
    n = int(min(len(w.pts), max(2000, 1000 * target_s / max(dt, 1e-3))))
    sample = w.pts[:n]
    t = time.perf_counter()
    c, e, r, d2 = om.findpts(sample)
    om.eval(w.field, c, e, r)
    dt = time.perf_counter() - t
    cores = oracle.num_threads()
    # the same on one core, on a sample of about a second of its work
    n1 = max(200, int(n / max(cores, 1) * 1.0 / max(dt, 1e-3)))
    oracle.set_num_threads(1)
    t = time.perf_counter()
    c, e, r, d2 = om.findpts(w.pts[:n1])
    om.eval(w.field, c, e, r)
    dt1 = time.perf_counter() - t
    oracle.set_num_threads(cores)
    return {"value": n / dt, "unit": "points/s", "cores": cores, "kind": "oracle",
            "sample": f"first {n} points of the workload ({dt:.1f} s): brute-force box test over "
                      f"all {w.NE} elements + Newton + eval, FP64, OpenMP",
            "one_core": {"value": n1 / dt1, "unit": "points/s", "sample": f"first {n1} points ({dt1:.1f} s)"}}


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle timed on the host cores."""
    if rank != 0:
        return
    from paper_2501_12349_b300 import workloads as W
    import oracle
    w = W.config2()
    om = oracle.OracleMesh(w.coords, w.d, w.dr, w.N)
    per_step = 5000
    ts = []
    for s in range(args.warmup + args.steps):
        sl = w.pts[(s * per_step) % len(w.pts):][:per_step]
        t = time.perf_counter()
        c, e, r, d2 = om.findpts(sl)
        om.eval(w.field, c, e, r)
        dt = time.perf_counter() - t
        if s >= args.warmup:
            ts.append(dt)
    v = per_step * len(ts) / sum(ts)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "points/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(ts) / len(ts), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_points_per_step": per_step},
            "cpu_baseline": {"value": v, "unit": "points/s", "kind": "oracle", "cores": oracle.num_threads(),
                             "sample": f"{per_step} points per step of the 10^6-point workload"},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def mixed_block(fp, W, torch, dev, st, flush, args, rank, world, dist, peaks):
    """The 10^7-point, 3-component workload on the same mesh, find + eval,
    timed with the FP64 path and with the mixed path (FP32 filter and early
    Newton, FP64 final steps); both results are checked against each other."""
    w = W.config3(seed=3 + rank)
    coords = torch.from_numpy(w.coords).to(dev)
    field = torch.from_numpy(w.field).to(dev)
    pts = torch.from_numpy(w.pts).to(dev)
    n = pts.shape[0]
    mesh = fp.Mesh(coords, 3, 3, w.order)
    outs = {}
    res = {"workload": "hex3d_32^3_p4_kershaw0.3_1e7pts_nc3"}
    steps = max(3, args.steps // 2)
    for prec in ("f64", "mixed"):
        mesh.set_precision(fp.FP_MIXED if prec == "mixed" else fp.FP_F64)
        code = torch.empty(n, dtype=torch.int32, device=dev)
        elem = torch.empty(n, dtype=torch.int32, device=dev)
        r = torch.empty((n, 3), dtype=torch.float64, device=dev)
        d2 = torch.empty(n, dtype=torch.float64, device=dev)
        out = torch.empty((3, n), dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            flush.zero_()
            fp.fp_findpts(mesh.handle, pts, code, elem, r, d2)
            fp.fp_eval(mesh.handle, code, elem, r, field, 3, out)
        fms, ems = [], []
        fp.fp_kernel_times(mesh.handle)
        fp.fp_set_timing(mesh.handle, True)
        for _ in range(steps):
            flush.zero_()
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(st)
            fp.fp_findpts(mesh.handle, pts, code, elem, r, d2)
            b.record(st)
            fp.fp_eval(mesh.handle, code, elem, r, field, 3, out)
            c.record(st)
            c.synchronize()
            fms.append(a.elapsed_time(b))
            ems.append(b.elapsed_time(c))
        fp.fp_set_timing(mesh.handle, False)
        kms, kcalls = fp.fp_kernel_times(mesh.handle)
        kavg = [kms[i] / max(kcalls[i], 1) / 1e3 for i in range(fp.FP_NTIMES)]
        t = (sum(fms) + sum(ems)) / 1e3
        if world > 1:
            tt = torch.tensor([t], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t = float(tt.item())
        stats = torch.zeros(fp.FP_NSTATS, dtype=torch.int64, device=dev)
        fp.fp_findpts_stats(mesh.handle, pts, code, elem, r, d2, stats)
        sv = stats.cpu().numpy()
        outs[prec] = (code.clone(), elem.clone(), r.clone())
        fsec = statistics.mean(fms) / 1e3
        kernels = {}
        if prec == "f64":
            f32, f64 = 0.0, find_flops(sv, w.N, 3, 3, "node")
            model = iteration_model_flops(sv[0], sv[1], w.N, 3)
            kernels["k_find_f64"] = {"ms": kavg[fp.FP_TIME_FIND] * 1e3,
                                     "fp64_frac": model / kavg[fp.FP_TIME_FIND] / 1e12 / peaks[0],
                                     "fp64_frac_counted_work": f64 / kavg[fp.FP_TIME_FIND] / 1e12 / peaks[0]}
        else:
            f32, f64 = mixed_flop_model(sv, w.N, 3, 3)
            a32, a64m, a64f = mixed_flop_parts(sv, w.N, 3, 3)
            km, kf = kavg[fp.FP_TIME_FIND], kavg[fp.FP_TIME_FOLLOW]
            kernels["k_find_mixed"] = {"ms": km * 1e3, "fp32_tflops": a32 / km / 1e12,
                                       "fp32_frac": a32 / km / 1e12 / peaks[1],
                                       "fp64_tflops": a64m / km / 1e12, "fp64_frac": a64m / km / 1e12 / peaks[0]}
            kernels["fp64_follow_up"] = {"ms": kf * 1e3, "fp64_tflops": a64f / max(kf, 1e-9) / 1e12,
                                         "fp64_frac": a64f / max(kf, 1e-9) / 1e12 / peaks[0]}
        kernels["cell_order_ms"] = kavg[fp.FP_TIME_ORDER] * 1e3
        kernels["k_eval_f64_ms"] = kavg[fp.FP_TIME_EVAL] * 1e3
        res[prec] = {"value": world * n * steps / t, "unit": "points/s",
                     "find_ms": statistics.mean(fms), "eval_ms": statistics.mean(ems), "kernels": kernels,
                     "pipes": {"fp64": {"achieved": f64 / fsec / 1e12, "frac": f64 / fsec / 1e12 / peaks[0]},
                               "fp32": {"achieved": f32 / fsec / 1e12, "frac": f32 / fsec / 1e12 / peaks[1]},
                               "unit": "TFLOP/s", "time": "whole find call (all its kernels)"},
                     "counters": {"candidates": int(sv[0]), "iterations": int(sv[1]),
                                  "fp64_refine_evals": int(sv[4]), "fp64_box_tests": int(sv[5]),
                                  "to_fp64_kernel": int(sv[6]), "fp64_kernel_candidates": int(sv[8]),
                                  "fp64_kernel_iterations": int(sv[9])}}
    a, b = outs["f64"], outs["mixed"]
    same = (a[0] == b[0]) & (a[1] == b[1])
    res["code_elem_mismatch_vs_f64"] = int((~same).sum().item())
    found = same & (a[0] != 2)
    res["max_abs_dr_vs_f64"] = float((a[2] - b[2]).abs().max(dim=1).values[found].max().item())
    res["speedup_vs_f64"] = res["mixed"]["value"] / res["f64"]["value"]
    res["peaks_tflops"] = {"fp64": peaks[0], "fp32": peaks[1]}
    res["status"] = mesh.device_status()
    mesh.close()
    return res


def projection_block(fp, W, torch, dev, st, flush, args):
    """Closest-point projection on line elements (the paper's tangential
    relaxation example, boxes expanded by 100%): a curved closed boundary of
    2^16 cubic line elements, every node moved along and off the curve
    (262144 points); find + interpolation of the coordinate field (the
    closest points), FP64 and mixed precision."""
    import numpy as np
    coords = W.star_lines(1 << 16, 3)
    pts = torch.from_numpy(W.projection_points(coords, np.random.default_rng(7))).to(dev)
    xc = torch.from_numpy(coords).to(dev)
    mesh = fp.Mesh(xc, 2, 1, 3, bbox_tol=1.0)
    n = pts.shape[0]
    res = {"workload": "star curve, 65536 cubic line elements, 262144 moved nodes, bbox_tol 1.0"}
    code = torch.empty(n, dtype=torch.int32, device=dev)
    elem = torch.empty(n, dtype=torch.int32, device=dev)
    r = torch.empty((n, 1), dtype=torch.float64, device=dev)
    d2 = torch.empty(n, dtype=torch.float64, device=dev)
    out = torch.empty((2, n), dtype=torch.float64, device=dev)
    for prec in ("f64", "mixed"):
        mesh.set_precision(fp.FP_MIXED if prec == "mixed" else fp.FP_F64)
        for _ in range(args.warmup):
            fp.fp_findpts(mesh.handle, pts, code, elem, r, d2)
            fp.fp_eval(mesh.handle, code, elem, r, xc, 2, out)
        ts = []
        for _ in range(max(3, args.steps)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fp.fp_findpts(mesh.handle, pts, code, elem, r, d2)
            fp.fp_eval(mesh.handle, code, elem, r, xc, 2, out)
            b.record(st)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        codes = torch.bincount(code.long(), minlength=3).tolist()
        res[prec] = {"value": n / (statistics.mean(ts) / 1e3), "unit": "points/s", "ms": statistics.mean(ts),
                     "codes": {"interior": codes[0], "border": codes[1], "not_found": codes[2]}}
    res["status"] = mesh.device_status()
    mesh.close()
    return res


def surface_points(fp, torch, dev, mesh, w):
    """Query points of a surface mesh (sphere or torus): x_e(r) of the
    workload's (element, r) pairs, evaluated by the library's interpolation
    of the coordinate field, and for the 1% of pairs with an offset, moved
    0.1 h along the unit normal of the analytic surface at that point (it
    differs from the element's normal by the interpolation error).  Input
    preparation, outside any timed region."""
    n = len(w.fwd_elem)
    code = torch.zeros(n, dtype=torch.int32, device=dev)
    elem = torch.from_numpy(w.fwd_elem).to(dev)
    r = torch.from_numpy(np.ascontiguousarray(w.fwd_r)).to(dev)
    x = mesh.eval(code, elem, r, torch.from_numpy(w.coords).to(dev)).T.contiguous()  # [n][3]
    if "sphere" in w.name:
        nrm = x / x.norm(dim=1, keepdim=True)
    else:  # torus: from the tube's centre circle (radius 1 in the xy plane)
        ring = x.clone()
        ring[:, 2] = 0.0
        ring = ring / ring.norm(dim=1, keepdim=True)
        nrm = x - ring
        nrm = nrm / nrm.norm(dim=1, keepdim=True)
    off = torch.from_numpy(w.fwd_offset).to(dev)
    return (x + off[:, None] * nrm).contiguous()


def batch_block(fp, W, torch, dev, st, flush, args):
    """The 64-mesh workload (quads, hexes, sphere/torus surfaces, p = 2..7,
    1e3-5e4 elements, 1e3-1e6 points each, scalar fields; surface points 99%
    x_e(r), 1% moved 0.1 h off the surface): one autotuned graph launch per
    run, against the same work issued as separate per-mesh fp_findpts +
    fp_eval calls; FP64 and mixed precision."""
    t0 = time.perf_counter()
    ws = W.config4()
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    meshes = [fp.Mesh(torch.from_numpy(w.coords).to(dev), w.d, w.dr, w.order) for w in ws]
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    entries = [(m, surface_points(fp, torch, dev, m, w) if w.dr < w.d else torch.from_numpy(w.pts).to(dev),
                torch.from_numpy(w.field).to(dev)) for m, w in zip(meshes, ws)]
    total = sum(e[1].shape[0] for e in entries)
    res = {"workload": "64 meshes: quad2d/hex3d/sphere+torus surfaces, p=2..7, NE 1e3-5e4, 1e3-1e6 pts, nc=1",
           "meshes": len(ws), "points": total, "elements": int(sum(w.NE for w in ws)),
           "generate_s": gen_s, "setup_s": setup_s}
    reps = max(3, args.steps // 2)

    def timed(fn):
        ms = []
        for k in range(args.warmup + reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            b.record(st)
            b.synchronize()
            if k >= args.warmup:
                ms.append(a.elapsed_time(b))
        return statistics.mean(ms)

    for prec, code_ in (("f64", fp.FP_F64), ("mixed", fp.FP_MIXED)):
        b = fp.Batch(entries, code_)
        t0 = time.perf_counter()
        b.autotune()
        tune_s = time.perf_counter() - t0
        ms_batch = timed(b.run)
        b.set_fused(True)  # every shape in one persistent find launch
        ms_fused = timed(b.run)
        b.set_fused(False)
        outs = b.outputs

        def separate():
            for (m, pts, fld), o in zip(entries, outs):
                fp.fp_findpts(m.handle, pts, o[0], o[1], o[2], o[3])
                fp.fp_eval(m.handle, o[0], o[1], o[2], fld, o[4].shape[0], o[4])

        for m in meshes:
            m.set_precision(code_)
        ms_sep = timed(separate)
        for m in meshes:
            m.set_precision(fp.FP_F64)
        res[prec] = {"value": total / (ms_batch / 1e3), "unit": "points/s", "ms_per_run": ms_batch,
                     "separate_calls_ms": ms_sep, "speedup_vs_separate": ms_sep / ms_batch,
                     "fused_launch_ms": ms_fused, "fused_vs_per_shape": ms_batch / ms_fused,
                     "autotune_s": tune_s,
                     "classes": [{"N": i.N, "d": i.d, "dr": i.dr, "items": i.n_items, "points": int(i.n_points),
                                  "ctas_per_sm": i.ctas_per_sm, "chunk": i.chunk_points,
                                  "ms": round(float(i.tuned_ms), 3)} for i in b.classes()]}
        b.close()
    res["speedup_mixed_vs_f64"] = res["mixed"]["value"] / res["f64"]["value"]
    for m in meshes:
        m.close()
    return res


def serve_block(fp, W, torch, dev, args):
    """Serving: 8 resident hex meshes (p = 3..7, 1e4-1e5 elements); requests
    of log-uniform size 1e2-1e6, half remap (find + interpolate a scalar
    field), half particle (4 explicit-midpoint steps through the interpolated
    velocity u = (sin pi x cos pi y, -cos pi x sin pi y, 0.1), dt = 0.1 h_min /
    |u|_max).  First a burst measures the served capacity, then Poisson
    arrivals at 0.5, 0.7 and 0.9 of it give latency percentiles.  Results of
    the load requests land in a shared pinned host sink (timing only)."""
    t0 = time.perf_counter()
    ws = W.config5_meshes()
    entries, meshes = [], []
    for w in ws:
        m = fp.Mesh(torch.from_numpy(w.coords).to(dev), 3, 3, w.order)
        meshes.append(m)
        entries.append((m, torch.from_numpy(w.field).to(dev), torch.from_numpy(W.velocity_field(w.coords)).to(dev)))
    gen_s = time.perf_counter() - t0
    h_min = min(w.h for w in ws)
    dt = 0.1 * h_min / np.sqrt(1.01)
    policy = fp.FP_SCHED_SLACK if args.serve_policy == "slack" else fp.FP_SCHED_SRPT
    srv = fp.Server(entries, mem_budget=8 << 30, max_active=64, precision=fp.FP_MIXED,
                    tick_points=args.serve_tick_points, policy=policy,
                    slack_base=args.serve_slack_base, slack_factor=args.serve_slack_factor)
    rng = np.random.default_rng(5)
    nmax = 10 ** 6
    pool_r = torch.from_numpy(rng.uniform(-0.01, 1.01, (nmax, 3))).pin_memory()
    pool_p = torch.from_numpy(rng.uniform(0.05, 0.95, (nmax, 3))).pin_memory()
    sink = (torch.empty(nmax, dtype=torch.int32).pin_memory(), torch.empty(nmax, dtype=torch.int32).pin_memory(),
            torch.empty((nmax, 3), dtype=torch.float64).pin_memory(), torch.empty(nmax, dtype=torch.float64).pin_memory(),
            torch.empty((nmax, 3), dtype=torch.float64).pin_memory())

    def draw(k):
        out = []
        for _ in range(k):
            n = int(np.exp(rng.uniform(np.log(1e2), np.log(1e6))))
            kind = fp.FP_REQ_REMAP if rng.integers(0, 2) == 0 else fp.FP_REQ_PARTICLE
            mesh = int(rng.integers(0, len(ws)))
            off = int(rng.integers(0, nmax - n + 1))
            out.append((mesh, kind, n, off))
        return out

    def submit(req):
        mesh, kind, n, off = req
        pool = pool_r if kind == fp.FP_REQ_REMAP else pool_p
        return srv.submit(mesh, kind, pool[off:off + n], rk_steps=4 if kind else 0, dt=dt, outputs=sink)

    def stage_points(reqs):
        return sum(n * (1 if k == fp.FP_REQ_REMAP else 9) for _, k, n, _ in reqs)

    def collect(ids):
        lat = []
        for i in ids:
            srv.wait(i, timeout_s=600)
            lat.append(srv.timing(i)[1])
            srv.release(i)
        return lat

    res = {"workload": "8 hex meshes p=3..7 NE 1e4-1e5; requests 1e2-1e6 pts, half remap, half particle (4 RK2 steps)",
           "generate_and_setup_s": gen_s, "precision": "mixed", "dt": dt,
           "tick_points": args.serve_tick_points, "policy": args.serve_policy,
           "slack_base": args.serve_slack_base, "slack_factor": args.serve_slack_factor}
    burst = draw(args.serve_burst)

    def serial_f64(reqs):
        """The same requests one at a time through the plain FP64 calls:
        upload, find + eval per stage (particles: midpoint steps with a torch
        update), download."""
        st = torch.cuda.current_stream()
        for mesh, kind, n, off in reqs:
            m, fld, vel = entries[mesh]
            pool = pool_r if kind == fp.FP_REQ_REMAP else pool_p
            x = pool[off:off + n].to(dev, non_blocking=True)
            code = torch.empty(n, dtype=torch.int32, device=dev)
            elem = torch.empty(n, dtype=torch.int32, device=dev)
            r = torch.empty((n, 3), dtype=torch.float64, device=dev)
            d2 = torch.empty(n, dtype=torch.float64, device=dev)
            if kind == fp.FP_REQ_REMAP:
                u = torch.empty((1, n), dtype=torch.float64, device=dev)
                fp.fp_findpts(m.handle, x, code, elem, r, d2)
                fp.fp_eval(m.handle, code, elem, r, fld, 1, u)
                sink[4].view(-1)[:n].copy_(u.view(-1), non_blocking=True)
            else:
                u = torch.empty((3, n), dtype=torch.float64, device=dev)
                for _ in range(4):
                    fp.fp_findpts(m.handle, x, code, elem, r, d2)
                    fp.fp_eval(m.handle, code, elem, r, vel, 3, u)
                    xm = (x + 0.5 * dt * u.T).contiguous()
                    fp.fp_findpts(m.handle, xm, code, elem, r, d2)
                    fp.fp_eval(m.handle, code, elem, r, vel, 3, u)
                    x = (x + dt * u.T).contiguous()
                fp.fp_findpts(m.handle, x, code, elem, r, d2)
                sink[4][:n].copy_(x, non_blocking=True)
            sink[0][:n].copy_(code, non_blocking=True)
            sink[1][:n].copy_(elem, non_blocking=True)
            sink[2][:n].copy_(r, non_blocking=True)
            sink[3][:n].copy_(d2, non_blocking=True)
        st.synchronize()

    t0 = time.perf_counter()
    serial_f64(burst)
    wall_serial = time.perf_counter() - t0
    res["serial_f64_same_requests"] = {"wall_s": wall_serial, "requests_per_s": len(burst) / wall_serial,
                                       "stage_points_per_s": stage_points(burst) / wall_serial}

    def burst_run(server):
        t0 = time.perf_counter()
        ids = []
        for q in burst:
            mesh, kind, n, off = q
            pool = pool_r if kind == fp.FP_REQ_REMAP else pool_p
            ids.append(server.submit(mesh, kind, pool[off:off + n], rk_steps=4 if kind else 0, dt=dt, outputs=sink))
        for i in ids:
            server.wait(i, timeout_s=600)
            server.release(i)
        return time.perf_counter() - t0

    srv64 = fp.Server(entries, mem_budget=8 << 30, max_active=64, precision=fp.FP_F64)
    wall64 = burst_run(srv64)
    srv64.close()
    res["served_f64_capacity"] = {"wall_s": wall64, "requests_per_s": len(burst) / wall64,
                                  "stage_points_per_s": stage_points(burst) / wall64}
    wall = burst_run(srv)
    cap_rps = len(burst) / wall
    res["capacity"] = {"requests": len(burst), "wall_s": wall, "requests_per_s": cap_rps,
                       "request_points_per_s": sum(q[2] for q in burst) / wall,
                       "stage_points_per_s": stage_points(burst) / wall,
                       "speedup_vs_serial_f64": wall_serial / wall,
                       "speedup_vs_served_f64": wall64 / wall}
    res["load"] = []
    for rho in (0.5, 0.7, 0.9):
        reqs = draw(args.serve_requests)
        lam = rho * cap_rps
        arrivals = np.cumsum(rng.exponential(1.0 / lam, len(reqs)))
        ids = []
        t0 = time.perf_counter()
        for a, q in zip(arrivals, reqs):
            now = time.perf_counter() - t0
            if a > now:
                time.sleep(a - now)
            ids.append(submit(q))
        lat = collect(ids)
        wall = time.perf_counter() - t0
        sizes = np.array([q[2] for q in reqs])
        lat_a = np.array(lat)
        by_size = []
        for lo, hi in ((1e2, 1e3), (1e3, 1e4), (1e4, 1e5), (1e5, 1e6 + 1)):
            sel = (sizes >= lo) & (sizes < hi)
            if sel.any():
                by_size.append({"points": f"[{lo:.0e}, {min(hi, 1e6):.0e})", "requests": int(sel.sum()),
                                "p50_ms": 1e3 * float(np.percentile(lat_a[sel], 50)),
                                "p99_ms": 1e3 * float(np.percentile(lat_a[sel], 99))})
        res["load"].append({"rho": rho, "arrival_rate_rps": lam, "requests": len(reqs), "wall_s": wall,
                            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                            "mean_ms": 1e3 * float(np.mean(lat)), "by_size": by_size,
                            "request_points_per_s": sum(q[2] for q in reqs) / wall,
                            "stage_points_per_s": stage_points(reqs) / wall})
    st = srv.stats()
    res["server"] = {"ticks": st.ticks, "completed": st.completed, "timeouts": st.timeouts}
    srv.close()
    for m in meshes:
        m.close()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f64", choices=["f64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-mixed", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-burst", type=int, default=200)
    ap.add_argument("--serve-tick-points", type=int, default=1 << 19,
                    help="points per server tick (fp_server_opts.tick_points)")
    ap.add_argument("--serve-policy", default="slack", choices=["slack", "srpt"],
                    help="server tick policy (fp_server_opts.policy)")
    ap.add_argument("--serve-slack-base", type=float, default=float(1 << 20))
    ap.add_argument("--serve-slack-factor", type=float, default=4.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    import paper_2501_12349_b300 as fp
    from paper_2501_12349_b300 import workloads as W

    w = W.config2(seed=2 + rank)
    dev = torch.device("cuda", local)
    st = torch.cuda.current_stream()
    coords = torch.from_numpy(w.coords).to(dev)
    field = torch.from_numpy(w.field).to(dev)
    pts = torch.from_numpy(w.pts).to(dev)
    n = pts.shape[0]
    t0 = time.perf_counter()
    mesh = fp.Mesh(coords, 3, 3, w.order, precision=fp.FP_MIXED if args.precision == "mixed" else fp.FP_F64)
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t0)
    code = torch.empty(n, dtype=torch.int32, device=dev)
    elem = torch.empty(n, dtype=torch.int32, device=dev)
    r = torch.empty((n, 3), dtype=torch.float64, device=dev)
    dist2 = torch.empty(n, dtype=torch.float64, device=dev)
    out = torch.empty((1, n), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        fp.fp_findpts(mesh.handle, pts, code, elem, r, dist2)
        fp.fp_eval(mesh.handle, code, elem, r, field, 1, out)

    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    time.sleep(0.3)  # nvidia-smi is sampling by now

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    fp.fp_kernel_times(mesh.handle)  # start the per-kernel intervals afresh
    fp.fp_set_timing(mesh.handle, True)
    barrier()
    torch.cuda.synchronize()
    clocks.mark(True)
    wall0 = time.perf_counter()
    for s in range(args.steps):
        flush.zero_()
        ev[s][0].record(st)
        fp.fp_findpts(mesh.handle, pts, code, elem, r, dist2)
        ev[s][1].record(st)
        fp.fp_eval(mesh.handle, code, elem, r, field, 1, out)
        ev[s][2].record(st)
    torch.cuda.synchronize()
    clocks.mark(False)
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    fp.fp_set_timing(mesh.handle, False)
    kms, kcalls = fp.fp_kernel_times(mesh.handle)
    kernel_ms = {name: kms[i] / max(kcalls[i], 1) for i, name in
                 ((fp.FP_TIME_ORDER, "cell_order"), (fp.FP_TIME_FIND, "find_kernel"),
                  (fp.FP_TIME_FOLLOW, "fp64_follow_up"), (fp.FP_TIME_EVAL, "eval")) if kcalls[i]}
    find_ms = [ev[s][0].elapsed_time(ev[s][1]) for s in range(args.steps)]
    eval_ms = [ev[s][1].elapsed_time(ev[s][2]) for s in range(args.steps)]
    step_ms = [a + b for a, b in zip(find_ms, eval_ms)]
    t_local = sum(step_ms) / 1e3
    if world > 1:
        tt = torch.tensor([t_local], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    else:
        t_max = t_local
    value = world * n * args.steps / t_max

    # counters for the algorithmic flop count (untimed)
    stats = torch.zeros(fp.FP_NSTATS, dtype=torch.int64, device=dev)
    fp.fp_findpts_stats(mesh.handle, pts, code, elem, r, dist2, stats)
    sv = stats.cpu().numpy()
    n_found = int((code != 2).sum().item())
    fl_find, fl_eval = flop_model(sv, w.N, 3, 3, n_found, 1)
    peak64 = fp.fp_alu_peak(0, 4000) / 1e3  # TFLOP/s
    peak32 = fp.fp_alu_peak(1, 4000) / 1e3
    find_avg = statistics.mean(find_ms) / 1e3
    eval_avg = statistics.mean(eval_ms) / 1e3
    peak_src = "FP64 FMA pipe, measured live by fp_alu_peak (no FP64 entry in the measured peaks file)"
    # the dominant kernel's own average duration (CUDA events recorded by
    # the library between the kernels of each timed call, on its stream)
    kfind = kernel_ms.get("find_kernel", statistics.mean(find_ms)) / 1e3
    if args.precision == "f64":
        model = iteration_model_flops(sv[0], sv[1], w.N, 3)
        ach = model / kfind / 1e12
        traffic, tnote = traffic_of("k_find_f64")
        roofline = {"bound": "alu", "achieved": ach, "peak": peak64, "unit": "TFLOP/s", "frac": ach / peak64,
                    "traffic": traffic, "traffic_source": tnote, "kernel": "k_find_f64",
                    "kernel_ms": kfind * 1e3, "peak_source": peak_src,
                    "flop_model": "per candidate 30 + 3 d N^3, per iteration 2(6N^3+9N^2+12N) + 30N + 60",
                    "flops_per_launch": model,
                    "counted_work": {"achieved": fl_find / kfind / 1e12, "frac": fl_find / kfind / 1e12 / peak64,
                                     "flops_per_launch": fl_find,
                                     "model": "only the evaluations the kernel performs (node start without a "
                                              "full evaluation), face-restricted beta term, 60 per step"},
                    "whole_call": {"ms": find_avg * 1e3, "frac": model / find_avg / 1e12 / peak64}}
    else:
        f32, f64 = mixed_flop_model(sv, w.N, 3, 3)
        a64, a32 = f64 / find_avg / 1e12, f32 / find_avg / 1e12
        traffic, tnote = traffic_of("k_find_mixed")
        roofline = {"bound": "alu", "achieved": a64, "peak": peak64, "unit": "TFLOP/s", "frac": a64 / peak64,
                    "traffic": traffic, "traffic_source": tnote,
                    "kernel": "k_find_mixed + k_find_f64 (FP64 pipe)", "peak_source": peak_src,
                    "fp32": {"achieved": a32, "peak": peak32, "frac": a32 / peak32}}
    info = mesh.info()
    fb = boxes_flops(w.NE, w.N, info.M, 3, 3)
    setup_roofline = {"kernel": "k_boxes", "bound": "alu", "ms": info.setup_boxes_ms,
                      "achieved": fb / (info.setup_boxes_ms / 1e3) / 1e12, "peak": peak64, "unit": "TFLOP/s",
                      "frac": fb / (info.setup_boxes_ms / 1e3) / 1e12 / peak64, "flops": fb,
                      "grid_build_ms": info.setup_grid_ms, "setup_call_ms": setup_ms}

    # end to end through host buffers: fp_findpts_host, the public call for
    # host data (pinned points in; code, elem, r, dist2 and the interpolated
    # values out; its copies overlap the kernels chunk by chunk)
    hp = torch.from_numpy(w.pts).pin_memory()
    hc = torch.empty(n, dtype=torch.int32).pin_memory()
    he = torch.empty(n, dtype=torch.int32).pin_memory()
    hr = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    hd = torch.empty(n, dtype=torch.float64).pin_memory()
    hu = torch.empty((1, n), dtype=torch.float64).pin_memory()
    e2e_ms = []
    for s in range(args.warmup + args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        fp.fp_findpts_host(mesh.handle, hp, hc, he, hr, hd, field, 1, hu, 0, st)
        b.record(st)
        b.synchronize()
        if s >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
    h2d = n * 3 * 8
    d2h = n * (4 + 4 + 24 + 8 + 8)
    e2e_t = sum(e2e_ms) / 1e3
    if world > 1:
        tt = torch.tensor([e2e_t], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_t = float(tt.item())
    e2e_v = world * n * args.steps / e2e_t
    status = mesh.device_status()
    mesh.close()
    mixed = None if args.skip_mixed else mixed_block(fp, W, torch, dev, st, flush, args, rank, world, dist, (peak64, peak32))
    batched = None if (args.skip_batch or rank != 0) else batch_block(fp, W, torch, dev, st, flush, args)
    projection = None if (args.skip_batch or rank != 0) else projection_block(fp, W, torch, dev, st, flush, args)
    serving = None if (args.skip_serve or rank != 0) else serve_block(fp, W, torch, dev, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, 1)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "f64" else "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "points_per_gpu": n, "precision": args.precision,
                       "nc": 1, "l2": "flushed (256 MB write) before each timed step",
                       "parallelism": f"replicas{world}"},
            # per step: the cell order (k_point_cells; the bucket scan
            # k_scan_tiles, k_scan, k_scan_add; k_point_scatter), the find
            # (k_find_f64; mixed: k_find_mixed + the FP64 kernel on the
            # handed-over points) and k_eval_f64
            "gpu_launches": (7 if args.precision == "f64" else 8) * args.steps,
            "roofline": roofline,
            "setup_roofline": setup_roofline,
            "kernels_ms": {"find_call": statistics.mean(find_ms), "eval_call": statistics.mean(eval_ms),
                           **kernel_ms},
            "eval_roofline": {"bound": "alu", "achieved": fl_eval / eval_avg / 1e12, "peak": peak64,
                              "unit": "TFLOP/s", "frac": fl_eval / eval_avg / 1e12 / peak64},
            "find_counters": {"candidates": int(sv[0]), "iterations": int(sv[1]), "rejected": int(sv[2]),
                              "beta_iterations": int(sv[3]), "evaluations": int(sv[7]),
                              "per_point_iterations": float(sv[1]) / n},
            "setup_ms": setup_ms, "wall_s_timed": wall, "device_status": status,
            "e2e": {"value": e2e_v, "unit": "points/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "cpu_baseline": cpu, "clocks": clk, "mixed": mixed, "batched": batched, "projection": projection, "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
