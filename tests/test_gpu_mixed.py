"""Mixed-precision find (FP32 filter and early Newton, FP64 final steps)
against the FP64 oracle: element ids and codes identical, r within 1e-10,
dist2 within the FP64 tolerance; the error per result is reported."""
import numpy as np
import pytest

import oracle
from paper_2501_12349_b300 import workloads as W
from parity_util import compare_eval, compare_find, to_np
from test_gpu_parity import CASES, gpu_find, gpu_mesh, surface_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


@pytest.fixture(scope="module")
def fp():
    import paper_2501_12349_b300 as f
    f.lib()
    return f


def mixed_mesh(fp, torch, coords, d, dr, order):
    m = gpu_mesh(fp, torch, coords, d, dr, order)
    m.set_precision(fp.FP_MIXED)
    return m


def error_report(o, g):
    same = (o[0] == g[0]) & (o[1] == g[1]) & (o[0] != 2)
    dr = np.max(np.abs(o[2][same] - g[2][same]), axis=1)
    return {"max_dr": float(dr.max()) if dr.size else 0.0,
            "p9999_dr": float(np.quantile(dr, 0.9999)) if dr.size else 0.0,
            "mismatch": int((~((o[0] == g[0]) & (o[1] == g[1]))).sum())}


@pytest.mark.parametrize("case", list(CASES))
def test_mixed_cases(fp, torch, case):
    coords, d, dr, order, h = CASES[case]()
    om = oracle.OracleMesh(coords, d, dr, order + 1)
    rng = np.random.default_rng(21)
    if dr == d:
        pts = rng.uniform(-0.03, 1.03, (20000, d))
        if case == "quad2d_p3":
            w = W.config1()
            pts = np.concatenate([om.forward_map(w.fwd_elem, w.fwd_r), w.pts])
    else:
        pts = surface_points(om, rng, 20000, h)
    m = mixed_mesh(fp, torch, coords, d, dr, order)
    g = gpu_find(torch, m, pts)
    o = om.findpts(pts)
    compare_find(o, g, label="mixed " + case, xscale=1.3)
    print(case, error_report(o, g))
    assert m.device_status() == 0
    m.close()


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("shape", ["quad2d", "hex3d"])
def test_mixed_every_order(fp, torch, shape, order):
    rng = np.random.default_rng(200 + order)
    if shape == "quad2d":
        coords, d, dr = W.quad_mesh(5, order, amp=0.2, kind="kershaw"), 2, 2
    else:
        coords, d, dr = W.hex_mesh(3, order, 0.25), 3, 3
    om = oracle.OracleMesh(coords, d, dr, order + 1)
    pts = rng.uniform(-0.05, 1.05, (3000, d))
    m = mixed_mesh(fp, torch, coords, d, dr, order)
    compare_find(om.findpts(pts), gpu_find(torch, m, pts), label=f"mixed {shape} p{order}")
    m.close()


def test_mixed_config3_full_size_sampled(fp, torch):
    """10^7 points on the 32^3 p=4 mesh with a 3-component field, mixed
    precision, as the benchmark runs it; the oracle checks the 10^6-point
    subsample of every tenth point, and the per-result error against it is
    reported: max and 99.99th percentile of |dr| and of |du|/scale, and the
    code/element mismatch count."""
    w = W.config3()
    m = mixed_mesh(fp, torch, w.coords, 3, 3, w.order)
    st = torch.zeros(fp.FP_NSTATS, dtype=torch.int64, device="cuda")
    code, elem, r, dist2 = m.find(torch.from_numpy(w.pts).cuda(), stats=st)
    u = m.eval(code, elem, r, torch.from_numpy(w.field).cuda())
    g = tuple(to_np(t) for t in (code, elem, r, dist2))
    idx = np.arange(0, len(w.pts), 10)
    om = oracle.OracleMesh(w.coords, 3, 3, w.N)
    o = om.findpts(w.pts[idx])
    gs = tuple(a[idx] for a in g)
    compare_find(o, gs, label="mixed config3 subsample")
    uo = om.eval(w.field, *o[:3])
    ug = to_np(u)[:, idx]
    compare_eval(w.field, om.NE, w.N ** 3, o[1], uo, ug, "mixed config3 eval")
    rep = error_report(o, gs)
    f = w.field.reshape(3, om.NE, -1)
    found = o[1] >= 0
    scale = np.maximum(np.abs(uo), np.abs(f).max(axis=2)[:, np.where(found, o[1], 0)])
    du = (np.abs(uo - ug) / scale)[:, found].max(axis=0)
    rep.update(max_du_rel=float(du.max()), p9999_du_rel=float(np.quantile(du, 0.9999)))
    s = to_np(st)
    print("config3 mixed vs oracle on 1e6 points:", rep, "fallback fraction", s[6] / len(w.pts),
          "fp64 refinement evals/pt", s[4] / len(w.pts))
    assert rep["max_dr"] < 1e-10 and rep["max_du_rel"] < 1e-12
    assert s[6] < 0.05 * len(w.pts)
    assert m.device_status() == 0
    m.close()


def test_mixed_equals_f64_full_size(fp, torch):
    """All 10^6 points of the 3D workload: the mixed path and the FP64 path
    give the same element and code everywhere and r within 1e-10."""
    w = W.config2()
    m = gpu_mesh(fp, torch, w.coords, 3, 3, w.order)
    pts = torch.from_numpy(w.pts).cuda()
    a = tuple(to_np(t) for t in m.find(pts))
    m.set_precision(fp.FP_MIXED)
    b = tuple(to_np(t) for t in m.find(pts))
    compare_find(a, b, label="mixed vs f64")
    m.close()
