"""Element-partitioned Find across ranks (Psi_G, Sec. 3.1.4; multi-rank
Find, Sec. 3.2) as gloo process groups on the CPU, world sizes 2 and 3.
Each rank holds a partition of the mesh and searches it with the FP64
oracle (the stand-in for the GPU find of a real multi-GPU run); the routed
and merged result must equal the oracle's search of the whole mesh."""
import os
import socket
from datetime import timedelta

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2501_12349_b300 import distributed as D
from paper_2501_12349_b300 import workloads as W
from parity_util import R_TOL, D2_ABS, D2_REL, D2_X


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _mesh(kind):
    if kind == "quad2d":
        return W.config1().coords, 2, 2, 4
    if kind == "hex3d":
        return W.hex_mesh(4, 3, 0.25), 3, 3, 4
    return W.cubed_sphere(2, 3), 3, 2, 4


def _partition(NE, P, how):
    e = np.arange(NE)
    owner = (e * P) // NE if how == "blocks" else (e * 7) % P
    return [np.flatnonzero(owner == p) for p in range(P)]


def _points(coords, d, dr, N, rank, n=1500):
    om = oracle.OracleMesh(coords, d, dr, N)
    rng = np.random.default_rng(600 + rank)
    if dr == d:
        return rng.uniform(-0.1, 1.1, (n, d))
    el = rng.integers(0, om.NE, n).astype(np.int32)
    x = om.forward_map(el, rng.uniform(-1, 1, (n, dr)))
    x[: n // 3] *= 1.0 + rng.uniform(-0.02, 0.02, (n // 3, 1))  # off the sphere: BORDER / NOT_FOUND
    return x


def _worker(rank, world, port, kind, how, errfile):
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=120))
        coords, d, dr, N = _mesh(kind)
        parts = _partition(coords.shape[1], world, how)
        mine = parts[rank]
        local = oracle.OracleMesh(np.ascontiguousarray(coords[:, mine]), d, dr, N)

        def local_find(x):
            c, e, r, d2 = local.findpts(x.numpy())
            return torch.from_numpy(c), torch.from_numpy(e), torch.from_numpy(r), torch.from_numpy(d2)

        gmap = D.GlobalMap.build(torch.from_numpy(local.aabb), d, group=None)
        # Psi_G against brute force over every rank's boxes
        allb = [oracle.OracleMesh(np.ascontiguousarray(coords[:, p]), d, dr, N).aabb for p in parts]
        for lc in range(gmap.start.shape[0] - 1):
            g = lc * world + rank
            ci = [(g // gmap.n ** k) % gmap.n for k in range(d)]
            lo = gmap.lo.numpy() + np.array(ci) / gmap.scale.numpy()
            expect = []
            for p, b in enumerate(allb):
                c0 = D._cells(torch.from_numpy(b[:, :d]), gmap.lo, gmap.scale, gmap.n).numpy()
                c1 = D._cells(torch.from_numpy(b[:, d:]), gmap.lo, gmap.scale, gmap.n).numpy()
                if np.any(np.all((c0 <= ci) & (c1 >= ci), axis=1)):
                    expect.append(p)
            got = gmap.ranks[gmap.start[lc]:gmap.start[lc + 1]].tolist()
            assert got == expect, (lc, got, expect, lo)
        pts = _points(coords, d, dr, N, rank)
        code, rk, el, r, d2 = (t.numpy() for t in D.find(local_find, torch.from_numpy(pts), gmap))
        ref = oracle.OracleMesh(coords, d, dr, N).findpts(pts)
        gel = np.where(rk >= 0, np.array([parts[q][e] if q >= 0 else -1 for q, e in zip(rk, el)]), -1)
        np.testing.assert_array_equal(code, ref[0])
        same = gel == ref[1]
        tol = D2_REL * ref[3] + D2_X * np.sqrt(np.where(np.isfinite(ref[3]), ref[3], 0)) + D2_ABS
        tie = ~same & (code == 1) & (np.abs(d2 - ref[3]) <= tol)
        assert np.all(same | tie), np.flatnonzero(~(same | tie))[:5]
        f = same & (code != 2)
        assert np.max(np.abs(r[f] - ref[2][f]), initial=0.0) <= R_TOL
        assert np.all(np.abs(d2[f] - ref[3][f]) <= tol[f])
        nf = code == 2
        assert np.all(rk[nf] == -1) and np.all(np.isinf(d2[nf]))
        # the exchange found points that the local search alone did not
        lc_, _, _, _ = local_find(torch.from_numpy(pts))
        assert np.sum(lc_.numpy() != code) > 0
        dist.destroy_process_group()
    except BaseException as ex:  # reported to the parent
        with open(errfile, "a") as fh:
            fh.write(f"rank {rank}: {type(ex).__name__}: {ex}\n")
        raise


@pytest.mark.parametrize("world,kind,how", [(2, "quad2d", "blocks"), (3, "quad2d", "scatter"),
                                            (2, "hex3d", "scatter"), (3, "sphere", "blocks")])
def test_partitioned_find_equals_global(tmp_path, world, kind, how):
    err = str(tmp_path / "err.txt")
    try:
        mp.spawn(_worker, args=(world, _free_port(), kind, how, err), nprocs=world, join=True)
    except Exception:
        msg = open(err).read() if os.path.exists(err) else ""
        raise AssertionError(msg)


def _worker_empty(rank, world, port, errfile):
    """A rank that owns no elements and issues no points still takes part."""
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=120))
        coords, d, dr, N = _mesh("quad2d")
        mine = np.arange(coords.shape[1]) if rank == 0 else np.arange(0)
        local = oracle.OracleMesh(np.ascontiguousarray(coords[:, mine]), d, dr, N) if mine.size else None

        def local_find(x):
            n = x.shape[0]
            if local is None or n == 0:
                return (torch.full((n,), 2, dtype=torch.int32), torch.full((n,), -1, dtype=torch.int32),
                        torch.zeros((n, dr)), torch.full((n,), float("inf")))
            c, e, r, d2 = local.findpts(x.numpy())
            return torch.from_numpy(c), torch.from_numpy(e), torch.from_numpy(r), torch.from_numpy(d2)

        aabb = torch.from_numpy(local.aabb) if local is not None else torch.zeros((0, 2 * d), dtype=torch.float64)
        gmap = D.GlobalMap.build(aabb, d)
        pts = np.random.default_rng(9).uniform(0, 1, (500 if rank == 1 else 0, d))
        code, rk, el, r, d2 = (t.numpy() for t in D.find(local_find, torch.from_numpy(pts), gmap))
        if rank == 1:
            ref = oracle.OracleMesh(coords, d, dr, N).findpts(pts)
            np.testing.assert_array_equal(code, ref[0])
            np.testing.assert_array_equal(el[code != 2], ref[1][code != 2])
            assert np.all(rk[code != 2] == 0)
        dist.destroy_process_group()
    except BaseException as ex:
        with open(errfile, "a") as fh:
            fh.write(f"rank {rank}: {type(ex).__name__}: {ex}\n")
        raise


def test_partitioned_find_empty_rank(tmp_path):
    err = str(tmp_path / "err.txt")
    try:
        mp.spawn(_worker_empty, args=(2, _free_port(), err), nprocs=2, join=True)
    except Exception:
        msg = open(err).read() if os.path.exists(err) else ""
        raise AssertionError(msg)
