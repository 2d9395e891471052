"""The allocation-free mixed find (fp_findpts_mixed_noalloc) against the
allocating mixed find (fp_findpts with FP_MIXED), through the C ABI.

Some callers cannot let a library allocate device memory (they reserve the
GPU's memory up front, or cannot afford an allocation's synchronisation or
failure mid-step); this entry point keeps its scratch in a fixed array
inside the library.  The test checks two calls in a row on different point
sets — the second must not see the first call's scratch contents — and
that a size above the fixed limit is refused before anything runs.  This
file is collected last and builds its own mesh, so it runs the same alone
or after the other tests.
"""
import numpy as np
import pytest

from paper_2501_12349_b300 import workloads as W
from parity_util import compare_find, to_np

pytestmark = pytest.mark.gpu


def _outputs(torch, n):
    dev = "cuda"
    return (torch.full((n,), 7, dtype=torch.int32, device=dev),
            torch.full((n,), -5, dtype=torch.int32, device=dev),
            torch.full((n, 3), float("nan"), dtype=torch.float64, device=dev),
            torch.full((n,), -1.0, dtype=torch.float64, device=dev))


def test_noalloc_matches_allocating_mixed_find():
    import torch

    import paper_2501_12349_b300 as fp

    w = W.hex_config(41, 300000, 1, n=16)
    mesh = fp.Mesh(torch.from_numpy(w.coords).cuda(), 3, 3, w.order)
    mesh.set_precision(fp.FP_MIXED)
    rng = np.random.default_rng(42)
    sets = [w.pts[:200000],
            np.concatenate([w.pts[200000:], rng.uniform(-0.2, 1.2, (50000, 3))])]
    for call, pts_np in enumerate(sets):
        pts = torch.from_numpy(np.ascontiguousarray(pts_np)).cuda()
        ref = tuple(to_np(t) for t in mesh.find(pts))  # the allocating entry point
        out = _outputs(torch, pts.shape[0])
        fp.fp_findpts_mixed_noalloc(mesh.handle, pts, *out)
        torch.cuda.synchronize()
        got = tuple(to_np(t) for t in out)
        compare_find(ref, got, label=f"no-alloc call {call}")
        assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
        assert (got[0] == 1).any() or call == 0  # the second set has BORDER points
    # beyond the fixed scratch size: refused, outputs untouched
    big = torch.zeros((fp.FP_NOALLOC_MAX_POINTS + 1, 3), dtype=torch.float64, device="cuda")
    out = _outputs(torch, big.shape[0])
    with pytest.raises(fp.FindptsError) as err:
        fp.fp_findpts_mixed_noalloc(mesh.handle, big, *out)
    assert err.value.status == fp.FP_EINVAL
    assert int((out[0] != 7).sum().item()) == 0
    assert mesh.device_status() == 0
    mesh.close()
