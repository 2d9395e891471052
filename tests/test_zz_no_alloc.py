"""The allocation-free mixed find (fp_findpts_mixed_noalloc) against the
allocating mixed find (fp_findpts with FP_MIXED), through the C ABI.

Some callers cannot let a library allocate device memory: solvers that
reserve the GPU's memory up front and run under a hard budget, and code
that must not meet an allocation's implicit synchronisation or its possible
failure in the middle of a time step.  This entry point keeps its scratch
in a fixed array inside the library.  The test checks two calls in a row on
different point sets (the second must not see the first call's scratch
contents), that device memory in use does not change across a call, that a
size above the fixed limit is refused before anything runs, and that
outputs too short for the points are refused by the binding.  This file is
collected last and builds its own mesh, so it runs the same alone or after
the other tests.
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


def _device_memory_in_use(torch):
    """(bytes the driver reports in use on the device, bytes in use in the
    device's default stream-ordered pool, bytes torch's allocator holds)."""
    from cuda.bindings import runtime as rt
    free, total = torch.cuda.mem_get_info()
    err, dev = rt.cudaGetDevice()
    assert err == rt.cudaError_t.cudaSuccess
    err, pool = rt.cudaDeviceGetDefaultMemPool(dev)
    assert err == rt.cudaError_t.cudaSuccess
    err, used = rt.cudaMemPoolGetAttribute(pool, rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemCurrent)
    assert err == rt.cudaError_t.cudaSuccess
    return total - free, int(used), torch.cuda.memory_allocated()


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
        torch.cuda.synchronize()
        before = _device_memory_in_use(torch)
        fp.fp_findpts_mixed_noalloc(mesh.handle, pts, *out)
        torch.cuda.synchronize()
        after = _device_memory_in_use(torch)
        if call > 0:  # the first call on the device may load the library's module
            assert after == before, (before, after)
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
    # outputs shorter than the points, or points of the wrong dimension:
    # refused by the binding before the library is called
    pts = torch.from_numpy(np.ascontiguousarray(w.pts[:1000])).cuda()
    code, elem, r, d2 = _outputs(torch, 1000)
    with pytest.raises(ValueError):
        fp.fp_findpts_mixed_noalloc(mesh.handle, pts, code, elem, r[:999], d2)
    with pytest.raises(ValueError):
        fp.fp_findpts_mixed_noalloc(mesh.handle, pts, code[:10], elem, r, d2)
    with pytest.raises(ValueError):
        fp.fp_findpts_mixed_noalloc(mesh.handle, pts[:, :2].contiguous(), code, elem, r, d2)
    assert int((code != 7).sum().item()) == 0
    assert mesh.device_status() == 0
    mesh.close()
