"""Many meshes in one graph launch (fp_batch_*): every item's result matches
the single-mesh call (same element and code, r and dist2 within the FP64
tolerance: the batch and single-mesh kernels are separate instantiations
of the same code, whose floating-point contractions may differ), parity
with the oracle on a capped version of the 64-mesh workload, eval in the
batch, autotuning."""
import numpy as np
import pytest

import oracle
from paper_2501_12349_b300 import workloads as W
from parity_util import compare_eval, compare_find, to_np

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


def workload_points(w, om):
    """Physical points of a config-4 mesh: volume points as drawn; surface
    points from the oracle's forward map of the (elem, r) pairs, displaced
    along the normal where the generator asks for it."""
    if w.fwd_elem is None:
        return w.pts
    x, J = om.forward_map(w.fwd_elem, w.fwd_r, jacobian=True)
    nrm = np.cross(J[:, :, 0], J[:, :, 1])
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    return x + w.fwd_offset[:, None] * nrm


@pytest.fixture(scope="module")
def config4_small(fp, torch):
    ws = W.config4(max_points=3000, max_elems=1500)
    meshes, pts, oms = [], [], []
    for w in ws:
        om = oracle.OracleMesh(w.coords, w.d, w.dr, w.N)
        p = workload_points(w, om)
        oms.append(om)
        pts.append(p)
        meshes.append(fp.Mesh(torch.from_numpy(w.coords).cuda(), w.d, w.dr, w.order))
    yield ws, meshes, pts, oms
    for m in meshes:
        m.close()


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_batch_equals_single_and_oracle(fp, torch, config4_small, precision):
    ws, meshes, pts, oms = config4_small
    prec = fp.FP_MIXED if precision == "mixed" else fp.FP_F64
    entries = [(m, torch.from_numpy(p).cuda(), torch.from_numpy(w.field).cuda())
               for m, p, w in zip(meshes, pts, ws)]
    b = fp.Batch(entries, prec)
    assert len(b.classes()) >= 6
    b.run()
    torch.cuda.synchronize()
    for (m, pt, fld), outs, w, om, p in zip(entries, b.outputs, ws, oms, pts):
        m.set_precision(prec)
        single = tuple(to_np(t) for t in m.find(pt))
        got = tuple(to_np(t) for t in outs[:4])
        compare_find(single, got, label=f"batch vs single {precision} {w.name}", xscale=1.3)
        assert np.array_equal(single[0], got[0]) and np.array_equal(single[1], got[1]), w.name
        o = om.findpts(p)
        compare_find(o, got, label=f"{precision} {w.name}", xscale=1.3)
        u = to_np(outs[4])
        compare_eval(w.field, om.NE, w.N ** w.dr, o[1], om.eval(w.field, *o[:3]), u, w.name + " eval")
        assert m.device_status() == 0
        m.set_precision(fp.FP_F64)
    # the fused form (one persistent find launch over every shape): the same
    # elements and codes, r and dist2 within the tolerance (another
    # compilation of the same loops, whose contractions may differ), and the
    # same interpolated values to the eval tolerance
    check_fused_same(fp, torch, b, ws)
    b.close()


def check_fused_same(fp, torch, b, ws, sels=None):
    first = [[to_np(t) for t in o] for o in b.outputs]
    b.set_fused(True)
    for o in b.outputs:
        o[0].fill_(7)
    b.run()
    torch.cuda.synchronize()
    for i, (f, o) in enumerate(zip(first, b.outputs)):
        g = [to_np(t) for t in o]
        sel = slice(None) if sels is None else sels[i]
        a = tuple(x[sel] for x in f[:4])
        c = tuple(x[sel] for x in g[:4])
        compare_find(a, c, label=f"fused {ws[i].name}", xscale=1.3)
        assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])
        if f[4] is not None:
            compare_eval(ws[i].field, ws[i].NE, ws[i].N ** ws[i].dr, a[1], f[4][..., sel], g[4][..., sel],
                         f"fused eval {ws[i].name}")
    b.set_fused(False)


def test_batch_autotune_and_rerun(fp, torch, config4_small):
    ws, meshes, pts, oms = config4_small
    entries = [(m, torch.from_numpy(p).cuda(), None) for m, p in zip(meshes[:16], pts[:16])]
    b = fp.Batch(entries, fp.FP_MIXED)
    b.run()
    torch.cuda.synchronize()
    first = [tuple(t.clone() for t in o[:4]) for o in b.outputs]
    b.autotune()
    infos = b.classes()
    assert all(i.tuned_ms > 0 and 1 <= i.ctas_per_sm <= 4 and i.chunk_points in (32, 128, 512) for i in infos)
    for o in b.outputs:  # the autotuner overwrote the outputs: clear them
        o[0].fill_(7)
    b.run()
    torch.cuda.synchronize()
    for f, o in zip(first, b.outputs):
        for a, s in zip(f, o[:4]):
            assert torch.equal(a, s)
    # a second plan of the same shapes picks up the tuned launch shapes
    b2 = fp.Batch(entries, fp.FP_MIXED)
    assert [(i.ctas_per_sm, i.chunk_points) for i in b2.classes()] == [(i.ctas_per_sm, i.chunk_points) for i in infos]
    b.close()
    b2.close()


def test_batch_rejects_bad_items(fp, torch, config4_small):
    ws, meshes, pts, oms = config4_small
    p = torch.from_numpy(pts[0]).cuda()
    bad = fp.FpBatchItem(5, p.data_ptr(), p.shape[0], 0, 0, 0, 0, None, 0, None)
    with pytest.raises(fp.FindptsError):
        fp.fp_batch_create([meshes[0].handle], [bad])


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_batch_cell_order_invariance(fp, torch, config4_small, precision):
    """The cell-grouped order of a batch's points leaves every output bit for
    bit unchanged (plans over meshes set to FP_ORDER_GIVEN take the points
    as given)."""
    ws, meshes, pts, oms = config4_small
    prec = fp.FP_MIXED if precision == "mixed" else fp.FP_F64
    entries = [(m, torch.from_numpy(p).cuda(), torch.from_numpy(w.field).cuda())
               for m, p, w in zip(meshes, pts, ws)]
    outs = []
    for order in (fp.FP_ORDER_CELL, fp.FP_ORDER_GIVEN):
        for m in meshes:
            m.set_point_order(order)
        b = fp.Batch(entries, prec)
        b.run()
        torch.cuda.synchronize()
        outs.append([[t.clone() for t in o] for o in b.outputs])
        b.close()
    for m in meshes:
        m.set_point_order(fp.FP_ORDER_CELL)
    for a, b in zip(*outs):
        for x, y in zip(a, b):
            assert torch.equal(x, y)


def workload_points_dev(fp, torch, mesh, w):
    """As workload_points, with x_e(r) from the library's interpolation of
    the coordinate field and the analytic surface normal (the benchmark's
    recipe), on the device."""
    if w.fwd_elem is None:
        return torch.from_numpy(w.pts).cuda()
    n = len(w.fwd_elem)
    x = mesh.eval(torch.zeros(n, dtype=torch.int32, device="cuda"), torch.from_numpy(w.fwd_elem).cuda(),
                  torch.from_numpy(np.ascontiguousarray(w.fwd_r)).cuda(), torch.from_numpy(w.coords).cuda()).T
    if "sphere" in w.name:
        nrm = x / x.norm(dim=1, keepdim=True)
    else:
        ring = x.clone()
        ring[:, 2] = 0.0
        ring = ring / ring.norm(dim=1, keepdim=True)
        nrm = (x - ring) / (x - ring).norm(dim=1, keepdim=True)
    return (x + torch.from_numpy(w.fwd_offset).cuda()[:, None] * nrm).contiguous()


def test_batch_full_size_sampled(fp, torch):
    """The full 64-mesh workload (7.3 million points over 645k elements) in the
    launch configuration the benchmark times (one autotuned graph, FP64 and
    mixed, surface points as the benchmark draws them): on every mesh, 2,000
    points spread over its point set match the oracle (code and element
    exactly, r and dist2 to the FP64 tolerance, the interpolated field
    relative to the field's scale); the fused form gives the same elements
    and codes on all points, r, dist2 and values within the tolerances."""
    ws = W.config4()
    meshes = [fp.Mesh(torch.from_numpy(w.coords).cuda(), w.d, w.dr, w.order) for w in ws]
    entries = [(m, workload_points_dev(fp, torch, m, w), torch.from_numpy(w.field).cuda())
               for m, w in zip(meshes, ws)]
    sels = [np.linspace(0, e[1].shape[0] - 1, 2000).astype(np.int64) for e in entries]
    ref = []
    for (m, pt, fld), w, sel in zip(entries, ws, sels):
        om = oracle.OracleMesh(w.coords, w.d, w.dr, w.N)
        p = to_np(pt)[sel]
        o = om.findpts(p)
        ref.append((om, p, o, om.eval(w.field, *o[:3])))
    for prec in (fp.FP_F64, fp.FP_MIXED):
        b = fp.Batch(entries, prec)
        b.autotune()
        b.run()
        torch.cuda.synchronize()
        for i, w in enumerate(ws):
            om, p, o, uo = ref[i]
            got = tuple(to_np(t)[sels[i]] for t in b.outputs[i][:4])
            compare_find(o, got, label=f"full batch {prec} {w.name}", xscale=1.3, om=om, pts=p)
            u = to_np(b.outputs[i][4])[..., sels[i]]
            compare_eval(w.field, om.NE, w.N ** w.dr, o[1], uo, u, w.name + " eval")
        check_fused_same(fp, torch, b, ws)
        b.close()
    for m in meshes:
        assert m.device_status() == 0
        m.close()
