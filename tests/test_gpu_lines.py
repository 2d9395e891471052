"""Line elements in 2D and 3D (Sec. 2, Eq. x_tensor_surf; Sec. 4.2 Rodrigues
frame; Sec. 4.4 codes) on the GPU against the FP64 oracle: boxes, find in
FP64 and mixed precision, interpolation, and the closest-point projection
workload of the paper's tangential-relaxation example (boxes expanded by
100%)."""
import numpy as np
import pytest

import oracle
from paper_2501_12349_b300 import workloads as W
from parity_util import compare_eval, compare_find, to_np

pytestmark = pytest.mark.gpu

LINES = {
    "circle2d_p4": lambda: (W.circle_lines(40, 4), 2, 4),
    "star2d_p3": lambda: (W.star_lines(96, 3), 2, 3),
    "helix3d_p5": lambda: (W.helix_lines(48, 5), 3, 5),
    "segment3d_p2": lambda: (W.segment_lines(20, 2, (0.1, -0.2, 0.3), (0.9, 0.5, -0.4)), 3, 2),
    "circle2d_p7": lambda: (W.circle_lines(16, 7), 2, 7),
    "helix3d_p1": lambda: (W.helix_lines(64, 1), 3, 1),
}


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


def near_points(om, rng, n, sigma=0.003):
    """Points near the curve (forward map plus noise) and a few far away."""
    el = rng.integers(0, om.NE, n).astype(np.int32)
    x = om.forward_map(el, rng.uniform(-1, 1, (n, 1)))
    x = x + sigma * rng.standard_normal(x.shape)
    x[: n // 20] = rng.uniform(om.aabb[:, : om.d].min(0), om.aabb[:, om.d:].max(0), (n // 20, om.d))
    return x


@pytest.mark.parametrize("case", list(LINES))
def test_line_boxes(fp, torch, case):
    coords, d, order = LINES[case]()
    om = oracle.OracleMesh(coords, d, 1, order + 1)
    m = fp.Mesh(torch.from_numpy(coords).cuda(), d, 1, order)
    aabb, oc, oA = (to_np(t) for t in m.boxes())
    scale = np.abs(om.aabb).max(axis=1, keepdims=True)
    assert np.max(np.abs(aabb - om.aabb) / scale) < 1e-12
    assert np.max(np.abs(oc - om.obb_c) / scale) < 1e-12
    Ascale = np.abs(om.obb_A).reshape(om.NE, -1).max(axis=1)[:, None, None]
    # a nearly straight element has a thin OBB: its half-width across the
    # curve (the sagitta) is a small difference of O(h) bounds, so its
    # relative rounding error grows with the aspect ratio of the box
    rows = np.linalg.norm(om.obb_A, axis=2)
    aspect = (rows.max(axis=1) / rows.min(axis=1))[:, None, None]
    assert np.all(np.abs(oA - om.obb_A) / Ascale <= 1e-12 + 1e-13 * aspect)
    assert m.device_status() == 0
    m.close()


@pytest.mark.parametrize("precision", ["f64", "mixed"])
@pytest.mark.parametrize("case", list(LINES))
def test_line_find_eval(fp, torch, case, precision):
    coords, d, order = LINES[case]()
    N = order + 1
    om = oracle.OracleMesh(coords, d, 1, N)
    rng = np.random.default_rng(40)
    pts = near_points(om, rng, 20000)
    m = fp.Mesh(torch.from_numpy(coords).cuda(), d, 1, order)
    m.set_precision(fp.FP_MIXED if precision == "mixed" else fp.FP_F64)
    g = tuple(to_np(t) for t in m.find(torch.from_numpy(pts).cuda()))
    o = om.findpts(pts)
    res = compare_find(o, g, label=f"{precision} {case}", xscale=1.3)
    assert res["codes"][1] > 500
    fld, _ = W.polynomial_field(coords, rng, order, nc=2)
    oc, oe, orr = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in o[:3])
    u = to_np(m.eval(oc, oe, orr, torch.from_numpy(fld).cuda()))
    compare_eval(fld, om.NE, N, o[1], om.eval(fld, *o[:3]), u, case + " eval")
    assert m.device_status() == 0
    m.close()


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_closest_point_projection(fp, torch, precision):
    """The closest-point projection of the paper's tangential-relaxation
    example: boundary nodes of a curved 2D boundary moved along and off the
    curve; find with boxes expanded by 100%, then x(r*) by interpolating the
    coordinate field gives the closest points, which match the oracle's."""
    coords = W.star_lines(512, 3)
    om = oracle.OracleMesh(coords, 2, 1, 4, tol=1.0)
    pts = W.projection_points(coords, np.random.default_rng(41))
    m = fp.Mesh(torch.from_numpy(coords).cuda(), 2, 1, 3, bbox_tol=1.0)
    m.set_precision(fp.FP_MIXED if precision == "mixed" else fp.FP_F64)
    code, elem, r, d2 = m.find(torch.from_numpy(pts).cuda())
    g = tuple(to_np(t) for t in (code, elem, r, d2))
    o = om.findpts(pts)
    compare_find(o, g, label="projection " + precision, xscale=1.3)
    found = g[0] != 2
    assert found.mean() > 0.9
    xc = to_np(m.eval(code, elem, r, torch.from_numpy(coords).cuda()))  # [2][n] closest points
    xo = om.eval(coords, *o[:3])
    same = found & (g[1] == o[1])
    assert np.max(np.abs(xc[:, same] - xo[:, same])) < 1e-12
    # the moved node's distance to its projection is the reported distance
    # (the eval's rounding enters as 2 |dx| eps: in FP64 a few ulp of the
    # coordinates; in mixed precision the double-float contraction's bound,
    # 1e-13 of the nodal scale, about 1.2 here)
    d2 = np.sum((xc[:, found].T - pts[found]) ** 2, axis=1)
    eps = 1.3e-13 if precision == "mixed" else 5e-15
    assert np.all(np.abs(d2 - g[3][found]) <= 1e-9 * g[3][found] + 2 * eps * np.sqrt(g[3][found]) + 1e-28)
    m.close()
