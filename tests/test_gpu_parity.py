"""GPU (CUDA path, through the C ABI) against the FP64 oracle: boxes, Psi_L,
find and eval on every element shape and order, small cases in full and
the full-size 3D workload (10^6 points) in full."""
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


def gpu_mesh(fp, torch, coords, d, dr, order, **opts):
    return fp.Mesh(torch.from_numpy(np.ascontiguousarray(coords)).cuda(), d, dr, order, **opts)


def gpu_find(torch, mesh, pts):
    out = mesh.find(torch.from_numpy(np.ascontiguousarray(pts)).cuda())
    return tuple(to_np(t) for t in out)


def surface_points(om, rng, n, h, frac_off=0.1):
    elem = rng.integers(0, om.NE, n).astype(np.int32)
    rt = rng.uniform(-1.0, 1.0, (n, 2))
    x, J = om.forward_map(elem, rt, jacobian=True)
    nrm = np.cross(J[:, :, 0], J[:, :, 1])
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    off = rng.uniform(size=n) < frac_off
    x[off] += 0.01 * h * nrm[off]
    return x


CASES = {
    "quad2d_p3": lambda: (W.config1().coords, 2, 2, 3, 1.0 / 8),
    "hex3d_p4": lambda: (W.hex_mesh(6, 4, 0.3), 3, 3, 4, 1.0 / 6),
    "sphere_p4": lambda: (W.cubed_sphere(3, 4), 3, 2, 4, np.pi / 6),
    "torus_p3": lambda: (W.torus(12, 4, 3), 3, 2, 3, 2 * np.pi * 0.3 / 4),
}


@pytest.mark.parametrize("case", list(CASES))
def test_boxes_and_grid(fp, torch, case):
    coords, d, dr, order, h = CASES[case]()
    N = order + 1
    om = oracle.OracleMesh(coords, d, dr, N)
    m = gpu_mesh(fp, torch, coords, d, dr, order)
    aabb, oc, oA = (to_np(t) for t in m.boxes())
    scale = np.abs(om.aabb).max(axis=1, keepdims=True)
    assert np.max(np.abs(aabb - om.aabb) / scale) < 1e-12
    assert np.max(np.abs(oc - om.obb_c) / scale) < 1e-12
    Ascale = np.abs(om.obb_A).reshape(om.NE, -1).max(axis=1)[:, None, None]
    assert np.max(np.abs(oA - om.obb_A) / Ascale) < 1e-12
    # Psi_L: recomputed from the GPU's own boxes with the same rounded
    # formulas, it must match the GPU's CSR exactly (integer work).
    info = m.info()
    NL = info.n_grid
    assert NL ** d >= om.NE and (NL - 1) ** d < om.NE
    lo = np.array(info.grid_lo[:d])
    hi = np.array(info.grid_hi[:d])
    np.testing.assert_array_equal(lo, aabb[:, :d].min(0))
    np.testing.assert_array_equal(hi, aabb[:, d:].max(0))
    sc = np.where(hi > lo, NL / np.where(hi > lo, hi - lo, 1.0), 0.0)

    def cell(x, c):
        t = (x - lo[c]) * sc[c]
        return np.clip(np.where(t >= NL, NL - 1, np.floor(t)), 0, NL - 1).astype(np.int64)

    lists = [[] for _ in range(NL ** d)]
    for e in range(om.NE):
        c0 = [cell(aabb[e, c], c) for c in range(d)]
        c1 = [cell(aabb[e, d + c], c) for c in range(d)]
        rng3 = [range(c0[c], c1[c] + 1) for c in range(d)]
        if d == 2:
            for j in rng3[1]:
                for i in rng3[0]:
                    lists[i + NL * j].append(e)
        else:
            for k in rng3[2]:
                for j in rng3[1]:
                    for i in rng3[0]:
                        lists[i + NL * (j + NL * k)].append(e)
    cs, ce = (to_np(t) for t in m.grid())
    exp_start = np.concatenate([[0], np.cumsum([len(l) for l in lists])])
    np.testing.assert_array_equal(cs, exp_start)
    np.testing.assert_array_equal(ce, np.concatenate([np.array(l, np.int32) for l in lists]))
    assert m.device_status() == 0
    m.close()


def test_find_eval_config1_full(fp, torch):
    w = W.config1()
    om = oracle.OracleMesh(w.coords, 2, 2, w.N)
    pts = np.concatenate([om.forward_map(w.fwd_elem, w.fwd_r), w.pts])
    m = gpu_mesh(fp, torch, w.coords, 2, 2, w.order)
    g = gpu_find(torch, m, pts)
    o = om.findpts(pts)
    compare_find(o, g, label="config1")
    assert np.array_equal(g[1][:len(w.fwd_elem)], w.fwd_elem)
    assert np.max(np.abs(g[2][:len(w.fwd_elem)] - w.fwd_r)) < 1e-10
    code, elem, r = (torch.from_numpy(a).cuda() for a in g[:3])
    u = to_np(m.eval(code, elem, r, torch.from_numpy(w.field).cuda()))
    compare_eval(w.field, om.NE, w.N ** 2, o[1], om.eval(w.field, *o[:3]), u, "config1 eval")
    m.close()


@pytest.mark.parametrize("case", ["hex3d_p4", "sphere_p4", "torus_p3"])
def test_find_eval_small_full(fp, torch, case):
    coords, d, dr, order, h = CASES[case]()
    N = order + 1
    om = oracle.OracleMesh(coords, d, dr, N)
    rng = np.random.default_rng(11)
    if dr == 3:
        pts = rng.uniform(-0.02, 1.02, (20000, 3))
    else:
        pts = surface_points(om, rng, 20000, h)
    m = gpu_mesh(fp, torch, coords, d, dr, order)
    g = gpu_find(torch, m, pts)
    o = om.findpts(pts)
    res = compare_find(o, g, label=case)
    assert res["codes"][0] > 0
    fld, _ = W.polynomial_field(coords, rng, order, nc=3)
    code, elem, r = (torch.from_numpy(a).cuda() for a in g[:3])
    u = to_np(m.eval(code, elem, r, torch.from_numpy(fld).cuda()))
    compare_eval(fld, om.NE, N ** dr, o[1], om.eval(fld, *o[:3]), u, case + " eval")
    # coordinate-field invariant on the GPU alone: |u_x - x*|^2 = dist2
    ux = to_np(m.eval(code, elem, r, torch.from_numpy(coords).cuda()))
    found = g[0] != 2
    err = np.sum((ux[:, found].T - pts[found]) ** 2, axis=1)
    np.testing.assert_allclose(err, g[3][found], rtol=1e-9, atol=1e-22)
    assert m.device_status() == 0
    m.close()


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("shape", ["quad2d", "hex3d"])
def test_every_order(fp, torch, shape, order):
    rng = np.random.default_rng(100 + order)
    if shape == "quad2d":
        coords, d, dr = W.quad_mesh(5, order, amp=0.2, kind="kershaw"), 2, 2
    else:
        coords, d, dr = W.hex_mesh(3, order, 0.25), 3, 3
    om = oracle.OracleMesh(coords, d, dr, order + 1)
    pts = rng.uniform(-0.05, 1.05, (3000, d))
    m = gpu_mesh(fp, torch, coords, d, dr, order)
    compare_find(om.findpts(pts), gpu_find(torch, m, pts), label=f"{shape} p{order}")
    m.close()


@pytest.fixture(scope="module")
def config2_oracle():
    """The full 32^3, p=4 workload (10^6 points) and the oracle's find and
    eval of every point."""
    w = W.config2()
    om = oracle.OracleMesh(w.coords, 3, 3, w.N)
    o = om.findpts(w.pts)
    u = om.eval(w.field, *o[:3])
    return w, om, o, u


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_config2_full_size(fp, torch, config2_oracle, precision):
    """The full 32^3, p=4 workload in one call, as the benchmark runs it
    (cell order, persistent launch): every one of the 10^6 outputs against
    the oracle, find and eval, in the FP64 path and in the mixed path."""
    w, om, o, uo = config2_oracle
    m = gpu_mesh(fp, torch, w.coords, 3, 3, w.order)
    if precision == "mixed":
        m.set_precision(fp.FP_MIXED)
    pts_t = torch.from_numpy(w.pts).cuda()
    code, elem, r, dist2 = m.find(pts_t)
    u = m.eval(code, elem, r, torch.from_numpy(w.field).cuda())
    g = tuple(to_np(t) for t in (code, elem, r, dist2))
    res = compare_find(o, g, label=f"config2 {precision}")
    assert res["n"] == 10 ** 6 and min(res["codes"]) > 0
    # properties that do not rest on the oracle: the mesh covers the unit
    # cube exactly, so points inside it are INTERIOR, and NOT_FOUND only
    # happens outside
    inside = np.all((w.pts > 1e-9) & (w.pts < 1 - 1e-9), axis=1)
    assert np.all(g[0][inside] == 0) and np.all(~inside[g[0] == 2])
    compare_eval(w.field, om.NE, w.N ** 3, o[1], uo, to_np(u), f"config2 {precision} eval")
    assert m.device_status() == 0
    m.close()


def test_edge_cases(fp, torch):
    w = W.config1()
    m = gpu_mesh(fp, torch, w.coords, 2, 2, w.order)
    info = m.info()
    # n == 0 is a no-op
    e = torch.empty((0, 2), dtype=torch.float64, device="cuda")
    c, el, r, d2 = m.find(e)
    assert c.numel() == 0
    # non-finite points, points beyond the grid bounds, huge values, and
    # points clearly inside / outside the domain (points exactly on element
    # faces or box faces are left out: rounding of equal-valued quantities
    # decides them, and several answers are correct there)
    hi = info.grid_hi
    pts = np.array([[np.nan, 0.5], [0.5, np.inf], [-np.inf, 0.2], [hi[0] + 1e-9, 0.5],
                    [1e300, -1e300], [0.3, 0.7], [-0.05, 0.5], [1.05, 1.05]])
    om = oracle.OracleMesh(w.coords, 2, 2, w.N)
    g = gpu_find(torch, m, pts)
    compare_find(om.findpts(pts), g, label="edge")
    assert np.all(g[0][:5] == 2) and g[0][5] == 0 and np.all(g[0][6:] != 0)
    # a ragged size that is not a multiple of any block size
    rng = np.random.default_rng(3)
    p2 = rng.uniform(-0.2, 1.2, (1237, 2))
    compare_find(om.findpts(p2), gpu_find(torch, m, p2), label="ragged")
    assert m.device_status() == 0
    m.close()


@pytest.mark.parametrize("case", ["quad2d_p3", "hex3d_p4", "hex3d_p6_strong"])
def test_curvature_bound(fp, torch, case):
    """The per-element curvature bound behind the certified stops of the find
    kernels bounds the map's second derivatives, sum_jk |d2 x_c / dr_j dr_k|,
    at dense samples of the element (second derivatives from the oracle's
    Lagrange basis and its derivatives), and is no more than 30x above them."""
    if case == "hex3d_p6_strong":
        coords, d, dr, order = W.hex_mesh(4, 6, 0.6), 3, 3, 6
    else:
        coords, d, dr, order, _ = CASES[case]()
    N = order + 1
    m = gpu_mesh(fp, torch, coords, d, dr, order)
    L = to_np(m.curvature())
    X = np.asarray(coords).reshape(d, -1, N ** dr)
    rng = np.random.default_rng(5)
    els = rng.choice(X.shape[1], size=min(12, X.shape[1]), replace=False)
    tabs = [oracle.lagrange(N, r) for r in np.linspace(-1, 1, 9)]
    P, D1, D2 = (np.array([t[q] for t in tabs]) for q in range(3))  # [sample][basis]
    for e in els:
        worst = 0.0
        for c in range(d):
            if dr == 3:
                U = X[c, e].reshape(N, N, N)  # [k][j][i], i along r_0

                def sec(A0, A1, A2):
                    return np.abs(np.einsum("kji,ai,bj,gk->abg", U, A0, A1, A2))
                s = (sec(D2, P, P) + sec(P, D2, P) + sec(P, P, D2)
                     + 2 * (sec(D1, D1, P) + sec(D1, P, D1) + sec(P, D1, D1)))
            else:
                U = X[c, e].reshape(N, N)  # [j][i]

                def sec(A0, A1):
                    return np.abs(np.einsum("ji,ai,bj->ab", U, A0, A1))
                s = sec(D2, P) + sec(P, D2) + 2 * sec(D1, D1)
            worst = max(worst, float(s.max()))
        assert worst <= L[e], (case, e, worst, L[e])
        assert L[e] <= 30 * worst + 1e-12, (case, e, worst, L[e])
    m.close()


def test_stats_counters(fp, torch):
    w = W.hex_config(13, 5000, 1, n=6)
    om = oracle.OracleMesh(w.coords, 3, 3, w.N)
    m = gpu_mesh(fp, torch, w.coords, 3, 3, w.order)
    st = torch.zeros(fp.FP_NSTATS, dtype=torch.int64, device="cuda")
    m.find(torch.from_numpy(w.pts).cuda(), stats=st)
    gs = to_np(st)
    os_ = np.zeros(8, np.int64)
    om.findpts(w.pts, stats=os_)
    assert gs[0] == os_[0]                       # candidates: exact
    # iterations: the same algorithm, except that a certified stop (volumes)
    # ends an iteration one step before the sub-tolerance step the oracle
    # takes, so each one [4] accounts for exactly one oracle iteration
    assert gs[4] > 0.3 * gs[0]
    assert abs(gs[1] + gs[4] - os_[1]) <= 0.01 * os_[1]
    m.close()


@pytest.mark.parametrize("precision", ["f64", "mixed"])
@pytest.mark.parametrize("case", ["quad2d_p3", "hex3d_p4", "sphere_p4"])
def test_point_order_invariance(fp, torch, case, precision):
    """The cell-grouped traversal (the default, for calls of >= 16384 points)
    gives bit-identical outputs to the points taken as given, also for points
    outside the grid and with non-finite coordinates; and it agrees with the
    oracle."""
    coords, d, dr, order, h = CASES[case]()
    om = oracle.OracleMesh(coords, d, dr, order + 1)
    rng = np.random.default_rng(77)
    n = 40000
    if dr == d:
        pts = rng.uniform(-0.2, 1.2, (n, d))
    else:
        pts = surface_points(om, rng, n, h)
        pts[: n // 50] = rng.uniform(-2, 2, (n // 50, d))
    pts[5] = np.nan
    pts[17, 0] = np.inf
    m = gpu_mesh(fp, torch, coords, d, dr, order)
    m.set_precision(fp.FP_MIXED if precision == "mixed" else fp.FP_F64)
    tp = torch.from_numpy(pts).cuda()
    a = tuple(to_np(t) for t in m.find(tp))
    m.set_point_order(fp.FP_ORDER_GIVEN)
    b = tuple(to_np(t) for t in m.find(tp))
    for x, y in zip(a, b):
        assert np.array_equal(x, y, equal_nan=True)
    assert a[0][5] == 2 and a[0][17] == 2
    compare_find(om.findpts(pts), a, label=f"ordered {precision} {case}", xscale=1.3)
    assert m.device_status() == 0
    m.close()


@pytest.mark.parametrize("case,field_order", [("hex3d_p4", 2), ("hex3d_p4", 7), ("quad2d_p3", 5),
                                              ("sphere_p4", 1), ("torus_p3", 6)])
def test_eval_field_order(fp, torch, case, field_order):
    """fp_eval_order (a field of another order than the mesh, Sec. 2 after
    Eq. u_tensor) against the oracle's interpolation at the oracle's find
    output, 3 components; random nodal values."""
    coords, d, dr, order, h = CASES[case]()
    N = order + 1
    Nf = field_order + 1
    om = oracle.OracleMesh(coords, d, dr, N)
    rng = np.random.default_rng(13)
    if dr == d:
        pts = rng.uniform(-0.05, 1.05, (20000, d))
    else:
        pts = surface_points(om, rng, 20000, h)
    m = gpu_mesh(fp, torch, coords, d, dr, order)
    g = gpu_find(torch, m, pts)
    o = om.findpts(pts)
    compare_find(o, g, label=case)
    fld = rng.uniform(-1, 1, (3, om.NE * Nf ** dr))
    # the oracle's find output as input: random nodal values make the field
    # discontinuous across elements, so tied BORDER answers would differ
    code, elem, r = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in o[:3])
    u = to_np(m.eval(code, elem, r, torch.from_numpy(fld).cuda(), order=field_order))
    uo = om.eval(fld, *o[:3], field_N=Nf)
    compare_eval(fld, om.NE, Nf ** dr, o[1], uo, u, f"{case} field order {field_order}")
    assert m.device_status() == 0
    m.close()


def test_many_fields_one_find(fp, torch):
    """Several fields evaluated from one find output (Sec. 3.3: Find once,
    interpolate every field): one call per field equals one call with all
    fields as components, bit for bit, and matches the oracle."""
    coords, d, dr, order, h = CASES["hex3d_p4"]()
    om = oracle.OracleMesh(coords, d, dr, order + 1)
    rng = np.random.default_rng(14)
    pts = rng.uniform(0, 1, (30000, 3))
    m = gpu_mesh(fp, torch, coords, d, dr, order)
    code, elem, r, d2 = m.find(torch.from_numpy(pts).cuda())
    fields = [rng.uniform(-1, 1, (1, om.NE * (order + 1) ** 3)) for _ in range(4)]
    sep = [to_np(m.eval(code, elem, r, torch.from_numpy(f).cuda())) for f in fields]
    allf = to_np(m.eval(code, elem, r, torch.from_numpy(np.concatenate(fields)).cuda()))
    assert np.array_equal(np.concatenate(sep), allf)
    o = om.findpts(pts)
    oc, oe, orr = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in o[:3])
    uo = to_np(m.eval(oc, oe, orr, torch.from_numpy(np.concatenate(fields)).cuda()))
    compare_eval(np.concatenate(fields), om.NE, (order + 1) ** 3, o[1], om.eval(np.concatenate(fields), *o[:3]),
                 uo, "many fields")
    m.close()


def test_distributed_find_single_rank_nccl(fp, torch):
    """The multi-rank Find (Psi_G, Sec. 3.1.4; Sec. 3.2) on CUDA tensors over
    NCCL with one rank, the library's find as the local search: identical to
    the plain find (the routing moves nothing, and the device path of every
    exchange and of the merge runs)."""
    import socket
    import torch.distributed as dist
    from paper_2501_12349_b300 import distributed as Dm
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("nccl", rank=0, world_size=1, init_method=f"tcp://127.0.0.1:{port}")
    try:
        coords, d, dr, order, h = CASES["hex3d_p4"]()
        m = gpu_mesh(fp, torch, coords, d, dr, order)
        aabb, _, _ = m.boxes()
        gmap = Dm.GlobalMap.build(aabb, d)
        pts = torch.from_numpy(np.random.default_rng(15).uniform(-0.1, 1.1, (20000, 3))).cuda()
        code, rank, elem, r, d2 = Dm.find(m.find, pts, gmap)
        ref = m.find(pts)
        assert torch.equal(code, ref[0]) and torch.equal(elem, ref[1])
        assert torch.equal(r, ref[2]) and torch.equal(d2, ref[3])
        assert torch.all(rank[code != 2] == 0) and torch.all(rank[code == 2] == -1)
        m.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("precision", ["f64", "mixed"])
@pytest.mark.parametrize("variant", ["offset_scaled", "strong_deformation", "single_element"])
def test_robustness_cases(fp, torch, variant, precision):
    """Meshes far from the origin and scaled (the FP32 prefilters work on
    coordinates relative to each element, so they must keep their rounding
    margins there), strongly deformed elements (ill-conditioned Jacobians,
    which the mixed path hands to FP64), and a one-element mesh; points at
    interior GLL nodes (the closest-node start is the answer) included."""
    rng = np.random.default_rng(16)
    if variant == "offset_scaled":
        coords = W.hex_mesh(5, 4, 0.3) * 3.7 + np.array([1000.0, -2000.0, 500.0])[:, None, None]
        lo, hi = np.array([1000.0, -2000.0, 500.0]) - 0.1, np.array([1000.0, -2000.0, 500.0]) + 3.8
    elif variant == "strong_deformation":
        coords = W.hex_mesh(5, 4, 0.45)  # diagonally dominant Jacobian: still bijective
        lo, hi = np.full(3, -0.05), np.full(3, 1.05)
    else:
        coords = W.hex_mesh(1, 5, 0.3)
        lo, hi = np.full(3, -0.1), np.full(3, 1.1)
    order = int(round(coords.shape[2] ** (1 / 3))) - 1
    N = order + 1
    om = oracle.OracleMesh(coords, 3, 3, N)
    pts = rng.uniform(lo, hi, (15000, 3))
    z = W.gll_points(N)[1:-1]
    el = rng.integers(0, om.NE, 500).astype(np.int32)
    rn = z[rng.integers(0, z.size, (500, 3))]
    pts = np.concatenate([pts, om.forward_map(el, rn)])
    m = gpu_mesh(fp, torch, coords, 3, 3, order)
    m.set_precision(fp.FP_MIXED if precision == "mixed" else fp.FP_F64)
    g = gpu_find(torch, m, pts)
    o = om.findpts(pts)
    xs = float(np.abs(coords).max())
    compare_find(o, g, label=f"{variant} {precision}", xscale=1.3 * xs)
    assert np.all(g[0][-500:] == 0)
    np.testing.assert_allclose(g[2][-500:], rn, atol=1e-10)
    assert m.device_status() == 0
    m.close()


def _random_case(seed):
    rng = np.random.default_rng(1000 + seed)
    kind = ["quad2d", "hex3d", "sphere", "torus", "circle", "helix"][seed % 6]
    order = int(rng.integers(1, 8))
    if kind == "quad2d":
        n = int(rng.integers(2, 9))
        return W.quad_mesh(n, order, amp=float(rng.uniform(0, 0.3)), kind="kershaw"), 2, 2, order, 1.0 / n
    if kind == "hex3d":
        n = int(rng.integers(1, 5))
        return W.hex_mesh(n, order, float(rng.uniform(0, 0.4))), 3, 3, order, 1.0 / n
    if kind == "sphere":
        n = int(rng.integers(1, 4))
        return W.cubed_sphere(n, order), 3, 2, order, np.pi / (2 * n)
    if kind == "torus":
        nu, nv = int(rng.integers(3, 12)), int(rng.integers(3, 8))
        return W.torus(nu, nv, order), 3, 2, order, 2 * np.pi * 0.3 / nv
    if kind == "circle":
        n = int(rng.integers(3, 40))
        return W.circle_lines(n, order), 2, 1, order, 2 * np.pi / n
    n = int(rng.integers(4, 40))
    return W.helix_lines(n, order), 3, 1, order, 1.0 / n


@pytest.mark.parametrize("precision", ["f64", "mixed"])
@pytest.mark.parametrize("seed", range(12))
def test_randomized_parity(fp, torch, seed, precision):
    """Seeded random meshes (shape, order 1-7, element count, deformation)
    and points inside, near and outside them: code and element exact, r,
    dist2 and interpolated values within the FP64 tolerances."""
    coords, d, dr, order, h = _random_case(seed)
    N = order + 1
    om = oracle.OracleMesh(coords, d, dr, N)
    rng = np.random.default_rng(2000 + seed)
    n = 6000
    el = rng.integers(0, om.NE, n).astype(np.int32)
    x = om.forward_map(el, rng.uniform(-1, 1, (n, dr)))
    x[: n // 3] += (0.05 * h) * rng.standard_normal((n // 3, d))
    lo, hi = om.aabb[:, :d].min(0), om.aabb[:, d:].max(0)
    x[n // 3: n // 2] = rng.uniform(lo - 0.05 * (hi - lo), hi + 0.05 * (hi - lo), (n // 2 - n // 3, d))
    m = gpu_mesh(fp, torch, coords, d, dr, order)
    m.set_precision(fp.FP_MIXED if precision == "mixed" else fp.FP_F64)
    g = gpu_find(torch, m, x)
    o = om.findpts(x)
    compare_find(o, g, label=f"random {seed} {precision}", xscale=1.3 * float(np.abs(coords).max()), om=om, pts=x)
    fld, _ = W.polynomial_field(coords, rng, min(order, 3), nc=1)
    oc, oe, orr = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in o[:3])
    u = to_np(m.eval(oc, oe, orr, torch.from_numpy(fld).cuda()))
    compare_eval(fld, om.NE, N ** dr, o[1], om.eval(fld, *o[:3]), u, f"random {seed} eval")
    assert m.device_status() == 0
    m.close()


@pytest.mark.parametrize("chunk", [0, 1000, 7919, 10 ** 9])
@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_findpts_host(fp, torch, chunk, precision):
    """fp_findpts_host (host buffers, chunked copies overlapping the search)
    gives the device path's outputs bit for bit, with and without a field."""
    coords, d, dr, order, h = CASES["hex3d_p4"]()
    rng = np.random.default_rng(17)
    pts = rng.uniform(-0.05, 1.05, (30000, 3))
    m = gpu_mesh(fp, torch, coords, d, dr, order)
    m.set_precision(fp.FP_MIXED if precision == "mixed" else fp.FP_F64)
    fld = torch.from_numpy(rng.uniform(-1, 1, (2, m.NE * (order + 1) ** 3))).cuda()
    ref = m.find(torch.from_numpy(pts).cuda())
    uref = m.eval(*ref[:3], fld)
    hp = torch.from_numpy(pts).pin_memory()
    got = m.find_host(hp, fld, chunk=chunk)
    for a, b in zip(list(ref) + [uref], got):
        assert torch.equal(a.cpu(), b)
    got2 = m.find_host(hp, None, chunk=chunk)
    for a, b in zip(ref, got2):
        assert torch.equal(a.cpu(), b)
    m.close()


@pytest.mark.parametrize("precision", ["f64", "mixed"])
@pytest.mark.parametrize("case", list(CASES) + ["circle_p3", "helix_p5"])
def test_points_at_interior_nodes(fp, torch, case, precision):
    """Points placed at interior GLL nodes of random elements, where the
    start at the closest node (x the node itself, G from the
    differentiation matrix) is already the answer: INTERIOR in that element
    at r = the node, for quads, hexes, surface quads and lines, and equal to
    the oracle."""
    if case == "circle_p3":
        coords, d, dr, order = W.circle_lines(64, 3), 2, 1, 3
    elif case == "helix_p5":
        coords, d, dr, order = W.helix_lines(48, 5), 3, 1, 5
    else:
        coords, d, dr, order, _ = CASES[case]()
    N = order + 1
    om = oracle.OracleMesh(coords, d, dr, N)
    rng = np.random.default_rng(31)
    z = W.gll_points(N)[1:-1]
    el = rng.integers(0, om.NE, 3000).astype(np.int32)
    rn = z[rng.integers(0, z.size, (3000, dr))]
    pts = om.forward_map(el, rn)
    m = gpu_mesh(fp, torch, coords, d, dr, order)
    m.set_precision(fp.FP_MIXED if precision == "mixed" else fp.FP_F64)
    g = gpu_find(torch, m, pts)
    o = om.findpts(pts)
    compare_find(o, g, label=f"nodes {case} {precision}", xscale=1.3 * float(np.abs(coords).max()))
    assert np.all(g[0] == 0), f"{case}: {np.bincount(g[0], minlength=3)}"
    assert np.array_equal(g[1], el)  # an interior node lies in no other element
    np.testing.assert_allclose(g[2], rn, atol=1e-10)
    assert m.device_status() == 0
    m.close()


def test_kernel_times(fp, torch):
    """fp_set_timing / fp_kernel_times: per-stage CUDA-event intervals of the
    timed calls only (cell order, find kernel, FP64 follow-up, eval), read
    once and then started afresh."""
    w = W.hex_config(14, 40000, 1, n=6)
    m = gpu_mesh(fp, torch, w.coords, 3, 3, w.order)
    pts = torch.from_numpy(w.pts).cuda()
    fld = torch.from_numpy(w.field).cuda()
    m.find(pts)  # not timed
    fp.fp_set_timing(m.handle, True)
    for prec in (fp.FP_F64, fp.FP_MIXED):
        m.set_precision(prec)
        c, e, r, d2 = m.find(pts)
        m.eval(c, e, r, fld)
    fp.fp_set_timing(m.handle, False)
    m.find(pts)  # not timed
    ms, calls = fp.fp_kernel_times(m.handle)
    assert calls == [2, 2, 1, 2], calls
    assert all(v > 0 for v in ms), ms
    ms2, calls2 = fp.fp_kernel_times(m.handle)
    assert calls2 == [0, 0, 0, 0] and ms2 == [0.0] * 4
    info = m.info()
    assert info.setup_boxes_ms > 0 and info.setup_grid_ms > 0
    m.close()
