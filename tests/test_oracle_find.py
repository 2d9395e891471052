"""Pins of the oracle's boxes, Newton, candidate selection and interpolation
(Secs. 3.1-3.3, 4) against closed forms, invariants and brute force."""
import numpy as np
import pytest
from numpy.polynomial import legendre as L

import oracle
from paper_2501_12349_b300 import workloads as W


def numpy_forward(coords, d, dr, N, e, r):
    """Independent evaluation of x_e(r) (Eq. x_tensor) with numpy Legendre fits."""
    z = W.gll_points(N)
    ne = N ** dr
    B = []
    for j in range(dr):
        vals = np.stack([L.legval(r[j], L.legfit(z, np.eye(N)[i], N - 1)) for i in range(N)])
        B.append(vals)
    idx = np.arange(ne)
    w = np.ones(ne)
    for j in range(dr):
        w = w * B[j][(idx // N ** j) % N]
    return np.array([coords[c, e] @ w for c in range(d)])


def affine_hex_mesh(seed=0, n=2, order=3):
    rng = np.random.default_rng(seed)
    X = np.stack(W._tensor_nodes((n, n, n), order + 1))  # [3][NE][ne]
    A = np.eye(3) + 0.3 * rng.uniform(-1, 1, (3, 3))
    b = rng.uniform(-1, 1, 3)
    return np.ascontiguousarray(np.einsum("ij,jen->ien", A, X) + b[:, None, None]), A, b


MESHES = {
    "quad2d": lambda: (W.config1().coords, 2, 2, 4),
    "hex3d": lambda: (W.hex_mesh(3, 4, 0.3), 3, 3, 5),
    "sphere": lambda: (W.cubed_sphere(2, 4), 3, 2, 5),
    "torus": lambda: (W.torus(9, 3, 3), 3, 2, 4),
}


@pytest.fixture(scope="module", params=list(MESHES))
def mesh(request):
    coords, d, dr, N = MESHES[request.param]()
    return request.param, oracle.OracleMesh(coords, d, dr, N)


def test_forward_map_matches_numpy(mesh):
    name, m = mesh
    rng = np.random.default_rng(1)
    for _ in range(5):
        e = int(rng.integers(0, m.NE))
        r = rng.uniform(-1, 1, m.dr)
        x = m.forward_map(np.array([e], np.int32), r[None])[0]
        np.testing.assert_allclose(x, numpy_forward(m.coords, m.d, m.dr, m.N, e, r), atol=1e-13)


def _dense_r(dr, k=7, nrand=60, seed=0):
    g = np.linspace(-1, 1, k)
    grid = np.stack(np.meshgrid(*([g] * dr), indexing="ij"), -1).reshape(-1, dr)
    rnd = np.random.default_rng(seed).uniform(-1, 1, (nrand, dr))
    return np.concatenate([grid, rnd])


def test_boxes_contain_element(mesh):
    """Dense samples of x_e(r), r in [-1,1]^dr, lie in the expanded AABB and
    OBB of element e (Secs. 3.1.1, 3.1.2, 4.1, 4.2)."""
    name, m = mesh
    R = _dense_r(m.dr)
    for e in range(m.NE):
        x = m.forward_map(np.full(len(R), e, np.int32), R)
        lo, hi = m.aabb[e, :m.d], m.aabb[e, m.d:]
        assert np.all(x >= lo - 1e-14) and np.all(x <= hi + 1e-14), (name, e)
        v = (x - m.obb_c[e]) @ m.obb_A[e].T
        assert np.max(np.abs(v)) <= 1.0 + 1e-12, (name, e, np.max(np.abs(v)))


def test_boxes_affine_closed_form():
    """For a parallelepiped the AABB is the corner hull grown by tol*L/2 per
    side and the OBB is the element itself grown by (1+tol): its corners
    satisfy |A (x - c)|_inf = 1/(1+tol) and c = x(0)."""
    coords, A, b = affine_hex_mesh()
    tol = 0.1
    m = oracle.OracleMesh(coords, 3, 3, 4, tol=tol)
    corners = np.array([[i, j, k] for i in (-1, 1) for j in (-1, 1) for k in (-1, 1)], float)
    for e in range(m.NE):
        xc = m.forward_map(np.full(8, e, np.int32), corners)
        lo, hi = xc.min(0), xc.max(0)
        Lx = hi - lo
        np.testing.assert_allclose(m.aabb[e, :3], lo - 0.5 * tol * Lx, atol=1e-13)
        np.testing.assert_allclose(m.aabb[e, 3:], hi + 0.5 * tol * Lx, atol=1e-13)
        np.testing.assert_allclose(m.obb_c[e], m.forward_map(np.array([e], np.int32), np.zeros((1, 3)))[0], atol=1e-13)
        v = (xc - m.obb_c[e]) @ m.obb_A[e].T
        np.testing.assert_allclose(np.abs(v), 1.0 / (1.0 + tol), atol=1e-12)


def test_newton_affine_closed_form():
    coords, A, b = affine_hex_mesh(seed=3)
    m = oracle.OracleMesh(coords, 3, 3, 4)
    rng = np.random.default_rng(4)
    for e in range(m.NE):
        r_true = rng.uniform(-0.99, 0.99, (20, 3))
        x = m.forward_map(np.full(20, e, np.int32), r_true)
        x0 = m.forward_map(np.array([e], np.int32), np.zeros((1, 3)))[0]
        J = m.forward_map(np.array([e], np.int32), np.zeros((1, 3)), jacobian=True)[1][0]
        for p in range(20):
            r, dist2, it = m.newton(e, x[p])
            np.testing.assert_allclose(r, np.linalg.solve(J, x[p] - x0), atol=1e-13)
            assert dist2 < 1e-26 and it <= 3


def test_newton_forward_map_recovery(mesh):
    """Points x_e(r) with known (e, r), r in [-0.95,0.95]^dr, are recovered
    to 1e-12 in r with dist2 ~ 0 (Sec. 3.2.1)."""
    name, m = mesh
    rng = np.random.default_rng(5)
    n = 300
    elem = rng.integers(0, m.NE, n).astype(np.int32)
    r_true = rng.uniform(-0.95, 0.95, (n, m.dr))
    x = m.forward_map(elem, r_true)
    iters = []
    for p in range(n):
        r, dist2, it = m.newton(elem[p], x[p])
        assert np.max(np.abs(r - r_true[p])) < 1e-12, (name, p, r, r_true[p])
        assert dist2 < 1e-24
        iters.append(it)
    assert np.mean(iters) < 8


def _gradient(m, e, r, xs):
    x, J = m.forward_map(np.array([e], np.int32), r[None], jacobian=True)
    dx = xs - x[0]
    return -(J[0].T @ dx), float(dx @ dx)


@pytest.mark.parametrize("name", ["quad2d", "hex3d"])
def test_newton_border_kkt_and_brute_force(name):
    """Points outside an element but near it: Newton ends on the boundary at a
    KKT point of min |x* - x(r)|^2 over the box (Sec. 3.2.1, closest point),
    and no dense boundary sample is closer."""
    coords, d, dr, N = MESHES[name]()
    m = oracle.OracleMesh(coords, d, dr, N)
    rng = np.random.default_rng(6)
    e = m.NE // 2
    lo, hi = m.aabb[e, :d], m.aabb[e, d:]
    g1 = np.linspace(-1, 1, 401)
    if dr == 2:
        S = np.stack(np.meshgrid(g1, g1, indexing="ij"), -1).reshape(-1, 2)
    else:
        g2 = np.linspace(-1, 1, 61)
        faces = []
        for fixed in range(3):
            for val in (-1.0, 1.0):
                a, b = np.meshgrid(g2, g2, indexing="ij")
                f = np.zeros((a.size, 3))
                others = [k for k in range(3) if k != fixed]
                f[:, fixed] = val
                f[:, others[0]] = a.ravel()
                f[:, others[1]] = b.ravel()
                faces.append(f)
        S = np.concatenate(faces)
    XS = m.forward_map(np.full(len(S), e, np.int32), S)
    tested = 0
    while tested < 20:
        xs = rng.uniform(lo, hi)
        code, rr, dd = m.locate_in_element(e, xs[None])
        if code[0] == 0:
            continue
        tested += 1
        r = rr[0]
        assert np.any(np.abs(r) == 1.0)
        g, F = _gradient(m, e, r, xs)
        scale = np.linalg.norm(g) + np.sqrt(F) * 1e-3
        for j in range(dr):
            if r[j] == 1.0:
                assert g[j] <= 1e-9 * scale
            elif r[j] == -1.0:
                assert g[j] >= -1e-9 * scale
            else:
                assert abs(g[j]) <= 1e-7 * max(scale, 1e-300) + 1e-14
        best = np.min(np.sum((XS - xs) ** 2, axis=1))
        assert dd[0] <= best * (1 + 1e-9) + 1e-15


def _np_in_boxes(m, e, pts):
    lo, hi = m.aabb[e, :m.d], m.aabb[e, m.d:]
    ok = np.all((pts >= lo) & (pts <= hi), axis=1)
    v = (pts - m.obb_c[e]) @ m.obb_A[e].T
    return ok & np.all(np.abs(v) <= 1.0, axis=1)


@pytest.fixture(scope="module")
def config1_oracle():
    w = W.config1()
    m = oracle.OracleMesh(w.coords, 2, 2, w.N)
    x = m.forward_map(w.fwd_elem, w.fwd_r)
    pts = np.concatenate([x, w.pts])
    return w, m, pts


def test_find_config1_forward_points(config1_oracle):
    w, m, pts = config1_oracle
    code, elem, r, dist2 = m.findpts(pts)
    nf = len(w.fwd_elem)
    assert np.all(code[:nf] == 0)
    np.testing.assert_array_equal(elem[:nf], w.fwd_elem)
    assert np.max(np.abs(r[:nf] - w.fwd_r)) < 1e-12
    assert np.all(code[nf:] != 0)
    cnt, _ = m.box_candidates(pts)
    np.testing.assert_array_equal(code == 2, cnt == 0)
    assert np.all(np.isinf(dist2[code == 2])) and np.all(elem[code == 2] == -1)


def test_find_exhaustive_selection(config1_oracle):
    """Newton in every element (no box test): every element in which the
    point is INTERIOR passes that element's boxes (no box false negative,
    Sec. 3.1), find returns the lowest such id, and a BORDER result is the
    candidate with the smallest dist2, ties to the lower id (Sec. 3.2)."""
    w, m, pts = config1_oracle
    rng = np.random.default_rng(7)
    sel = np.concatenate([rng.choice(len(w.fwd_elem), 300, replace=False), len(w.fwd_elem) + np.arange(100)])
    P = pts[sel]
    code, elem, r, dist2 = m.findpts(P)
    inter = np.zeros((len(P), m.NE), bool)
    dd = np.full((len(P), m.NE), np.inf)
    inbox = np.zeros((len(P), m.NE), bool)
    for e in range(m.NE):
        c, rr, d2 = m.locate_in_element(e, P)
        inbox[:, e] = _np_in_boxes(m, e, P)
        inter[:, e] = c == 0
        dd[:, e] = np.where(inbox[:, e], d2, np.inf)
    assert not np.any(inter & ~inbox)
    for p in range(len(P)):
        if inter[p].any():
            assert code[p] == 0 and elem[p] == np.argmax(inter[p] & inbox[p])
        elif inbox[p].any():
            assert code[p] == 1 and elem[p] == int(np.argmin(dd[p]))
            assert dist2[p] == dd[p, elem[p]]
        else:
            assert code[p] == 2


def test_eval_polynomial_exact_on_affine_mesh():
    """On an affine mesh a polynomial of total degree <= p in x is
    interpolated exactly (Eq. u_tensor)."""
    coords, A, b = affine_hex_mesh(seed=8, n=2, order=3)
    m = oracle.OracleMesh(coords, 3, 3, 4)
    rng = np.random.default_rng(9)
    exps, coef = W.polynomial_coeffs(rng, 3, 3)
    field = W.eval_polynomial(exps, coef, list(coords))[None]
    elem = rng.integers(0, m.NE, 500).astype(np.int32)
    pts = m.forward_map(elem, rng.uniform(-1, 1, (500, 3)))
    code, el, r, dist2 = m.findpts(pts)
    assert np.all(code == 0)
    out = m.eval(field, code, el, r)[0]
    exact = W.eval_polynomial(exps, coef, list(pts.T))
    np.testing.assert_allclose(out, exact, atol=1e-13 * np.abs(exact).max())


def test_eval_coordinate_field_invariant(config1_oracle):
    """Interpolating the coordinate fields at (e*, r*) gives x(r*), so
    |u_x(r*) - x*|^2 = dist2 for every found point, BORDER included."""
    w, m, pts = config1_oracle
    code, elem, r, dist2 = m.findpts(pts)
    ux = m.eval(m.coords, code, elem, r)
    found = code != 2
    err = np.sum((ux[:, found].T - pts[found]) ** 2, axis=1)
    np.testing.assert_allclose(err, dist2[found], rtol=1e-10, atol=1e-24)
    assert np.all(ux[:, ~found] == 0.0)


@pytest.mark.parametrize("name", ["sphere", "torus"])
def test_surface_codes(name):
    """Surface quads (Sec. 4.4): on-surface points are INTERIOR; points
    displaced along the normal are BORDER (if inside a box) or NOT_FOUND;
    never INTERIOR."""
    coords, d, dr, N = MESHES[name]()
    m = oracle.OracleMesh(coords, d, dr, N)
    rng = np.random.default_rng(10)
    elem = rng.integers(0, m.NE, 200).astype(np.int32)
    rt = rng.uniform(-0.95, 0.95, (200, 2))
    x, J = m.forward_map(elem, rt, jacobian=True)
    code, el, r, dist2 = m.findpts(x)
    assert np.all(code == 0)
    np.testing.assert_array_equal(el, elem)
    assert np.max(np.abs(r - rt)) < 1e-11
    nrm = np.cross(J[:, :, 0], J[:, :, 1])
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    off = x + 1e-3 * nrm
    code, el, r, dist2 = m.findpts(off)
    assert np.all(code != 0)
    b = code == 1
    np.testing.assert_allclose(dist2[b], 1e-6, rtol=0.05)


def test_nonfinite_points_not_found(config1_oracle):
    w, m, pts = config1_oracle
    bad = np.array([[np.nan, 0.5], [0.5, np.inf], [-np.inf, -np.inf]])
    code, elem, r, dist2 = m.findpts(bad)
    assert np.all(code == 2) and np.all(elem == -1)


@pytest.mark.parametrize("dr,N,Nf", [(3, 5, 3), (3, 3, 6), (3, 4, 4), (2, 2, 8), (2, 6, 2), (2, 4, 7),
                                     (1, 4, 3), (1, 3, 8)])
def test_eval_field_order_differs(dr, N, Nf):
    """A field of N~ nodes per direction (Sec. 2, after Eq. u_tensor: N~ may
    differ from the mesh's N): values P(zeta~_i, zeta~_j[, zeta~_k]) of a
    polynomial P of degree <= N~-1 in each reference variable are
    interpolated exactly at any r, whatever N is; a polynomial of degree N~
    in one variable is not (so the N~-point basis is the one used)."""
    d = 3
    if dr == 3:
        coords = W.hex_mesh(2, N - 1, 0.2)
    elif dr == 2:
        coords = W.cubed_sphere(1, N - 1)
    else:
        coords = W.helix_lines(5, N - 1)
    m = oracle.OracleMesh(coords, d, dr, N)
    rng = np.random.default_rng(100 + 10 * N + Nf)
    z = W.gll_points(Nf)
    grids = np.meshgrid(*([z] * dr), indexing="ij")  # grids[j][i0, i1, (i2)]
    nodes = [g.transpose(*reversed(range(dr))).reshape(-1) for g in grids]  # r_j of node q, r fastest

    def poly(c, pts):
        v = np.zeros(pts[0].shape)
        for idx in np.ndindex(*c.shape):
            t = c[idx]
            for j in range(dr):
                t = t * pts[j] ** idx[j]
            v = v + t
        return v

    c = rng.uniform(-1, 1, (Nf,) * dr)
    scale = 1.0 + np.arange(m.NE)[:, None]
    field = (scale * poly(c, nodes)[None, :])[None]
    n = 400
    elem = rng.integers(0, m.NE, n).astype(np.int32)
    r = rng.uniform(-1, 1, (n, dr))
    code = np.zeros(n, np.int32)
    out = m.eval(field, code, elem, r, field_N=Nf)[0]
    exact = (1.0 + elem) * poly(c, list(r.T))
    np.testing.assert_allclose(out, exact, atol=1e-12 * np.abs(exact).max())
    c2 = np.zeros((Nf + 1,) * dr)
    c2[(Nf,) + (0,) * (dr - 1)] = 1.0  # r^N~
    field2 = np.tile(poly(c2, nodes), (m.NE, 1))[None]
    out2 = m.eval(field2, code, elem, r, field_N=Nf)[0]
    assert np.max(np.abs(out2 - r[:, 0] ** Nf)) > 1e-3


# ---- line elements (Sec. 2, Eq. x_tensor_surf; Sec. 4.2 Rodrigues frame) ----

LINES = {
    "circle2d": lambda: (W.circle_lines(12, 4), 2, 5),
    "star2d": lambda: (W.star_lines(24, 3), 2, 4),
    "helix3d": lambda: (W.helix_lines(16, 5), 3, 6),
    "segment3d": lambda: (W.segment_lines(5, 3, (0.1, -0.2, 0.3), (0.9, 0.5, -0.4)), 3, 4),
}


@pytest.mark.parametrize("name", list(LINES))
def test_line_boxes_contain_samples(name):
    """Every expanded AABB and OBB contains dense samples of its curved line
    element (Secs. 3.1.1-3.1.2 with the line bounds and frame of Sec. 4)."""
    coords, d, N = LINES[name]()
    m = oracle.OracleMesh(coords, d, 1, N)
    rs = np.linspace(-1, 1, 401)
    for e in range(m.NE):
        x = m.forward_map(np.full(rs.size, e, np.int32), rs[:, None])
        lo, hi = m.aabb[e, :d], m.aabb[e, d:]
        assert np.all(x >= lo - 1e-14) and np.all(x <= hi + 1e-14)
        y = (x - m.obb_c[e]) @ m.obb_A[e].T
        assert np.max(np.abs(y)) <= 1 + 1e-12


@pytest.mark.parametrize("name", ["circle2d", "helix3d", "segment3d"])
def test_line_frame_is_rodrigues(name):
    """The OBB matrix is diag(1/hw) R with R the rotation taking the unit
    tangent at r = 0 to the x axis: its rows are orthogonal, row 0 is
    parallel to the tangent, and R t / |t| = e1 (sign included)."""
    coords, d, N = LINES[name]()
    m = oracle.OracleMesh(coords, d, 1, N)
    elem = np.arange(m.NE, dtype=np.int32)
    _, J = m.forward_map(elem, np.zeros((m.NE, 1)), jacobian=True)
    for e in range(m.NE):
        A = m.obb_A[e]
        Rn = A / np.linalg.norm(A, axis=1, keepdims=True)
        np.testing.assert_allclose(Rn @ Rn.T, np.eye(d), atol=1e-12)
        t = J[e, :, 0] / np.linalg.norm(J[e, :, 0])
        np.testing.assert_allclose(Rn @ t, np.eye(d)[0], atol=1e-12)
        assert np.linalg.det(Rn) > 0


def test_line_projection_affine_closed_form():
    """Straight line elements: the closest point of x* is the clamped
    orthogonal projection on the element's chord, r* = clamp(2 t - 1) with
    t = (x* - x_a).(x_b - x_a) / |x_b - x_a|^2, and dist2 its squared
    distance (Sec. 3.2.1 constrained Newton, Sec. 4.4 codes)."""
    xa, xb = np.array([0.1, -0.2, 0.3]), np.array([0.9, 0.5, -0.4])
    coords = W.segment_lines(1, 3, xa, xb)
    m = oracle.OracleMesh(coords, 3, 1, 4, tol=1.0)
    rng = np.random.default_rng(30)
    u = xb - xa
    perp = np.cross(u, [0.3, 0.7, 0.1])
    perp /= np.linalg.norm(perp)
    t = rng.uniform(-0.3, 1.3, 300)
    off = rng.uniform(-0.2, 0.2, 300) * np.linalg.norm(u) * 0.05
    pts = xa + t[:, None] * u + off[:, None] * perp
    code, elem, r, dist2 = m.findpts(pts)
    tt = np.clip(((pts - xa) @ u) / (u @ u), 0, 1)
    q = xa + tt[:, None] * u
    found = code != 2
    assert found.sum() > 100
    np.testing.assert_allclose(r[found, 0], 2 * tt[found] - 1, atol=1e-12)
    np.testing.assert_allclose(dist2[found], np.sum((pts - q) ** 2, axis=1)[found], rtol=1e-10, atol=1e-28)
    assert np.all(code[found & (np.abs(off) * np.linalg.norm(u) > 1e-4)] == 1)


@pytest.mark.parametrize("name", ["circle2d", "star2d", "helix3d"])
def test_line_closest_point_brute_force(name):
    """Points near a curved line mesh: the oracle's dist2 equals the minimum
    over dense samples of the candidate elements' curves (those whose AABB
    and OBB contain the point; to the sampling resolution, never above it by
    more than rounding), and at an interior r* the residual is orthogonal to
    the tangent (the KKT condition)."""
    coords, d, N = LINES[name]()
    m = oracle.OracleMesh(coords, d, 1, N, tol=1.0)
    rng = np.random.default_rng(31)
    el = rng.integers(0, m.NE, 300).astype(np.int32)
    rt = rng.uniform(-1, 1, (300, 1))
    x, J = m.forward_map(el, rt, jacobian=True)
    pts = x + 0.003 * rng.standard_normal(x.shape)
    code, elem, r, dist2 = m.findpts(pts)
    rs = np.linspace(-1, 1, 4001)
    curves = np.stack([m.forward_map(np.full(rs.size, e, np.int32), rs[:, None]) for e in range(m.NE)])
    checked = 0
    for p in np.flatnonzero(code == 1):
        in_aabb = np.all((pts[p] >= m.aabb[:, :d]) & (pts[p] <= m.aabb[:, d:]), axis=1)
        in_obb = np.max(np.abs(np.einsum("eij,ej->ei", m.obb_A, pts[p] - m.obb_c)), axis=1) <= 1
        cand = np.flatnonzero(in_aabb & in_obb)  # the method's candidates (Sec. 3.2)
        best = min(np.min(np.sum((curves[e] - pts[p]) ** 2, axis=1)) for e in cand)
        assert dist2[p] <= best * (1 + 1e-9) + 1e-24
        # the samples miss the true minimum by at most delta = half the sample spacing
        delta = 0.5 * max(np.max(np.linalg.norm(np.diff(curves[e], axis=0), axis=1)) for e in cand)
        assert dist2[p] >= best - 2 * np.sqrt(best) * delta - delta ** 2
        if abs(r[p, 0]) < 1 - 1e-9:
            xr, Jr = m.forward_map(elem[p:p + 1], r[p:p + 1], jacobian=True)
            assert abs((pts[p] - xr[0]) @ Jr[0, :, 0]) <= 1e-9 * np.linalg.norm(Jr[0, :, 0]) * np.sqrt(dist2[p]) + 1e-14
        checked += 1
    assert checked > 100


@pytest.mark.parametrize("name", ["circle2d", "helix3d"])
def test_line_forward_map_recovered(name):
    """Points x_e(r) on the curve are INTERIOR in element e with r recovered
    to 1e-12 (Sec. 4.4: dist2 below eps_d)."""
    coords, d, N = LINES[name]()
    m = oracle.OracleMesh(coords, d, 1, N)
    rng = np.random.default_rng(32)
    el = rng.integers(0, m.NE, 500).astype(np.int32)
    rt = rng.uniform(-0.98, 0.98, (500, 1))
    code, elem, r, dist2 = m.findpts(m.forward_map(el, rt))
    assert np.all(code == 0)
    np.testing.assert_array_equal(elem, el)
    np.testing.assert_allclose(r, rt, atol=1e-12)


def numpy_jacobian(coords, d, dr, N, e, r):
    """Independent dx_c/dr_j of x_e (Eq. jacobian) at one r, with numpy
    Legendre fits of the 1D Lagrange bases and their derivatives."""
    z = W.gll_points(N)
    ne = N ** dr
    fits = [L.legfit(z, np.eye(N)[i], N - 1) for i in range(N)]
    V = [np.array([L.legval(r[j], f) for f in fits]) for j in range(dr)]
    D = [np.array([L.legval(r[j], L.legder(f)) for f in fits]) for j in range(dr)]
    idx = np.arange(ne)
    J = np.zeros((d, dr))
    for j in range(dr):
        w = np.ones(ne)
        for k in range(dr):
            w = w * (D[k] if k == j else V[k])[(idx // N ** k) % N]
        J[:, j] = [coords[c, e] @ w for c in range(d)]
    return J


def _frame_checks(J):
    """Sec. 4.2 on one 3x2 Jacobian: R1 is a proper rotation taking the unit
    normal n = t1 x t2 / |t1 x t2| to e3, and R = R2 R1 takes t1, t2, n to
    e1, e2, e3 (R2 is the inverse of [R1 t1, R1 t2, e3])."""
    t1, t2 = J[:, 0], J[:, 1]
    n = np.cross(t1, t2)
    n /= np.linalg.norm(n)
    R1, R = oracle.surface_frame(J)
    np.testing.assert_allclose(R1 @ R1.T, np.eye(3), atol=1e-14)
    assert abs(np.linalg.det(R1) - 1.0) < 1e-14
    np.testing.assert_allclose(R1 @ n, [0.0, 0.0, 1.0], atol=1e-14)
    np.testing.assert_allclose(R @ np.column_stack([t1, t2, n]), np.eye(3), atol=1e-13)
    return R, n


@pytest.mark.parametrize("name", ["sphere", "torus"])
def test_surface_frame_is_sec42(name):
    """The surface OBB frame (Sec. 4.2) of every element of the sphere and
    torus meshes: the checks of _frame_checks on J_c = G(0) computed
    independently with numpy, and the stored OBB matrix A = diag(1/hw) R
    (Eq. OBB_test) maps t1, t2, n onto positive multiples of e1, e2, e3."""
    coords, d, dr, N = MESHES[name]()
    m = oracle.OracleMesh(coords, d, dr, N)
    for e in range(m.NE):
        J = numpy_jacobian(m.coords, 3, 2, N, e, np.zeros(2))
        _, n = _frame_checks(J)
        M = m.obb_A[e] @ np.column_stack([J[:, 0], J[:, 1], n])
        diag = np.diag(M)
        assert np.all(diag > 0), (name, e)
        off = M - np.diag(diag)
        assert np.max(np.abs(off)) <= 1e-12 * np.max(diag), (name, e)


def test_surface_frame_special_orientations():
    """Frames for tangents whose normal is +e3, -e3 (the rotation's axis is
    undefined there), nearly -e3, and random orientations and shears."""
    rng = np.random.default_rng(42)
    cases = [np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]]),        # n = +e3
             np.array([[0.0, 1.0], [1.0, 0.0], [0.0, 0.0]]),        # n = -e3
             np.array([[0.0, 1.0], [1.0, 0.0], [1e-9, 0.0]]),       # n close to -e3
             np.array([[0.2, 0.0], [0.0, -3.0], [0.0, 0.0]])]       # scaled, n = -e3
    for _ in range(40):
        cases.append(rng.normal(size=(3, 2)) * rng.uniform(0.01, 10.0))
    for J in cases:
        _frame_checks(J)


@pytest.mark.parametrize("N", [2, 4, 6])
def test_surface_obb_affine_closed_form(N):
    """A flat parallelogram quad x = x_c + t1 r + t2 s in 3D (any
    orientation): in the frame R of Sec. 4.2 its nodes are (r, s, 0), so the
    expanded frame box has half-widths (1+tol)(1, 1) and, for the zero
    normal extent (Sec. 4.1), tol * Lmin / 2 = tol with Lmin = 2: the stored
    A is diag(1/1.1, 1/1.1, 1/0.1) [t1 t2 n]^{-1} and the OBB centre is x_c."""
    rng = np.random.default_rng(7 + N)
    z = W.gll_points(N)
    rr, ss = np.meshgrid(z, z, indexing="xy")  # node i + N j: r fastest
    rr, ss = rr.reshape(-1), ss.reshape(-1)
    elems, frames = [], []
    for _ in range(6):
        t1, t2 = rng.normal(size=3), rng.normal(size=3)
        xc = rng.uniform(-2, 2, 3)
        x = xc[:, None] + t1[:, None] * rr[None] + t2[:, None] * ss[None]
        elems.append(x)
        n = np.cross(t1, t2)
        n /= np.linalg.norm(n)
        frames.append((xc, np.column_stack([t1, t2, n])))
    coords = np.ascontiguousarray(np.stack(elems, axis=1))  # [3][NE][N^2]
    m = oracle.OracleMesh(coords, 3, 2, N)
    for e, (xc, B) in enumerate(frames):
        A = np.diag([1 / 1.1, 1 / 1.1, 1 / 0.1]) @ np.linalg.inv(B)
        np.testing.assert_allclose(m.obb_A[e], A, rtol=1e-11, atol=1e-11 * np.abs(A).max())
        np.testing.assert_allclose(m.obb_c[e], xc, atol=1e-12 * (1 + np.abs(xc).max()))
