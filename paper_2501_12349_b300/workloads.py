"""Seeded synthetic workloads for findpts: meshes, query points, fields.

This module holds none of the method's arithmetic.  Mesh nodes are GLL
reference points (numpy's Legendre roots) mapped through analytic maps;
fields are analytic functions sampled at the nodes; query points are drawn in
physical space, or as (element, r) pairs that the caller maps to x with an
element-map evaluation of its choice.  The paper's own meshes (triple point,
turbine blade, NekRS channel) are not available, so these stand in for them
with the same element types, orders, sizes and point distributions.

Layouts: coords [d][NE][N^dr] with node n = i + N*j (+ N*N*k) and element
e = ex + nx*(ey + ny*ez); points [n][d]; r [n][dr]; fields [nc][NE][N^dr].
"""
from __future__ import annotations

from dataclasses import dataclass, field
from itertools import product

import numpy as np
from numpy.polynomial import legendre as _npleg


def gll_points(N: int) -> np.ndarray:
    """The N Gauss-Lobatto-Legendre points: -1, +1 and the roots of P'_{N-1}."""
    if N == 2:
        return np.array([-1.0, 1.0])
    c = np.zeros(N)
    c[-1] = 1.0
    inner = np.sort(np.real(_npleg.legroots(_npleg.legder(c))))
    return np.concatenate([[-1.0], inner, [1.0]])


# --------------------------------------------------------------------------
# structured meshes


def _tensor_nodes(n: tuple[int, ...], N: int) -> list[np.ndarray]:
    """Undeformed nodes of an n[0] x n[1] (x n[2]) box mesh of [0,1]^d, one
    array per coordinate, shaped [NE, N^d]."""
    z = gll_points(N)
    d = len(n)
    axes = []
    for a in range(d):
        e = np.arange(n[a])[:, None]
        axes.append((e + 0.5 * (1.0 + z[None, :])) / n[a])  # [n_a, N]
    if d == 2:
        ny, nx = n[1], n[0]
        X = np.broadcast_to(axes[0][None, :, None, :], (ny, nx, N, N))
        Y = np.broadcast_to(axes[1][:, None, :, None], (ny, nx, N, N))
        return [np.ascontiguousarray(X).reshape(nx * ny, N * N),
                np.ascontiguousarray(Y).reshape(nx * ny, N * N)]
    nz, ny, nx = n[2], n[1], n[0]
    shape = (nz, ny, nx, N, N, N)
    X = np.broadcast_to(axes[0][None, None, :, None, None, :], shape)
    Y = np.broadcast_to(axes[1][None, :, None, None, :, None], shape)
    Z = np.broadcast_to(axes[2][:, None, None, :, None, None], shape)
    NE = nx * ny * nz
    return [np.ascontiguousarray(A).reshape(NE, N ** 3) for A in (X, Y, Z)]


def sine_perturbation_2d(x, y, amp):
    """Config-1 map: both coordinates displaced by amp*sin(2 pi x) sin(2 pi y)."""
    s = amp * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    return x + s, y + s


def kershaw_like_3d(x, y, z, A):
    """Smooth, boundary-preserving deformation of the unit cube,
    x_i' = x_i + A/(2 pi) sin(2 pi x_i) prod_{j != i} sin(pi x_j).
    d x_i'/d x_i >= 1 - A and the off-diagonal row sum is <= A, so for A < 0.5
    the Jacobian is diagonally dominant and the map is a bijection."""
    sx, sy, sz = np.sin(np.pi * x), np.sin(np.pi * y), np.sin(np.pi * z)
    c = A / (2 * np.pi)
    return (x + c * np.sin(2 * np.pi * x) * sy * sz,
            y + c * np.sin(2 * np.pi * y) * sx * sz,
            z + c * np.sin(2 * np.pi * z) * sx * sy)


def kershaw_like_2d(x, y, A):
    c = A / (2 * np.pi)
    return (x + c * np.sin(2 * np.pi * x) * np.sin(np.pi * y),
            y + c * np.sin(2 * np.pi * y) * np.sin(np.pi * x))


def quad_mesh(n: int, order: int, amp: float = 0.0, kind: str = "sine") -> np.ndarray:
    N = order + 1
    X, Y = _tensor_nodes((n, n), N)
    if kind == "sine":
        X, Y = sine_perturbation_2d(X, Y, amp)
    else:
        X, Y = kershaw_like_2d(X, Y, amp)
    return np.ascontiguousarray(np.stack([X, Y]))


def hex_mesh(n: int, order: int, A: float = 0.3) -> np.ndarray:
    N = order + 1
    X, Y, Z = _tensor_nodes((n, n, n), N)
    X, Y, Z = kershaw_like_3d(X, Y, Z, A)
    return np.ascontiguousarray(np.stack([X, Y, Z]))


def cubed_sphere(n: int, order: int, radius: float = 1.0) -> np.ndarray:
    """6 n^2 quads on the sphere: each cube face gridded n x n and its nodes
    projected radially, so every node lies exactly on the sphere."""
    N = order + 1
    z = gll_points(N)
    a1 = (np.arange(n)[:, None] + 0.5 * (1 + z[None, :])) * (2.0 / n) - 1.0  # [n, N]
    A = np.broadcast_to(a1[None, :, None, :], (n, n, N, N))  # [eb, ea, j, i] -> a from (ea,i)
    B = np.broadcast_to(a1[:, None, :, None], (n, n, N, N))
    A = np.ascontiguousarray(A).reshape(n * n, N * N)
    B = np.ascontiguousarray(B).reshape(n * n, N * N)
    one = np.ones_like(A)
    faces = [(one, A, B), (-one, A, B), (A, one, B), (A, -one, B), (A, B, one), (A, B, -one)]
    xs, ys, zs = [], [], []
    for fx, fy, fz in faces:
        nrm = np.sqrt(fx * fx + fy * fy + fz * fz)
        xs.append(radius * fx / nrm)
        ys.append(radius * fy / nrm)
        zs.append(radius * fz / nrm)
    return np.ascontiguousarray(np.stack([np.concatenate(xs), np.concatenate(ys), np.concatenate(zs)]))


def torus(nu: int, nv: int, order: int, R: float = 1.0, r: float = 0.3) -> np.ndarray:
    N = order + 1
    z = gll_points(N)
    u1 = (np.arange(nu)[:, None] + 0.5 * (1 + z[None, :])) * (2 * np.pi / nu)
    v1 = (np.arange(nv)[:, None] + 0.5 * (1 + z[None, :])) * (2 * np.pi / nv)
    U = np.ascontiguousarray(np.broadcast_to(u1[None, :, None, :], (nv, nu, N, N))).reshape(nu * nv, N * N)
    V = np.ascontiguousarray(np.broadcast_to(v1[:, None, :, None], (nv, nu, N, N))).reshape(nu * nv, N * N)
    X = (R + r * np.cos(V)) * np.cos(U)
    Y = (R + r * np.cos(V)) * np.sin(U)
    Z = r * np.sin(V)
    return np.ascontiguousarray(np.stack([X, Y, Z]))


def circle_lines(n: int, order: int, radius: float = 1.0, centre=(0.0, 0.0)) -> np.ndarray:
    """n line elements on a circle in 2D, nodes at the GLL points of each
    element's angle interval (every node exactly on the circle): [2][n][N]."""
    N = order + 1
    z = gll_points(N)
    th = (np.arange(n)[:, None] + 0.5 * (1 + z[None, :])) * (2 * np.pi / n)
    return np.ascontiguousarray(np.stack([centre[0] + radius * np.cos(th), centre[1] + radius * np.sin(th)]))


def helix_lines(n: int, order: int, turns: float = 2.0, radius: float = 0.5, pitch: float = 0.25) -> np.ndarray:
    """n line elements along a helix in 3D (nodes on the helix): [3][n][N]."""
    N = order + 1
    z = gll_points(N)
    th = (np.arange(n)[:, None] + 0.5 * (1 + z[None, :])) * (2 * np.pi * turns / n)
    return np.ascontiguousarray(np.stack([radius * np.cos(th), radius * np.sin(th), pitch * th / (2 * np.pi)]))


def segment_lines(n: int, order: int, xa, xb) -> np.ndarray:
    """n straight (affine) line elements splitting the segment xa -> xb."""
    N = order + 1
    z = gll_points(N)
    t = (np.arange(n)[:, None] + 0.5 * (1 + z[None, :])) / n
    xa, xb = np.asarray(xa, float), np.asarray(xb, float)
    return np.ascontiguousarray(np.stack([xa[c] + t * (xb[c] - xa[c]) for c in range(len(xa))]))


def star_lines(n: int, order: int, a: float = 0.15, k: int = 5) -> np.ndarray:
    """n line elements on the closed curve rho(theta) = 1 + a cos(k theta) in
    2D (a curved boundary), nodes at the GLL points of each theta interval."""
    N = order + 1
    z = gll_points(N)
    th = (np.arange(n)[:, None] + 0.5 * (1 + z[None, :])) * (2 * np.pi / n)
    rho = 1.0 + a * np.cos(k * th)
    return np.ascontiguousarray(np.stack([rho * np.cos(th), rho * np.sin(th)]))


def projection_points(coords: np.ndarray, rng: np.random.Generator, tangential: float = 0.3,
                      normal: float = 0.5) -> np.ndarray:
    """Closest-point projection workload (the tangential relaxation of the
    paper's r-adaptivity example): every node of a 2D line mesh moved along
    the curve's tangent by up to +-tangential h (h = the element's chord)
    and off it by up to +-normal s (s = the element's sagitta, the largest
    distance of its nodes from the chord), as a mesh optimiser moves
    boundary nodes, its steps scaled down so the nodes stay inside the
    (100%-expanded) boxes.  Returns points [NE*N][2]."""
    d, NE, N = coords.shape
    chord = coords[:, :, -1] - coords[:, :, 0]
    h = np.linalg.norm(chord, axis=0)  # [NE]
    ch = chord / h
    rel = coords - coords[:, :, :1]
    sag = np.max(np.abs(rel[0] * ch[1][:, None] - rel[1] * ch[0][:, None]), axis=1)  # [NE]
    tan = np.gradient(coords, axis=2)
    tan = tan / np.linalg.norm(tan, axis=0, keepdims=True)
    nrm = np.stack([-tan[1], tan[0]])
    st = rng.uniform(-tangential, tangential, (NE, N)) * h[:, None]
    sn = rng.uniform(-normal, normal, (NE, N)) * sag[:, None]
    x = coords + st[None] * tan + sn[None] * nrm
    return np.ascontiguousarray(x.reshape(d, -1).T)


def boundary_lines(quad_coords: np.ndarray, n: int) -> np.ndarray:
    """The boundary of an n x n quad mesh of [0,1]^2 (node layout i + N j,
    elements row by row) as 4n line elements: [2][4n][N]."""
    N = int(round(np.sqrt(quad_coords.shape[2])))
    X = quad_coords.reshape(2, n, n, N, N)  # [c][ey][ex][j][i]
    edges = []
    for ex in range(n):
        edges.append(X[:, 0, ex, 0, :])            # bottom, i along +x
    for ey in range(n):
        edges.append(X[:, ey, n - 1, :, N - 1])    # right, j along +y
    for ex in reversed(range(n)):
        edges.append(X[:, n - 1, ex, N - 1, ::-1])  # top, towards -x
    for ey in reversed(range(n)):
        edges.append(X[:, ey, 0, ::-1, 0])         # left, towards -y
    return np.ascontiguousarray(np.stack(edges, axis=1))


# --------------------------------------------------------------------------
# fields and points


def polynomial_coeffs(rng: np.random.Generator, d: int, degree: int):
    exps = [e for e in product(range(degree + 1), repeat=d) if sum(e) <= degree]
    return exps, rng.uniform(-1.0, 1.0, size=len(exps))


def eval_polynomial(exps, coef, xs):
    out = np.zeros_like(xs[0])
    for e, c in zip(exps, coef):
        t = np.full_like(xs[0], c)
        for k, p in enumerate(e):
            if p:
                t = t * xs[k] ** p
        out += t
    return out


def polynomial_field(coords: np.ndarray, rng: np.random.Generator, degree: int, nc: int = 1):
    """nc random polynomials of total degree <= degree in the physical
    coordinates (coefficients U[-1,1]) sampled at the nodes: [nc][NE][ne]."""
    d = coords.shape[0]
    polys = [polynomial_coeffs(rng, d, degree) for _ in range(nc)]
    f = np.stack([eval_polynomial(e, c, list(coords)) for e, c in polys])
    return np.ascontiguousarray(f), polys


def uniform_box_points(rng, n: int, d: int, lo: float, hi: float) -> np.ndarray:
    return rng.uniform(lo, hi, size=(n, d))


def outside_unit_box_points(rng, n: int, d: int, lo: float = -0.1, hi: float = 1.1) -> np.ndarray:
    """n points uniform in [lo,hi]^d minus [0,1]^d (rejection sampling)."""
    out = np.empty((0, d))
    while out.shape[0] < n:
        p = rng.uniform(lo, hi, size=(4 * n, d))
        inside = np.all((p >= 0.0) & (p <= 1.0), axis=1)
        out = np.concatenate([out, p[~inside]])
    return out[:n]


def analytic_surface_points(rng, name: str, n: int, offset: np.ndarray) -> np.ndarray:
    """Points on the analytic sphere (radius 1) or torus (R = 1, r = 0.3)
    that the cubed-sphere / torus meshes interpolate, displaced by `offset`
    along the analytic normal (physical-space inputs for benchmarks; the
    interpolated surface differs from the analytic one by the interpolation
    error, so on-surface points end INTERIOR or BORDER by that error)."""
    if "sphere" in name:
        v = rng.normal(size=(n, 3))
        v /= np.linalg.norm(v, axis=1)[:, None]
        return v * (1.0 + offset)[:, None]
    u = rng.uniform(0, 2 * np.pi, n)
    t = rng.uniform(0, 2 * np.pi, n)
    rr = 0.3 + offset
    return np.stack([(1.0 + rr * np.cos(t)) * np.cos(u), (1.0 + rr * np.cos(t)) * np.sin(u), rr * np.sin(t)], 1)


def element_reference_points(rng, n: int, NE: int, dr: int, rmax: float = 0.95):
    """(elem, r) pairs: elem uniform in [0, NE), r uniform in [-rmax, rmax]^dr."""
    elem = rng.integers(0, NE, size=n).astype(np.int32)
    r = rng.uniform(-rmax, rmax, size=(n, dr))
    return elem, r


# --------------------------------------------------------------------------
# the five workloads


@dataclass
class Workload:
    name: str
    coords: np.ndarray
    d: int
    dr: int
    order: int
    field: np.ndarray | None
    pts: np.ndarray | None = None          # physical points, when drawn directly
    fwd_elem: np.ndarray | None = None     # (elem, r) pairs to be mapped by the caller
    fwd_r: np.ndarray | None = None
    fwd_offset: np.ndarray | None = None   # surface points: normal offset distance per pair
    h: float = 0.0
    extra: dict = field(default_factory=dict)

    @property
    def N(self):
        return self.order + 1

    @property
    def NE(self):
        return self.coords.shape[1]


def config1(seed: int = 1) -> Workload:
    """2D: 8x8 quads on [0,1]^2, p=3, both coordinates displaced by
    0.05 h sin(2 pi x) sin(2 pi y); 9,900 forward-map points (elem uniform,
    r uniform in [-0.95,0.95]^2) and 100 points outside the unit square in
    [-0.1,1.1]^2; a random degree-3 polynomial field."""
    rng = np.random.default_rng(seed)
    n, p = 8, 3
    coords = quad_mesh(n, p, amp=0.05 / n, kind="sine")
    elem, r = element_reference_points(rng, 9900, n * n, 2)
    outside = outside_unit_box_points(rng, 100, 2)
    fld, polys = polynomial_field(coords, rng, 3)
    return Workload("quad2d_8x8_p3", coords, 2, 2, p, fld, pts=outside, fwd_elem=elem, fwd_r=r,
                    h=1.0 / n, extra={"polys": polys})


def hex_config(seed: int, npts: int, nc: int, n: int = 32, order: int = 4, A: float = 0.3,
               delta: float = 0.0034) -> Workload:
    rng = np.random.default_rng(seed)
    coords = hex_mesh(n, order, A)
    pts = uniform_box_points(rng, npts, 3, -delta, 1.0 + delta)
    fld, polys = polynomial_field(coords, rng, order, nc)
    return Workload(f"hex3d_{n}^3_p{order}", coords, 3, 3, order, fld, pts=pts, h=1.0 / n,
                    extra={"polys": polys, "A": A, "delta": delta})


def config2(seed: int = 2, npts: int = 10 ** 6) -> Workload:
    """3D: 32^3 hexes on [0,1]^3, p=4, smooth deformation amplitude 0.3;
    10^6 points uniform in [-0.0034, 1.0034]^3 (about 2% outside); a random
    degree-4 polynomial field."""
    return hex_config(seed, npts, 1)


def config3(seed: int = 3, npts: int = 10 ** 7) -> Workload:
    """The config-2 mesh with 10^7 points and a 3-component field."""
    return hex_config(seed, npts, 3)


def config4(seed: int = 4, max_points: int | None = None, max_elems: int | None = None) -> list[Workload]:
    """64 meshes: type uniform in {quad 2D, hex 3D, quad surface in 3D
    (cubed sphere or torus)}, p uniform in 2..7, NE log-uniform in [1e3, 5e4],
    points per mesh log-uniform in [1e3, 1e6].  Volume points are uniform in
    the slightly enlarged unit box; surface points are 99% on the surface
    (forward-map pairs) and 1% displaced 0.1 h along the normal."""
    rng = np.random.default_rng(seed)
    out = []
    for m in range(64):
        kind = ["quad2d", "hex3d", "surf3d"][rng.integers(0, 3)]
        p = int(rng.integers(2, 8))
        NE_t = float(np.exp(rng.uniform(np.log(1e3), np.log(5e4))))
        npts = int(np.exp(rng.uniform(np.log(1e3), np.log(1e6))))
        if max_elems:
            NE_t = min(NE_t, max_elems)
        if max_points:
            npts = min(npts, max_points)
        amp = float(rng.uniform(0.05, 0.3))
        if kind == "quad2d":
            n = max(2, int(round(np.sqrt(NE_t))))
            coords = quad_mesh(n, p, amp=amp, kind="kershaw")
            h = 1.0 / n
            delta = 0.11 * h
            pts = uniform_box_points(rng, npts, 2, -delta, 1 + delta)
            w = Workload(f"m{m}_quad2d_n{n}_p{p}", coords, 2, 2, p, None, pts=pts, h=h)
        elif kind == "hex3d":
            n = max(2, int(round(NE_t ** (1 / 3))))
            coords = hex_mesh(n, p, A=amp)
            h = 1.0 / n
            delta = 0.11 * h
            pts = uniform_box_points(rng, npts, 3, -delta, 1 + delta)
            w = Workload(f"m{m}_hex3d_n{n}_p{p}", coords, 3, 3, p, None, pts=pts, h=h)
        else:
            if rng.integers(0, 2) == 0:
                n = max(1, int(round(np.sqrt(NE_t / 6))))
                coords = cubed_sphere(n, p)
                h = (np.pi / 2) / n
                name = f"m{m}_sphere_n{n}_p{p}"
            else:
                nv = max(2, int(round(np.sqrt(NE_t / 3))))
                nu = 3 * nv
                coords = torus(nu, nv, p)
                h = 2 * np.pi * 0.3 / nv
                name = f"m{m}_torus_{nu}x{nv}_p{p}"
            NE = coords.shape[1]
            elem, r = element_reference_points(rng, npts, NE, 2, rmax=1.0)
            off = np.where(rng.uniform(size=npts) < 0.01, 0.1 * h, 0.0)
            w = Workload(name, coords, 3, 2, p, None, fwd_elem=elem, fwd_r=r, fwd_offset=off, h=h)
            w.pts = analytic_surface_points(rng, name, npts, off)
        w.field, _ = polynomial_field(w.coords, rng, min(p, 3))
        out.append(w)
    return out


def config5_meshes(seed: int = 5, max_elems: int | None = None) -> list[Workload]:
    """8 resident hex meshes, p uniform in 3..7, NE log-uniform in
    [1e4, 1e5] (n^3), smooth deformations of random amplitude <= 0.3."""
    rng = np.random.default_rng(seed)
    out = []
    for m in range(8):
        p = int(rng.integers(3, 8))
        NE_t = float(np.exp(rng.uniform(np.log(1e4), np.log(1e5))))
        if max_elems:
            NE_t = min(NE_t, max_elems)
        n = max(2, int(round(NE_t ** (1 / 3))))
        A = float(rng.uniform(0.0, 0.3))
        coords = hex_mesh(n, p, A)
        fld, polys = polynomial_field(coords, rng, 3)
        out.append(Workload(f"s{m}_hex3d_n{n}_p{p}", coords, 3, 3, p, fld, h=1.0 / n,
                            extra={"A": A, "polys": polys}))
    return out


def velocity_field(coords: np.ndarray) -> np.ndarray:
    """Nodal values of u = (sin pi x cos pi y, -cos pi x sin pi y, 0.1): [3][NE][ne]."""
    x, y = coords[0], coords[1]
    return np.ascontiguousarray(np.stack([np.sin(np.pi * x) * np.cos(np.pi * y),
                                          -np.cos(np.pi * x) * np.sin(np.pi * y),
                                          np.full_like(x, 0.1)]))


@dataclass
class Request:
    t_arrival: float
    mesh: int
    kind: str          # "remap" or "particle"
    pts: np.ndarray    # [n][3]


def config5_requests(meshes: list[Workload], rate: float, n_req: int, seed: int = 5,
                     size_lo: float = 1e2, size_hi: float = 1e6) -> list[Request]:
    """Poisson arrivals at `rate` requests/s; sizes log-uniform in
    [size_lo, size_hi]; half remap, half particle; points uniform in the
    mesh's box (particles start inside the unit cube)."""
    rng = np.random.default_rng(seed + 1000)
    t = 0.0
    out = []
    for _ in range(n_req):
        t += rng.exponential(1.0 / rate)
        m = int(rng.integers(0, len(meshes)))
        n = int(np.exp(rng.uniform(np.log(size_lo), np.log(size_hi))))
        kind = "remap" if rng.integers(0, 2) == 0 else "particle"
        if kind == "remap":
            pts = rng.uniform(-0.01, 1.01, size=(n, 3))
        else:
            pts = rng.uniform(0.05, 0.95, size=(n, 3))
        out.append(Request(t, m, kind, pts))
    return out
