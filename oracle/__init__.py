"""FP64 CPU oracle for local findpts — TEST INFRASTRUCTURE ONLY.

A plain, slow restatement of arXiv 2501.12349 in C (oracle.c, OpenMP over
points), loaded with ctypes.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package; the CUDA
library never does, and the two share no code.

Functions take and return numpy arrays in the layouts of the C ABI:
coords [d][NE][N^dr], points [n][d], r [n][dr], aabb [NE][2d], obb_c [NE][d],
obb_A [NE][d][d].
"""
from __future__ import annotations

import ctypes
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "oracle.c"
LIB = HERE / "_oracle.so"

INTERIOR, BORDER, NOT_FOUND = 0, 1, 2

_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double


def build(force: bool = False) -> Path:
    """Compile oracle.c into _oracle.so with gcc (-O2, OpenMP, no fast-math)."""
    newest = max(SRC.stat().st_mtime, (HERE / "oracle.h").stat().st_mtime)
    if LIB.exists() and not force and LIB.stat().st_mtime >= newest:
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-fopenmp", "-fPIC", "-shared",
           "-o", str(LIB), str(SRC), "-lm"]
    subprocess.run(cmd, check=True)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(LIB))
        sig = {
            "or_gll_nodes": [_int, _D],
            "or_gauss_legendre": [_int, _D, _D],
            "or_lagrange": [_int, _D, _dbl, _D, _D, _D],
            "or_chebyshev_points": [_int, _D],
            "or_basis_bounds": [_int, _int, _int, _D, _D],
            "or_legendre_coeffs": [_int, _D, _D],
            "or_bound_1d": [_int, _int, _D, _D, _D],
            "or_bound_2d": [_int, _int, _D, _D, _D],
            "or_element_boxes": [_D, _int, _int, _int, _i64, _dbl, _int, _D, _D, _D],
            "or_newton": [_D, _int, _int, _int, _i64, _i64, _D, _dbl, _int, _D, _D, _I64],
            "or_findpts": [_D, _int, _int, _int, _i64, _D, _D, _D, _D, _i64, _dbl, _int, _dbl,
                           _I32, _I32, _D, _D, _I64],
            "or_locate_in_element": [_D, _int, _int, _int, _i64, _i64, _D, _i64, _dbl, _int, _dbl,
                                     _I32, _D, _D],
            "or_box_candidates": [_int, _i64, _D, _D, _D, _D, _i64, _I32, _I32],
            "or_eval": [_D, _int, _int, _int, _i64, _I32, _I32, _D, _i64, _D],
            "or_forward_map": [_D, _int, _int, _int, _i64, _I32, _D, _i64, _D, _D],
            "or_surface_frame": [_D, _D, _D],
            "or_num_threads": [],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _int
        L.or_lagrange.restype = None
        L.or_chebyshev_points.restype = None
        _lib = L
    return _lib


def _p(a, ty=_D):
    if a is None:
        return None
    return a.ctypes.data_as(ty)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(n: int) -> None:
    """OpenMP threads of later oracle calls."""
    f = lib().or_set_num_threads
    f.argtypes = [_int]
    f.restype = None
    f(int(n))


def gll_nodes(N: int) -> np.ndarray:
    z = np.zeros(N)
    assert lib().or_gll_nodes(N, _p(z)) == 0
    return z


def gauss_legendre(m: int):
    x, w = np.zeros(m), np.zeros(m)
    assert lib().or_gauss_legendre(m, _p(x), _p(w)) == 0
    return x, w


def lagrange(N: int, r: float, z=None):
    z = gll_nodes(N) if z is None else _f64(z)
    phi, dphi, d2phi = np.zeros(N), np.zeros(N), np.zeros(N)
    lib().or_lagrange(N, _p(z), float(r), _p(phi), _p(dphi), _p(d2phi))
    return phi, dphi, d2phi


def chebyshev_points(M: int) -> np.ndarray:
    eta = np.zeros(M)
    lib().or_chebyshev_points(M, _p(eta))
    return eta


def basis_bounds(N: int, M: int, reading: int = 0):
    lo, hi = np.zeros((N, M)), np.zeros((N, M))
    assert lib().or_basis_bounds(N, M, reading, _p(lo), _p(hi)) == 0
    return lo, hi


def legendre_coeffs(N: int):
    c0, c1 = np.zeros(N), np.zeros(N)
    assert lib().or_legendre_coeffs(N, _p(c0), _p(c1)) == 0
    return c0, c1


def bound_1d(u, M: int):
    u = _f64(u)
    lo, hi = _dbl(), _dbl()
    assert lib().or_bound_1d(len(u), M, _p(u), ctypes.byref(lo), ctypes.byref(hi)) == 0
    return lo.value, hi.value


def bound_2d(u, M: int):
    """u[b][a] (a fastest), i.e. u.ravel() = u_ab at a + N*b."""
    u = _f64(u)
    N = u.shape[-1]
    lo, hi = _dbl(), _dbl()
    assert lib().or_bound_2d(N, M, _p(u), ctypes.byref(lo), ctypes.byref(hi)) == 0
    return lo.value, hi.value


def surface_frame(Jc):
    """Sec. 4.2 frame of a surface quad from its 3x2 Jacobian at r = 0:
    returns (R1, R) with R1 the Rodrigues rotation and R = R2 R1."""
    Jc = _f64(Jc).reshape(3, 2)
    R1, R = np.zeros((3, 3)), np.zeros((3, 3))
    assert lib().or_surface_frame(_p(Jc), _p(R1), _p(R)) == 0
    return R1, R


def element_boxes(coords, d: int, dr: int, N: int, tol: float = 0.1, M: int = 0):
    coords = _f64(coords)
    NE = coords.size // (d * N ** dr)
    M = 2 * N if M == 0 else M
    aabb = np.zeros((NE, 2 * d))
    obb_c = np.zeros((NE, d))
    obb_A = np.zeros((NE, d, d))
    rc = lib().or_element_boxes(_p(coords), d, dr, N, NE, tol, M, _p(aabb), _p(obb_c), _p(obb_A))
    assert rc == 0, rc
    return aabb, obb_c, obb_A


class OracleMesh:
    """Coordinates plus the oracle's own boxes (Setup, Sec. 3.1)."""

    def __init__(self, coords, d: int, dr: int, N: int, tol: float = 0.1, M: int = 0,
                 newton_tol: float = 1e-10, max_iter: int = 50, dist_tol: float = 1e-10):
        self.coords = _f64(coords)
        self.d, self.dr, self.N = d, dr, N
        self.NE = self.coords.size // (d * N ** dr)
        self.newton_tol, self.max_iter, self.dist_tol = newton_tol, max_iter, dist_tol
        self.aabb, self.obb_c, self.obb_A = element_boxes(self.coords, d, dr, N, tol, M)

    def findpts(self, pts, stats=None):
        pts = _f64(pts).reshape(-1, self.d)
        n = pts.shape[0]
        code = np.zeros(n, np.int32)
        elem = np.zeros(n, np.int32)
        r = np.zeros((n, self.dr))
        dist2 = np.zeros(n)
        st = np.zeros(8, np.int64) if stats is None else stats
        rc = lib().or_findpts(_p(self.coords), self.d, self.dr, self.N, self.NE, _p(self.aabb),
                              _p(self.obb_c), _p(self.obb_A), _p(pts), n, self.newton_tol,
                              self.max_iter, self.dist_tol, _p(code, _I32), _p(elem, _I32),
                              _p(r), _p(dist2), _p(st, _I64))
        assert rc == 0
        return code, elem, r, dist2

    def newton(self, e: int, xs, stats=None):
        xs = _f64(xs)
        r = np.zeros(self.dr)
        dist2 = _dbl()
        st = np.zeros(8, np.int64) if stats is None else stats
        it = lib().or_newton(_p(self.coords), self.d, self.dr, self.N, self.NE, int(e), _p(xs),
                             self.newton_tol, self.max_iter, _p(r), ctypes.byref(dist2), _p(st, _I64))
        return r, dist2.value, it

    def locate_in_element(self, e: int, pts):
        pts = _f64(pts).reshape(-1, self.d)
        n = pts.shape[0]
        code = np.zeros(n, np.int32)
        r = np.zeros((n, self.dr))
        dist2 = np.zeros(n)
        assert lib().or_locate_in_element(_p(self.coords), self.d, self.dr, self.N, self.NE, int(e),
                                          _p(pts), n, self.newton_tol, self.max_iter, self.dist_tol,
                                          _p(code, _I32), _p(r), _p(dist2)) == 0
        return code, r, dist2

    def box_candidates(self, pts):
        pts = _f64(pts).reshape(-1, self.d)
        n = pts.shape[0]
        count = np.zeros(n, np.int32)
        first = np.zeros(n, np.int32)
        assert lib().or_box_candidates(self.d, self.NE, _p(self.aabb), _p(self.obb_c), _p(self.obb_A),
                                       _p(pts), n, _p(count, _I32), _p(first, _I32)) == 0
        return count, first

    def eval(self, field, code, elem, r, field_N=None):
        """Eq. u_tensor: the field on field_N GLL nodes per direction (the
        mesh's N unless given; Sec. 2 allows the two to differ)."""
        Nf = self.N if field_N is None else int(field_N)
        field = _f64(field)
        nc = field.size // (self.NE * Nf ** self.dr)
        code, elem, r = _i32(code), _i32(elem), _f64(r)
        n = code.shape[0]
        out = np.zeros((nc, n))
        assert lib().or_eval(_p(field), nc, self.dr, Nf, self.NE, _p(code, _I32), _p(elem, _I32),
                             _p(r), n, _p(out)) == 0
        return out

    def forward_map(self, elem, r, jacobian: bool = False):
        elem, r = _i32(elem), _f64(r).reshape(-1, self.dr)
        n = elem.shape[0]
        x = np.zeros((n, self.d))
        jac = np.zeros((n, self.d, self.dr)) if jacobian else None
        assert lib().or_forward_map(_p(self.coords), self.d, self.dr, self.N, self.NE, _p(elem, _I32),
                                    _p(r), n, _p(x), _p(jac)) == 0
        return (x, jac) if jacobian else x
