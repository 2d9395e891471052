"""Pins of the oracle's setup arithmetic (Sec. 2 and Sec. 3.1.1) against closed
forms, library routines and the paper's printed values — never against the
oracle itself."""
from pathlib import Path

import numpy as np
import pytest
from numpy.polynomial import legendre as L
from numpy.polynomial import polynomial as P

import oracle

GOLDEN = Path(__file__).parent / "golden"


def lagrange_poly(z, i):
    """Coefficients of the i-th Lagrange interpolant on nodes z (numpy)."""
    e = np.zeros(len(z))
    e[i] = 1.0
    return P.polyfit(z, e, len(z) - 1)


@pytest.mark.parametrize("N,expected", [
    (2, [-1, 1]),
    (3, [-1, 0, 1]),
    (4, [-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1]),
    (5, [-1, -np.sqrt(3 / 7), 0, np.sqrt(3 / 7), 1]),
    (6, [-1, -np.sqrt((7 + 2 * np.sqrt(7)) / 21), -np.sqrt((7 - 2 * np.sqrt(7)) / 21),
         np.sqrt((7 - 2 * np.sqrt(7)) / 21), np.sqrt((7 + 2 * np.sqrt(7)) / 21), 1]),
])
def test_gll_closed_forms(N, expected):
    np.testing.assert_allclose(oracle.gll_nodes(N), expected, rtol=0, atol=2e-16)


@pytest.mark.parametrize("N", range(2, 17))
def test_gll_quadrature_exactness(N):
    """GLL weights 2/(n(n+1) P_n(z)^2) (numpy legval) integrate x^k exactly
    for k <= 2N-3: a misplaced node breaks this."""
    z = oracle.gll_nodes(N)
    n = N - 1
    c = np.zeros(N)
    c[-1] = 1
    w = 2.0 / (n * (n + 1) * L.legval(z, c) ** 2)
    for k in range(2 * N - 2):
        exact = (1 - (-1) ** (k + 1)) / (k + 1)
        assert abs(np.sum(w * z ** k) - exact) < 1e-13
    assert np.all(np.diff(z) > 0)
    np.testing.assert_allclose(z, -z[::-1], atol=1e-15)


@pytest.mark.parametrize("m", [1, 2, 5, 9, 12])
def test_gauss_legendre_vs_numpy(m):
    x, w = oracle.gauss_legendre(m)
    xr, wr = L.leggauss(m)
    np.testing.assert_allclose(np.sort(x), xr, atol=1e-14)
    np.testing.assert_allclose(w[np.argsort(x)], wr, atol=1e-14)


@pytest.mark.parametrize("N", [2, 3, 5, 8, 12])
def test_lagrange_identities_and_numpy(N):
    z = oracle.gll_nodes(N)
    for j in range(N):
        phi, _, _ = oracle.lagrange(N, z[j])
        np.testing.assert_allclose(phi, np.eye(N)[j], atol=1e-14)
    rng = np.random.default_rng(0)
    for r in rng.uniform(-1, 1, 7):
        phi, dphi, d2phi = oracle.lagrange(N, r)
        assert abs(phi.sum() - 1) < 1e-13
        assert abs(dphi.sum()) < 1e-11
        assert abs(d2phi.sum()) < 1e-9
        assert abs((z * phi).sum() - r) < 1e-13
        assert abs((z * dphi).sum() - 1) < 1e-11
        if N >= 3:
            assert abs((z ** 2 * d2phi).sum() - 2) < 1e-9
        for i in range(N):
            c = lagrange_poly(z, i)
            assert abs(P.polyval(r, c) - phi[i]) < 1e-10
            assert abs(P.polyval(r, P.polyder(c)) - dphi[i]) < 1e-8
            assert abs(P.polyval(r, P.polyder(c, 2)) - d2phi[i]) < 1e-6


def test_chebyshev_points_closed_form():
    np.testing.assert_allclose(oracle.chebyshev_points(2), [-1, 1], atol=1e-16)
    np.testing.assert_allclose(oracle.chebyshev_points(3), [-1, 0, 1], atol=1e-16)
    np.testing.assert_allclose(oracle.chebyshev_points(5),
                               [-1, -np.sqrt(0.5), 0, np.sqrt(0.5), 1], atol=1e-15)


def _bounds_contain(N, M, reading, ns=20001):
    z = oracle.gll_nodes(N)
    eta = -np.cos(np.arange(M) * np.pi / (M - 1))
    lo, hi = oracle.basis_bounds(N, M, reading)
    x = np.linspace(-1, 1, ns)
    for i in range(N):
        f = P.polyval(x, lagrange_poly(z, i))
        if np.any(f < np.interp(x, eta, lo[i]) - 1e-12) or np.any(f > np.interp(x, eta, hi[i]) + 1e-12):
            return False
    return True


def _golden_mmin():
    rows = [l.split() for l in (GOLDEN / "mmin_footnote.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    return [(int(a), int(b)) for a, b in rows]


def test_mmin_footnote_reading():
    """The half-interval tangent reading of Eq. 1D_bases_bounds_2 reproduces
    the footnote's M_min(N) table exactly; the literal full-interval text
    does not (it gives different, smaller values)."""
    table = _golden_mmin()
    for N, mmin in table:
        assert _bounds_contain(N, mmin, 0), (N, mmin)
        if mmin > 2:
            assert not _bounds_contain(N, mmin - 1, 0), (N, mmin)
    mismatches = 0
    for N, mmin in table:
        M = 2
        while not _bounds_contain(N, M, 1):
            M += 1
        mismatches += (M != mmin)
    assert mismatches >= 5


@pytest.mark.parametrize("N", range(2, 9))
def test_default_M_2N_bounds_bases(N):
    """Sec. 3.1.1: M = 2N (the default) bounds the bases for these orders."""
    assert _bounds_contain(N, 2 * N, 0)


@pytest.mark.parametrize("N", [2, 3, 4, 6, 8])
def test_legendre_coeffs(N):
    """a_l = (2l+1)/2 int u P_l: exact for linear u (w = 0) and equal to
    numpy's Legendre projection of the interpolant."""
    z = oracle.gll_nodes(N)
    c0, c1 = oracle.legendre_coeffs(N)
    u = 0.3 - 1.7 * z
    assert abs(c0 @ u - 0.3) < 1e-14 and abs(c1 @ u + 1.7) < 1e-14
    rng = np.random.default_rng(N)
    u = rng.uniform(-1, 1, N)
    leg = L.legfit(z, u, N - 1)
    assert abs(c0 @ u - leg[0]) < 1e-13
    if N >= 2:
        assert abs(c1 @ u - leg[1]) < 1e-13


def _dense_1d(u, ns=20001):
    N = len(u)
    z = oracle.gll_nodes(N)
    c = L.legfit(z, u, N - 1)
    return L.legval(np.linspace(-1, 1, ns), c)


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 8])
def test_bound_1d_contains_and_linear_exact(N):
    rng = np.random.default_rng(10 + N)
    for _ in range(20):
        u = rng.uniform(-1, 1, N)
        lo, hi = oracle.bound_1d(u, 2 * N)
        f = _dense_1d(u)
        assert lo <= f.min() + 1e-12 and hi >= f.max() - 1e-12
    z = oracle.gll_nodes(N)
    u = 0.25 + 0.5 * z
    lo, hi = oracle.bound_1d(u, 2 * N)
    assert abs(lo + 0.25) < 1e-14 and abs(hi - 0.75) < 1e-14


def test_bound_1d_fig3_cubic_tightens_with_M():
    rows = {l.split()[0]: [float(v) for v in l.split()[1:]]
            for l in (GOLDEN / "fig3_cubic.txt").read_text().splitlines() if l.strip() and not l.startswith("#")}
    u = np.array(rows["u"])
    f = _dense_1d(u)
    widths = []
    for M in map(int, rows["M"]):
        lo, hi = oracle.bound_1d(u, M)
        assert lo <= f.min() + 1e-13 and hi >= f.max() - 1e-13
        widths.append(hi - lo)
    assert widths[0] >= widths[1] >= widths[2]
    assert widths[2] < 1.1 * (f.max() - f.min())


@pytest.mark.parametrize("N", [2, 3, 4, 5, 7])
def test_bound_2d_contains_and_linear_exact(N):
    rng = np.random.default_rng(20 + N)
    z = oracle.gll_nodes(N)
    ns = 301
    x = np.linspace(-1, 1, ns)
    basis = np.stack([P.polyval(x, lagrange_poly(z, i)) for i in range(N)])  # [N][ns]
    for _ in range(5):
        u = rng.uniform(-1, 1, (N, N))  # u[b][a]
        lo, hi = oracle.bound_2d(u, 2 * N)
        f = np.einsum("ba,ar,bs->rs", u, basis, basis)
        assert lo <= f.min() + 1e-12 and hi >= f.max() - 1e-12
    A, B = np.meshgrid(z, z)  # A[b][a] = z_a, B[b][a] = z_b
    u = 0.1 + 0.2 * A - 0.3 * B
    lo, hi = oracle.bound_2d(u, 2 * N)
    assert abs(lo - (0.1 - 0.2 - 0.3)) < 1e-13 and abs(hi - (0.1 + 0.2 + 0.3)) < 1e-13
