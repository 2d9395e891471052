/*
 * FP64 CPU oracle for local findpts — TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load this file's library.  It is a plain restatement of the method of
 * arXiv 2501.12349 in FP64, written for a reader checking it against the
 * paper: every basis sum is the direct sum over all nodes (no sum
 * factorisation), candidates come from a brute-force box test over every
 * element (no hash grid), and each function names the passage it follows.
 * Where the paper is silent or garbled, the reading taken is stated at the
 * point of use.  Parallelism: OpenMP over points only.
 */
#define _GNU_SOURCE
#include "oracle.h"

#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Sec. 2: Gauss-Lobatto-Legendre nodes zeta_1..zeta_N (the paper names them
 * but is silent on how to compute them).  They are -1, +1 and the N-2 roots
 * of P'_{N-1}.  Legendre values and derivatives come from the three-term
 * recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} together with
 * P'_{k+1} = P'_{k-1} + (2k+1) P_k and P''_{k+1} = P''_{k-1} + (2k+1) P'_k;
 * interior roots by Newton from the Chebyshev-Gauss-Lobatto points.         */
static void legendre_all(int n, double x, double* P, double* dP, double* d2P) {
  /* returns P_n(x), P'_n(x), P''_n(x) */
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0, s0 = 0.0, s1 = 0.0;
  if (n == 0) {
    *P = 1.0; *dP = 0.0; *d2P = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    double d2 = d0 + (2.0 * k + 1.0) * p1;
    double s2 = s0 + (2.0 * k + 1.0) * d1;
    p0 = p1; p1 = p2;
    d0 = d1; d1 = d2;
    s0 = s1; s1 = s2;
  }
  *P = p1; *dP = d1; *d2P = s1;
}

int or_gll_nodes(int N, double* z) {
  if (N < 2 || N > OR_MAXN) return -1;
  const int n = N - 1;
  z[0] = -1.0;
  z[N - 1] = 1.0;
  for (int j = 1; j < N - 1; ++j) {
    double x = -cos(M_PI * j / n);
    for (int it = 0; it < 100; ++it) {
      double P, dP, d2P;
      legendre_all(n, x, &P, &dP, &d2P);
      double dx = dP / d2P;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    z[j] = x;
  }
  return 0;
}

/* Gauss-Legendre rule with m points (roots of P_m); used only to evaluate
 * the Legendre projections of Sec. 3.1.1 exactly. */
int or_gauss_legendre(int m, double* x, double* w) {
  if (m < 1 || m > OR_MAXN + 2) return -1;
  for (int j = 0; j < m; ++j) {
    double t = -cos(M_PI * (j + 0.75) / (m + 0.5));
    double P = 0, dP = 1, d2P = 0;
    for (int it = 0; it < 100; ++it) {
      legendre_all(m, t, &P, &dP, &d2P);
      double dt = P / dP;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    legendre_all(m, t, &P, &dP, &d2P);
    x[j] = t;
    w[j] = 2.0 / ((1.0 - t * t) * dP * dP);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2, Eq. x: Lagrange interpolants phi_i on the GLL nodes, phi_i(zeta_j)
 * = delta_ij, in plain product form phi_i(r) = prod_{m!=i} (r - z_m)/(z_i - z_m),
 * with first and second derivatives by the product rule (each term drops one
 * or two factors).  Any output pointer may be NULL.                          */
void or_lagrange(int N, const double* z, double r, double* phi, double* dphi, double* d2phi) {
  for (int i = 0; i < N; ++i) {
    if (phi) {
      double p = 1.0;
      for (int m = 0; m < N; ++m)
        if (m != i) p *= (r - z[m]) / (z[i] - z[m]);
      phi[i] = p;
    }
    if (dphi) {
      double s = 0.0;
      for (int m = 0; m < N; ++m) {
        if (m == i) continue;
        double p = 1.0 / (z[i] - z[m]);
        for (int q = 0; q < N; ++q)
          if (q != i && q != m) p *= (r - z[q]) / (z[i] - z[q]);
        s += p;
      }
      dphi[i] = s;
    }
    if (d2phi) {
      double s = 0.0;
      for (int m = 0; m < N; ++m) {
        if (m == i) continue;
        for (int q = 0; q < N; ++q) {
          if (q == i || q == m) continue;
          double p = 1.0 / ((z[i] - z[m]) * (z[i] - z[q]));
          for (int t = 0; t < N; ++t)
            if (t != i && t != m && t != q) p *= (r - z[t]) / (z[i] - z[t]);
          s += p;
        }
      }
      d2phi[i] = s;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1.1, Eq. chebyshev: eta_j = -cos((j-1) pi / (M-1)), j = 1..M.      */
void or_chebyshev_points(int M, double* eta) {
  for (int j = 0; j < M; ++j) eta[j] = -cos(M_PI * (double)j / (double)(M - 1));
}

/* Sec. 3.1.1, Eqs. 1D_bases_bounds(_2,_3): piecewise-linear lower / upper
 * bounds vlo[i][j], vhi[i][j] (i basis, j Chebyshev point, row-major N x M)
 * of the basis functions.  At the end points the bound is the basis value
 * itself (the paper's "delta_ij" there is read as phi_i(-1) = delta_{i,1},
 * phi_i(+1) = delta_{i,N}).  At an interior point the candidate values are
 * the basis value and the two tangent lines taken at the neighbouring
 * interval midpoints eta_{j-} and eta_{j+}, evaluated at eta_j.
 * reading = 0: the tangent is evaluated at its geometric distance from the
 *   midpoint, (eta_j - eta_{j-}) and (eta_{j+} - eta_j) — this reading
 *   reproduces the paper's footnote table of M_min(N) exactly.
 * reading = 1: the literal garbled text, (eta_j - eta_{j-1}) and
 *   (eta_{j+1} - eta_j); kept only so the tests can show it does not.        */
int or_basis_bounds(int N, int M, int reading, double* vlo, double* vhi) {
  if (N < 2 || N > OR_MAXN || M < 2 || M > OR_MAXM) return -1;
  double z[OR_MAXN], eta[OR_MAXM];
  or_gll_nodes(N, z);
  or_chebyshev_points(M, eta);
  double phi[OR_MAXN], dphi[OR_MAXN];
  double phim[OR_MAXN], dphim[OR_MAXN], phip[OR_MAXN], dphip[OR_MAXN];
  for (int j = 0; j < M; ++j) {
    or_lagrange(N, z, eta[j], phi, dphi, NULL);
    if (j == 0 || j == M - 1) {
      for (int i = 0; i < N; ++i) {
        double v = (j == 0) ? (i == 0 ? 1.0 : 0.0) : (i == N - 1 ? 1.0 : 0.0);
        vlo[i * M + j] = v;
        vhi[i * M + j] = v;
      }
      continue;
    }
    double em = 0.5 * (eta[j] + eta[j - 1]);
    double ep = 0.5 * (eta[j] + eta[j + 1]);
    or_lagrange(N, z, em, phim, dphim, NULL);
    or_lagrange(N, z, ep, phip, dphip, NULL);
    double dm = (reading == 0) ? (eta[j] - em) : (eta[j] - eta[j - 1]);
    double dp = (reading == 0) ? (ep - eta[j]) : (eta[j + 1] - eta[j]);
    for (int i = 0; i < N; ++i) {
      double v0 = phi[i];
      double v1 = phim[i] + dm * dphim[i];
      double v2 = phip[i] - dp * dphip[i];
      double lo = v0, hi = v0;
      if (v1 < lo) lo = v1;
      if (v2 < lo) lo = v2;
      if (v1 > hi) hi = v1;
      if (v2 > hi) hi = v2;
      vlo[i * M + j] = lo;
      vhi[i * M + j] = hi;
    }
  }
  return 0;
}

/* Sec. 3.1.1: coefficients of the two-term Legendre truncation,
 * a_l = (2l+1)/2 * int_{-1}^{1} u(r) P_l(r) dr = sum_i c_l[i] u_i with
 * c_l[i] = (2l+1)/2 * int phi_i P_l.  The integral is evaluated exactly with
 * an (N+1)-point Gauss-Legendre rule (the paper is silent on quadrature).   */
int or_legendre_coeffs(int N, double* c0, double* c1) {
  double z[OR_MAXN], xq[OR_MAXN + 2], wq[OR_MAXN + 2], phi[OR_MAXN];
  if (or_gll_nodes(N, z)) return -1;
  const int m = N + 1;
  or_gauss_legendre(m, xq, wq);
  for (int i = 0; i < N; ++i) c0[i] = c1[i] = 0.0;
  for (int q = 0; q < m; ++q) {
    or_lagrange(N, z, xq[q], phi, NULL, NULL);
    for (int i = 0; i < N; ++i) {
      c0[i] += 0.5 * wq[q] * phi[i];          /* P_0 = 1 */
      c1[i] += 1.5 * wq[q] * phi[i] * xq[q];  /* P_1 = r */
    }
  }
  return 0;
}

/* Sec. 3.1.1, Eqs. 1D_bound_final_1/2: bounds of u(r) = sum_i u_i phi_i(r)
 * on [-1,1].  u is written as a0 + a1 r + sum_i w_i phi_i(r) with
 * w_i = u_i - a0 - a1 zeta_i; the lower / upper bound functions are
 * evaluated at the M Chebyshev points and the overall bound is their
 * minimum / maximum.                                                         */
int or_bound_1d(int N, int M, const double* u, double* lo, double* hi) {
  double z[OR_MAXN], eta[OR_MAXM], c0[OR_MAXN], c1[OR_MAXN];
  double vlo[OR_MAXN * OR_MAXM], vhi[OR_MAXN * OR_MAXM];
  if (or_basis_bounds(N, M, 0, vlo, vhi)) return -1;
  or_gll_nodes(N, z);
  or_chebyshev_points(M, eta);
  or_legendre_coeffs(N, c0, c1);
  double a0 = 0.0, a1 = 0.0;
  for (int i = 0; i < N; ++i) {
    a0 += c0[i] * u[i];
    a1 += c1[i] * u[i];
  }
  double w[OR_MAXN];
  for (int i = 0; i < N; ++i) w[i] = u[i] - a0 - a1 * z[i];
  double L = INFINITY, H = -INFINITY;
  for (int j = 0; j < M; ++j) {
    double l = a0 + a1 * eta[j], h = l;
    for (int i = 0; i < N; ++i) {
      double p = w[i] * vlo[i * M + j], q = w[i] * vhi[i * M + j];
      l += (p < q) ? p : q;
      h += (p > q) ? p : q;
    }
    if (l < L) L = l;
    if (h > H) H = h;
  }
  *lo = L;
  *hi = H;
  return 0;
}

/* Sec. 3.1.1, Eqs. 2D_function_bound_1/2: bounds of
 * u(r,s) = sum_{a,b} u_ab phi_a(r) phi_b(s) on [-1,1]^2 (u[a + N*b]), as the
 * plain O(N^2 M^2) double sum of the min / max of the four products of the
 * basis bounds at each Chebyshev grid point (eta_k, eta_l).  The paper
 * compacts only the 1D bound with a Legendre truncation; the reading taken in
 * 2D is the analogous total-degree-1 truncation a00 + a10 r + a01 s, with
 * w_ab = u_ab - a00 - a10 zeta_a - a01 zeta_b.                              */
int or_bound_2d(int N, int M, const double* u, double* lo, double* hi) {
  double z[OR_MAXN], eta[OR_MAXM], c0[OR_MAXN], c1[OR_MAXN];
  double vlo[OR_MAXN * OR_MAXM], vhi[OR_MAXN * OR_MAXM];
  if (or_basis_bounds(N, M, 0, vlo, vhi)) return -1;
  or_gll_nodes(N, z);
  or_chebyshev_points(M, eta);
  or_legendre_coeffs(N, c0, c1);
  double a00 = 0.0, a10 = 0.0, a01 = 0.0;
  for (int b = 0; b < N; ++b)
    for (int a = 0; a < N; ++a) {
      double v = u[a + N * b];
      a00 += c0[a] * c0[b] * v;
      a10 += c1[a] * c0[b] * v;
      a01 += c0[a] * c1[b] * v;
    }
  double w[OR_MAXN * OR_MAXN];
  for (int b = 0; b < N; ++b)
    for (int a = 0; a < N; ++a) w[a + N * b] = u[a + N * b] - a00 - a10 * z[a] - a01 * z[b];
  double L = INFINITY, H = -INFINITY;
  for (int l = 0; l < M; ++l)
    for (int k = 0; k < M; ++k) {
      double lsum = a00 + a10 * eta[k] + a01 * eta[l], hsum = lsum;
      for (int b = 0; b < N; ++b)
        for (int a = 0; a < N; ++a) {
          double wab = w[a + N * b];
          double ra[2] = {vlo[a * M + k], vhi[a * M + k]};
          double sb[2] = {vlo[b * M + l], vhi[b * M + l]};
          double mn = INFINITY, mx = -INFINITY;
          for (int x = 0; x < 2; ++x)
            for (int y = 0; y < 2; ++y) {
              double t = wab * ra[x] * sb[y];
              if (t < mn) mn = t;
              if (t > mx) mx = t;
            }
          lsum += mn;
          hsum += mx;
        }
      if (lsum < L) L = lsum;
      if (hsum > H) H = hsum;
    }
  *lo = L;
  *hi = H;
  return 0;
}

/* N^dr: nodes of a tensor-product element (lines, quads, hexes). */
static int nodes_per_elem(int N, int dr) { return dr == 1 ? N : (dr == 2 ? N * N : N * N * N); }

/* ------------------------------------------------------------------------ */
/* Direct evaluation of the element map, Eq. x / x_tensor: x_c(r) and, when
 * requested, G[c][j] = dx_c/dr_j (Eq. jacobian) and the second derivatives
 * S[c][j][k] = d^2 x_c / dr_j dr_k, as plain sums over all N^dr nodes.      */
static void eval_map(const double* coords, int d, int dr, int N, int64_t NE, int64_t e,
                     const double* z, const double* r, double* x, double* G, double* S) {
  double phi[3][OR_MAXN], dphi[3][OR_MAXN], d2phi[3][OR_MAXN];
  for (int j = 0; j < dr; ++j) or_lagrange(N, z, r[j], phi[j], dphi[j], d2phi[j]);
  const int ne = nodes_per_elem(N, dr);
  for (int c = 0; c < d; ++c) {
    x[c] = 0.0;
    if (G)
      for (int j = 0; j < dr; ++j) G[c * dr + j] = 0.0;
    if (S)
      for (int j = 0; j < dr * dr; ++j) S[c * dr * dr + j] = 0.0;
  }
  for (int n = 0; n < ne; ++n) {
    int idx[3] = {n % N, (n / N) % N, n / (N * N)};
    /* value and derivatives of the tensor-product basis function of node n */
    double B = 1.0, dB[3], d2B[3][3];
    for (int j = 0; j < dr; ++j) B *= phi[j][idx[j]];
    for (int j = 0; j < dr; ++j) {
      double t = 1.0;
      for (int q = 0; q < dr; ++q) t *= (q == j) ? dphi[q][idx[q]] : phi[q][idx[q]];
      dB[j] = t;
      for (int k = 0; k < dr; ++k) {
        double s = 1.0;
        for (int q = 0; q < dr; ++q) {
          if (q == j && q == k) s *= d2phi[q][idx[q]];
          else if (q == j || q == k) s *= dphi[q][idx[q]];
          else s *= phi[q][idx[q]];
        }
        d2B[j][k] = s;
      }
    }
    for (int c = 0; c < d; ++c) {
      double xn = coords[((int64_t)c * NE + e) * ne + n];
      x[c] += xn * B;
      if (G)
        for (int j = 0; j < dr; ++j) G[c * dr + j] += xn * dB[j];
      if (S)
        for (int j = 0; j < dr; ++j)
          for (int k = 0; k < dr; ++k) S[(c * dr + j) * dr + k] += xn * d2B[j][k];
    }
  }
}

/* 3x3 (or 2x2) inverse by cofactors; returns the determinant. */
static double inv_small(int d, const double* A, double* Ai) {
  if (d == 2) {
    double det = A[0] * A[3] - A[1] * A[2];
    Ai[0] = A[3] / det; Ai[1] = -A[1] / det;
    Ai[2] = -A[2] / det; Ai[3] = A[0] / det;
    return det;
  }
  double c00 = A[4] * A[8] - A[5] * A[7];
  double c01 = A[5] * A[6] - A[3] * A[8];
  double c02 = A[3] * A[7] - A[4] * A[6];
  double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  Ai[0] = c00 / det;
  Ai[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  Ai[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  Ai[3] = c01 / det;
  Ai[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  Ai[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  Ai[6] = c02 / det;
  Ai[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  Ai[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  return det;
}

/* Bounds of one scalar nodal function u[n] (n over the element's nodes) over
 * the element.  Volume elements: union of the bounds on the boundary pieces —
 * the 4 edges of a quad (Sec. 3.1.1, 1D bounds) or the 6 faces of a hex
 * (2D bounds); for a bijective map the extremes lie on the boundary.
 * Surface quads (Sec. 4.1): the element itself is a 2D function.           */
static void element_bounds(const double* u, int d, int dr, int N, int M, double* lo, double* hi) {
  double L = INFINITY, H = -INFINITY, l, h;
  double piece[OR_MAXN * OR_MAXN];
  if (dr == 1) {
    /* line elements (Sec. 2, Eq. x_tensor_surf): the element is a 1D function */
    or_bound_1d(N, M, u, &l, &h);
    *lo = l;
    *hi = h;
    return;
  }
  if (dr == 2 && d == 3) {
    or_bound_2d(N, M, u, &l, &h);
    *lo = l;
    *hi = h;
    return;
  }
  if (dr == 2) {
    for (int side = 0; side < 4; ++side) {
      for (int a = 0; a < N; ++a) {
        int i, j;
        if (side == 0) { i = a; j = 0; }
        else if (side == 1) { i = a; j = N - 1; }
        else if (side == 2) { i = 0; j = a; }
        else { i = N - 1; j = a; }
        piece[a] = u[i + N * j];
      }
      or_bound_1d(N, M, piece, &l, &h);
      if (l < L) L = l;
      if (h > H) H = h;
    }
  } else {
    for (int face = 0; face < 6; ++face) {
      int fixed = face / 2, val = (face % 2) ? N - 1 : 0;
      for (int b = 0; b < N; ++b)
        for (int a = 0; a < N; ++a) {
          int i, j, k;
          if (fixed == 0) { i = val; j = a; k = b; }
          else if (fixed == 1) { i = a; j = val; k = b; }
          else { i = a; j = b; k = val; }
          piece[a + N * b] = u[i + N * (j + N * k)];
        }
      or_bound_2d(N, M, piece, &l, &h);
      if (l < L) L = l;
      if (h > H) H = h;
    }
  }
  *lo = L;
  *hi = H;
}

/* Expansion of a box with raw extents (Sec. 3.1.1: "expanded by a nominal
 * percentage", 10% by default; Sec. 4.1 for zero extents).  Reading: the
 * extent L of each direction grows to (1+tol) L, tol*L/2 on each side.  A
 * direction whose extent is zero (L <= 1e-12 * max L, a flat element aligned
 * with that axis) is padded by tol * Lmin / 2 on each side, Lmin the smallest
 * extent of the other directions.  Returns the half-widths of the expanded
 * box in hw[] and its centre in mid[].                                       */
static void expand_box(int d, const double* lo, const double* hi, double tol, double* mid,
                       double* hw) {
  double Lmax = 0.0;
  for (int c = 0; c < d; ++c)
    if (hi[c] - lo[c] > Lmax) Lmax = hi[c] - lo[c];
  double Lmin = INFINITY;
  for (int c = 0; c < d; ++c) {
    double L = hi[c] - lo[c];
    if (L > 1e-12 * Lmax && L < Lmin) Lmin = L;
  }
  for (int c = 0; c < d; ++c) {
    double L = hi[c] - lo[c];
    double pad = (L > 1e-12 * Lmax) ? 0.5 * tol * L : 0.5 * tol * Lmin;
    if (!(pad == pad) || pad == INFINITY) pad = 0.0;
    mid[c] = 0.5 * (lo[c] + hi[c]);
    hw[c] = 0.5 * L + pad;
  }
}

/* Orientation frame of a surface quad, Sec. 4.2: with t1, t2 the tangents at
 * r = 0 and n = t1 x t2, R1 is the Rodrigues rotation taking n/|n| to the z
 * axis and R2 = [R1 t1, R1 t2, e3]^{-1} (columns); the frame is R = R2 R1.   */
static void surface_frame(const double* Jc /* 3x2 */, double* R1out, double* R) {
  double t1[3] = {Jc[0], Jc[2], Jc[4]}, t2[3] = {Jc[1], Jc[3], Jc[5]};
  double n[3] = {t1[1] * t2[2] - t1[2] * t2[1], t1[2] * t2[0] - t1[0] * t2[2],
                 t1[0] * t2[1] - t1[1] * t2[0]};
  double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  for (int c = 0; c < 3; ++c) n[c] /= nn;
  /* axis k = n x e3, sin = |k|, cos = n . e3 */
  double v[3] = {n[1], -n[0], 0.0};
  double s = sqrt(v[0] * v[0] + v[1] * v[1]), co = n[2];
  double R1[9];
  if (s == 0.0) {
    for (int i = 0; i < 9; ++i) R1[i] = 0.0;
    R1[0] = 1.0;
    R1[4] = (co > 0) ? 1.0 : -1.0;
    R1[8] = (co > 0) ? 1.0 : -1.0;
  } else {
    double k[3] = {v[0] / s, v[1] / s, 0.0};
    double K[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0};
    double K2[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double t = 0;
        for (int q = 0; q < 3; ++q) t += K[i * 3 + q] * K[q * 3 + j];
        K2[i * 3 + j] = t;
      }
    for (int i = 0; i < 9; ++i) R1[i] = ((i % 4) == 0 ? 1.0 : 0.0) + s * K[i] + (1.0 - co) * K2[i];
  }
  double a[3], b[3];
  for (int i = 0; i < 3; ++i) {
    a[i] = R1[i * 3 + 0] * t1[0] + R1[i * 3 + 1] * t1[1] + R1[i * 3 + 2] * t1[2];
    b[i] = R1[i * 3 + 0] * t2[0] + R1[i * 3 + 1] * t2[1] + R1[i * 3 + 2] * t2[2];
  }
  if (R1out)
    for (int i = 0; i < 9; ++i) R1out[i] = R1[i];
  double Mc[9] = {a[0], b[0], 0.0, a[1], b[1], 0.0, a[2], b[2], 1.0}, R2[9];
  inv_small(3, Mc, R2);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double t = 0;
      for (int q = 0; q < 3; ++q) t += R2[i * 3 + q] * R1[q * 3 + j];
      R[i * 3 + j] = t;
    }
}

/* Orientation frame of a line element, Sec. 4.2: the Rodrigues rotation R
 * that takes the unit tangent t/|t| at r = 0 to the x axis (2D: the plane
 * rotation by minus the tangent's angle; 3D: rotation about t x e1 by the
 * angle between t and e1; a tangent along -e1 turns by pi about e3).        */
static void line_frame(int d, const double* t, double* R) {
  double nt = 0.0;
  for (int c = 0; c < d; ++c) nt += t[c] * t[c];
  nt = sqrt(nt);
  double u[3] = {0.0, 0.0, 0.0};
  for (int c = 0; c < d; ++c) u[c] = t[c] / nt;
  if (d == 2) {
    R[0] = u[0];
    R[1] = u[1];
    R[2] = -u[1];
    R[3] = u[0];
    return;
  }
  /* axis k = u x e1 = (0, u2, -u1), sin = |k|, cos = u . e1 */
  double v[3] = {0.0, u[2], -u[1]};
  double s = sqrt(v[1] * v[1] + v[2] * v[2]), co = u[0];
  if (s == 0.0) {
    for (int i = 0; i < 9; ++i) R[i] = 0.0;
    R[0] = (co > 0) ? 1.0 : -1.0;
    R[4] = (co > 0) ? 1.0 : -1.0;
    R[8] = 1.0;
    return;
  }
  double k[3] = {0.0, v[1] / s, v[2] / s};
  double K[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0};
  double K2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double q = 0;
      for (int m = 0; m < 3; ++m) q += K[i * 3 + m] * K[m * 3 + j];
      K2[i * 3 + j] = q;
    }
  for (int i = 0; i < 9; ++i) R[i] = ((i % 4) == 0 ? 1.0 : 0.0) + s * K[i] + (1.0 - co) * K2[i];
}

/* The surface frame of Sec. 4.2 for a 3x2 Jacobian J_c at r = 0 (row-major,
 * J_c[c][j] = dx_c/dr_j): R1 (the Rodrigues rotation) and R = R2 R1, both
 * 3x3 row-major.  Exported for the tests; element boxes use the same call. */
int or_surface_frame(const double* Jc, double* R1, double* R) {
  surface_frame(Jc, R1, R);
  return 0;
}

/* Secs. 3.1.1-3.1.2 and 4.1-4.2: the expanded AABB and OBB of every element.
 * AABB: bounds of each coordinate function (element_bounds), expanded.
 * OBB: x_c = x(r=0), J_c = G(r=0); the nodes are mapped to the frame
 * x~ = T (x - x_c) with T = J_c^{-1} (volumes, Eq. OBB_transformation) or
 * T = R (surface quads: R2 R1; lines: the Rodrigues rotation); the AABB of x~ (centre m, expanded half-widths hw) is
 * mapped back: OBB centre x_c + T^{-1} m (the paper's x_c + J_c x_c-breve),
 * and the stored matrix A = diag(1/hw) T is J-acute^{-1}, so the test of
 * Eq. OBB_test is |A (x* - centre)|_inf <= 1.                              */
int or_element_boxes(const double* coords, int d, int dr, int N, int64_t NE, double tol,
                     int M, double* aabb, double* obb_c, double* obb_A) {
  if (!((d == 2 && dr == 2) || (d == 3 && dr == 3) || (d == 3 && dr == 2) || (dr == 1 && (d == 2 || d == 3))))
    return -1;
  if (N < 2 || N > OR_MAXN || M < 2 || M > OR_MAXM) return -1;
  const int ne = nodes_per_elem(N, dr);
  double z[OR_MAXN];
  or_gll_nodes(N, z);
  int err = 0;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t e = 0; e < NE; ++e) {
    double* u = (double*)malloc(sizeof(double) * ne * d);
    double lo[3], hi[3], mid[3], hw[3];
    for (int c = 0; c < d; ++c) {
      for (int n = 0; n < ne; ++n) u[c * ne + n] = coords[((int64_t)c * NE + e) * ne + n];
      element_bounds(u + c * ne, d, dr, N, M, &lo[c], &hi[c]);
    }
    expand_box(d, lo, hi, tol, mid, hw);
    for (int c = 0; c < d; ++c) {
      aabb[e * 2 * d + c] = mid[c] - hw[c];
      aabb[e * 2 * d + d + c] = mid[c] + hw[c];
    }
    /* OBB */
    double r0[3] = {0.0, 0.0, 0.0}, xc[3], Jc[9], T[9], Ti[9];
    eval_map(coords, d, dr, N, NE, e, z, r0, xc, Jc, NULL);
    if (dr == d) {
      double det = inv_small(d, Jc, T);
      if (!(det != 0.0)) {
#pragma omp atomic write
        err = 1;
      }
    } else if (dr == 2) {
      surface_frame(Jc, NULL, T);
    } else {
      line_frame(d, Jc, T); /* Jc is the d x 1 tangent */
    }
    inv_small(d, T, Ti);
    double* ut = (double*)malloc(sizeof(double) * ne * d);
    for (int n = 0; n < ne; ++n)
      for (int c = 0; c < d; ++c) {
        double s = 0.0;
        for (int q = 0; q < d; ++q) s += T[c * d + q] * (u[q * ne + n] - xc[q]);
        ut[c * ne + n] = s;
      }
    for (int c = 0; c < d; ++c) element_bounds(ut + c * ne, d, dr, N, M, &lo[c], &hi[c]);
    expand_box(d, lo, hi, tol, mid, hw);
    for (int c = 0; c < d; ++c) {
      double s = xc[c];
      for (int q = 0; q < d; ++q) s += Ti[c * d + q] * mid[q];
      obb_c[e * d + c] = s;
      for (int q = 0; q < d; ++q) obb_A[(e * d + c) * d + q] = T[c * d + q] / hw[c];
    }
    free(ut);
    free(u);
  }
  return err ? -2 : 0;
}

/* Solves H_FF s_F = -g_F on the free coordinates fr[0..nf-1] by Cholesky;
 * s is zero elsewhere.  Returns 0 (s untouched) when a pivot is not > 0.   */
static int chol_solve_free(int dr, int nf, const int* fr, const double* H, const double* g,
                           double* s) {
  double L[9] = {0}, y[3];
  for (int a = 0; a < nf; ++a)
    for (int b = 0; b <= a; ++b) {
      double t = H[fr[a] * dr + fr[b]];
      for (int q = 0; q < b; ++q) t -= L[a * 3 + q] * L[b * 3 + q];
      if (a == b) {
        if (!(t > 0.0)) return 0;
        L[a * 3 + a] = sqrt(t);
      } else {
        L[a * 3 + b] = t / L[b * 3 + b];
      }
    }
  for (int a = 0; a < nf; ++a) {
    double t = -g[fr[a]];
    for (int q = 0; q < a; ++q) t -= L[a * 3 + q] * y[q];
    y[a] = t / L[a * 3 + a];
  }
  double x[3];
  for (int a = nf - 1; a >= 0; --a) {
    double t = y[a];
    for (int q = a + 1; q < nf; ++q) t -= L[q * 3 + a] * x[q];
    x[a] = t / L[a * 3 + a];
  }
  for (int j = 0; j < dr; ++j) s[j] = 0.0;
  for (int a = 0; a < nf; ++a) s[fr[a]] = x[a];
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2.1: trust-region Newton for x* in element e, minimising
 * f(r) = 0.5 |x* - x(r)|^2 over r in [-1,1]^dr.
 *   r_0: the GLL node of e closest to x* (ties: lowest node index n).
 *   Each iteration l:  dx = x* - x(r_l);  gradient J_j = -sum_c G_cj dx_c
 *     (Eq. newton_jacobian); Hessian H_jk = (G^T G)_jk
 *     - beta sum_c dx_c d2x_c/dr_j dr_k (Eq. newton_hessian, the garbled
 *     "G_ji G_ik" read as (G^T G)_jk), beta = 1 iff l > 0 and some r_j = +-1.
 *   Constrained step (the paper states only dr in alpha[-1,1]^dr and
 *     r + dr in [-1,1]^dr): coordinates at a bound whose gradient points out
 *     of the box are held (dr_j = 0); the free block solves H_FF dr_F = -J_F
 *     by Cholesky; if that block is not positive definite and beta = 1, the
 *     beta = 0 block is used instead; if that also fails, dr = 0.  Each
 *     component is clipped to [-alpha, alpha], then r + dr is projected on
 *     [-1,1]^dr and dr recomputed as the projected difference.
 *   Stop when the step dr_l (after clipping and projection) has
 *     |dr_l|_inf < tol ("until |dr_l|_inf < eps" read as a test on the step
 *     itself): that step is applied without the trust-region test — its
 *     predicted decrease is at the rounding level of |dx|^2, where the
 *     decrease test would reject it at random — and x(r*) is evaluated for
 *     dist2.  Also stop after max_iter evaluated iterations (rejected ones
 *     count) or when the predicted decrease is not positive.
 *   Predicted decrease of |dx|^2: beta = 0, |dx|^2 - |dx - G dr|^2; beta = 1,
 *     the quadratic model -2 J.dr - dr^T H dr (the garbled "J^T dx" term read
 *     as the gradient term of that model).  If it is not positive the step
 *     cannot decrease f and the iteration stops.
 *   Actual decrease: |dx_l|^2 - |dx_{l+1}|^2.  alpha: x2 if decr >= 0.9 pred,
 *     kept if decr >= 0.01 pred, else /4 and the step is rejected — except
 *     that a step not shortened by alpha whose pred is below
 *     tau = 1e-12 X sqrt(|dx|^2) (X = largest |coordinate| of the element's
 *     AABB) is accepted with alpha kept: such a decrease is below the
 *     rounding error of the measured one.
 * Returns the number of evaluated iterations; r (dr values) and
 * dist2 = |dx|^2 at the final point.  stats (may be NULL): [1] += iterations,
 * [2] += rejected steps, [3] += iterations with beta = 1.                   */
static int newton_elem(const double* coords, int d, int dr, int N, int64_t NE, int64_t e,
                       const double* z, const double* xs, double xscale, double tol, int max_iter,
                       double* r, double* dist2, int64_t* st) {
  const int ne = nodes_per_elem(N, dr);
  /* initial guess: closest node */
  double best = INFINITY;
  int nbest = 0;
  for (int n = 0; n < ne; ++n) {
    double dd = 0.0;
    for (int c = 0; c < d; ++c) {
      double t = xs[c] - coords[((int64_t)c * NE + e) * ne + n];
      dd += t * t;
    }
    if (dd < best) {
      best = dd;
      nbest = n;
    }
  }
  int idx[3] = {nbest % N, (nbest / N) % N, nbest / (N * N)};
  for (int j = 0; j < dr; ++j) r[j] = z[idx[j]];
  double alpha = 1.0;
  double x[3], G[9], S[27], dx[3], F = 0.0;
  eval_map(coords, d, dr, N, NE, e, z, r, x, G, NULL);
  for (int c = 0; c < d; ++c) {
    dx[c] = xs[c] - x[c];
    F += dx[c] * dx[c];
  }
  int it = 0;
  for (int l = 0; l < max_iter; ++l) {
    int at_bound = 0;
    for (int j = 0; j < dr; ++j)
      if (r[j] == -1.0 || r[j] == 1.0) at_bound = 1;
    int beta = (l > 0 && at_bound) ? 1 : 0;
    double g[3];
    for (int j = 0; j < dr; ++j) {
      double s = 0.0;
      for (int c = 0; c < d; ++c) s -= G[c * dr + j] * dx[c];
      g[j] = s;
    }
    int fr[3], nf = 0;
    for (int j = 0; j < dr; ++j) {
      int held = (r[j] == -1.0 && g[j] > 0.0) || (r[j] == 1.0 && g[j] < 0.0);
      if (!held) fr[nf++] = j;
    }
    double H[9], HGN[9];
    for (int j = 0; j < dr; ++j)
      for (int k = 0; k < dr; ++k) {
        double s = 0.0;
        for (int c = 0; c < d; ++c) s += G[c * dr + j] * G[c * dr + k];
        HGN[j * dr + k] = s;
        H[j * dr + k] = s;
      }
    if (beta) {
      eval_map(coords, d, dr, N, NE, e, z, r, x, NULL, S);
      for (int j = 0; j < dr; ++j)
        for (int k = 0; k < dr; ++k) {
          double s = 0.0;
          for (int c = 0; c < d; ++c) s += dx[c] * S[(c * dr + j) * dr + k];
          H[j * dr + k] -= s;
        }
    }
    /* Cholesky solve on the free block, with the fallbacks described above */
    double step[3] = {0.0, 0.0, 0.0};
    int used_beta = beta;
    int solved = chol_solve_free(dr, nf, fr, H, g, step);
    if (!solved && beta) {
      used_beta = 0;
      solved = chol_solve_free(dr, nf, fr, HGN, g, step);
    }
    if (!solved) {
      used_beta = 0;
      for (int j = 0; j < dr; ++j) step[j] = 0.0;
    }
    /* trust region and box */
    double rn[3], dstep[3];
    int clipped = 0;
    for (int j = 0; j < dr; ++j) {
      double s = step[j];
      if (s > alpha) { s = alpha; clipped = 1; }
      if (s < -alpha) { s = -alpha; clipped = 1; }
      double v = r[j] + s;
      if (v > 1.0) v = 1.0;
      if (v < -1.0) v = -1.0;
      rn[j] = v;
      dstep[j] = v - r[j];
    }
    /* Sec. 3.2.1: iterate until |dr_l|_inf < tol, dr_l the (clipped,
     * projected) step of Eq. newton.  That last step is taken without the
     * trust-region test and x(r*) is evaluated for the distance. */
    double mx = 0.0;
    for (int j = 0; j < dr; ++j)
      if (fabs(dstep[j]) > mx) mx = fabs(dstep[j]);
    if (mx < tol) {
      ++it;
      if (st) st[1] += 1;
      for (int j = 0; j < dr; ++j) r[j] = rn[j];
      eval_map(coords, d, dr, N, NE, e, z, r, x, NULL, NULL);
      F = 0.0;
      for (int c = 0; c < d; ++c) {
        dx[c] = xs[c] - x[c];
        F += dx[c] * dx[c];
      }
      break;
    }
    /* predicted decrease of |dx|^2: beta = 0, |dx|^2 - |dx - G dr|^2, which
     * equals -2 J.dr - |G dr|^2 and is computed in that form (no cancellation
     * against |dx|^2); beta = 1, the quadratic model -2 J.dr - dr^T H dr. */
    double lin = 0.0, quad = 0.0;
    for (int j = 0; j < dr; ++j) lin += g[j] * dstep[j];
    if (!used_beta) {
      for (int c = 0; c < d; ++c) {
        double t = 0.0;
        for (int j = 0; j < dr; ++j) t += G[c * dr + j] * dstep[j];
        quad += t * t;
      }
    } else {
      for (int j = 0; j < dr; ++j)
        for (int k = 0; k < dr; ++k) quad += dstep[j] * H[j * dr + k] * dstep[k];
    }
    double pred = -2.0 * lin - quad;
    if (!(pred > 0.0)) break;
    ++it;
    if (st) {
      st[1] += 1;
      if (beta) st[3] += 1;
    }
    double xn[3], Gn[9], dxn[3], Fn = 0.0;
    eval_map(coords, d, dr, N, NE, e, z, rn, xn, Gn, NULL);
    for (int c = 0; c < d; ++c) {
      dxn[c] = xs[c] - xn[c];
      Fn += dxn[c] * dxn[c];
    }
    double decr = F - Fn;
    /* decr carries a rounding error of about 1e-14 X sqrt(F) (X the size of
     * the coordinates); a full-length step whose predicted decrease is below
     * 100 times that cannot be judged by the ratio test and is accepted
     * (alpha unchanged) — the paper is silent on rounding. */
    double tau = 1e-12 * xscale * sqrt(F);
    int accept;
    if (!clipped && pred < tau) {
      accept = 1;
    } else if (decr >= 0.9 * pred) {
      alpha *= 2.0;
      accept = 1;
    } else if (decr >= 0.01 * pred) {
      accept = 1;
    } else {
      alpha *= 0.25;
      accept = 0;
      if (st) st[2] += 1;
    }
    if (accept) {
      for (int j = 0; j < dr; ++j) r[j] = rn[j];
      for (int c = 0; c < d; ++c) dx[c] = dxn[c];
      for (int c = 0; c < d * dr; ++c) G[c] = Gn[c];
      F = Fn;
    }
  }
  *dist2 = F;
  return it;
}

/* X of the rounding threshold: the largest |coordinate| of the AABB. */
static double aabb_scale(int d, const double* box) {
  double X = 0.0;
  for (int c = 0; c < 2 * d; ++c)
    if (fabs(box[c]) > X) X = fabs(box[c]);
  return X;
}

/* the expanded AABB of one element (as in or_element_boxes) */
static void one_aabb(const double* coords, int d, int dr, int N, int64_t NE, int64_t e,
                     double tol, int M, double* box) {
  const int ne = nodes_per_elem(N, dr);
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, mid[3], hw[3];
  double* u = (double*)malloc(sizeof(double) * ne);
  for (int c = 0; c < d; ++c) {
    for (int n = 0; n < ne; ++n) u[n] = coords[((int64_t)c * NE + e) * ne + n];
    element_bounds(u, d, dr, N, M, &lo[c], &hi[c]);
  }
  free(u);
  expand_box(d, lo, hi, tol, mid, hw);
  for (int c = 0; c < d; ++c) {
    box[c] = mid[c] - hw[c];
    box[d + c] = mid[c] + hw[c];
  }
}

int or_newton(const double* coords, int d, int dr, int N, int64_t NE, int64_t e,
              const double* xs, double tol, int max_iter, double* r, double* dist2,
              int64_t* stats) {
  double z[OR_MAXN], box[6];
  if (or_gll_nodes(N, z)) return -1;
  one_aabb(coords, d, dr, N, NE, e, 0.1, 2 * N, box);
  return newton_elem(coords, d, dr, N, NE, e, z, xs, aabb_scale(d, box), tol, max_iter, r,
                     dist2, stats);
}

/* Box tests of Sec. 3.1.1 (Eq. AABB_test, written as lo <= x <= hi, the same
 * set as the product form) and Sec. 3.1.2 (Eq. OBB_test on the expanded OBB). */
static int in_boxes(int d, int64_t e, const double* aabb, const double* obb_c,
                    const double* obb_A, const double* xs) {
  for (int c = 0; c < d; ++c)
    if (!(xs[c] >= aabb[e * 2 * d + c] && xs[c] <= aabb[e * 2 * d + d + c])) return 0;
  for (int c = 0; c < d; ++c) {
    double s = 0.0;
    for (int q = 0; q < d; ++q) s += obb_A[(e * d + c) * d + q] * (xs[q] - obb_c[e * d + q]);
    if (!(fabs(s) <= 1.0)) return 0;
  }
  return 1;
}

static int all_finite(int d, const double* x) {
  for (int c = 0; c < d; ++c)
    if (!isfinite(x[c])) return 0;
  return 1;
}

/* Sec. 3.2 (local search): candidates are the elements whose expanded AABB
 * and OBB contain x* — here found by testing every element, in ascending
 * id (the hash grid of Sec. 3.1.3 only narrows this set).  Newton runs in
 * each candidate in turn; the first with r* in (-1,1)^dr (and, for surfaces,
 * dist2 < dist_tol, Sec. 4.4) is INTERIOR and ends the search; otherwise the
 * candidate with the smallest dist2 (ties: the lower id) is BORDER; no
 * candidate: NOT_FOUND (elem -1, r 0, dist2 +inf).
 * stats (may be NULL, 8 values): [0] candidates, [1] iterations, [2] rejected
 * steps, [3] beta = 1 iterations.                                           */
int or_findpts(const double* coords, int d, int dr, int N, int64_t NE, const double* aabb,
               const double* obb_c, const double* obb_A, const double* pts, int64_t n,
               double tol, int max_iter, double dist_tol, int32_t* code, int32_t* elem,
               double* r, double* dist2, int64_t* stats) {
  double z[OR_MAXN];
  if (or_gll_nodes(N, z)) return -1;
  int64_t s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : s0, s1, s2, s3)
  for (int64_t p = 0; p < n; ++p) {
    const double* xs = pts + p * d;
    int64_t st[8] = {0};
    int bcode = 2, be = -1;
    double br[3] = {0, 0, 0}, bd = INFINITY;
    if (all_finite(d, xs)) {
      for (int64_t e = 0; e < NE; ++e) {
        if (!in_boxes(d, e, aabb, obb_c, obb_A, xs)) continue;
        st[0] += 1;
        double rr[3], dd;
        newton_elem(coords, d, dr, N, NE, e, z, xs, aabb_scale(d, aabb + e * 2 * d), tol,
                    max_iter, rr, &dd, st);
        int inside = 1;
        for (int j = 0; j < dr; ++j)
          if (!(fabs(rr[j]) < 1.0)) inside = 0;
        if (dr < d && !(dd < dist_tol)) inside = 0;
        if (inside) {
          bcode = 0;
          be = (int)e;
          bd = dd;
          for (int j = 0; j < dr; ++j) br[j] = rr[j];
          break;
        }
        if (dd < bd) {
          bcode = 1;
          be = (int)e;
          bd = dd;
          for (int j = 0; j < dr; ++j) br[j] = rr[j];
        }
      }
    }
    code[p] = bcode;
    elem[p] = be;
    for (int j = 0; j < dr; ++j) r[p * dr + j] = br[j];
    dist2[p] = bd;
    s0 += st[0];
    s1 += st[1];
    s2 += st[2];
    s3 += st[3];
  }
  if (stats) {
    stats[0] += s0;
    stats[1] += s1;
    stats[2] += s2;
    stats[3] += s3;
  }
  return 0;
}

/* Newton of Sec. 3.2.1 for every point in one given element (no box test):
 * used to show that the boxes have no false negatives.  code: 0 when r* is
 * in (-1,1)^dr (and dist2 < dist_tol for surfaces), else 1.                  */
int or_locate_in_element(const double* coords, int d, int dr, int N, int64_t NE, int64_t e,
                         const double* pts, int64_t n, double tol, int max_iter,
                         double dist_tol, int32_t* code, double* r, double* dist2) {
  double z[OR_MAXN], box[6];
  if (or_gll_nodes(N, z)) return -1;
  one_aabb(coords, d, dr, N, NE, e, 0.1, 2 * N, box);
  const double X = aabb_scale(d, box);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t p = 0; p < n; ++p) {
    double rr[3], dd;
    newton_elem(coords, d, dr, N, NE, e, z, pts + p * d, X, tol, max_iter, rr, &dd, NULL);
    int inside = 1;
    for (int j = 0; j < dr; ++j)
      if (!(fabs(rr[j]) < 1.0)) inside = 0;
    if (dr < d && !(dd < dist_tol)) inside = 0;
    code[p] = inside ? 0 : 1;
    for (int j = 0; j < dr; ++j) r[p * dr + j] = rr[j];
    dist2[p] = dd;
  }
  return 0;
}

/* Brute-force candidate count and first candidate of each point. */
int or_box_candidates(int d, int64_t NE, const double* aabb, const double* obb_c,
                      const double* obb_A, const double* pts, int64_t n, int32_t* count,
                      int32_t* first) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t p = 0; p < n; ++p) {
    int cnt = 0, f = -1;
    if (all_finite(d, pts + p * d))
      for (int64_t e = 0; e < NE; ++e)
        if (in_boxes(d, e, aabb, obb_c, obb_A, pts + p * d)) {
          if (f < 0) f = (int)e;
          ++cnt;
        }
    count[p] = cnt;
    first[p] = f;
  }
  return 0;
}

/* Sec. 3.3, Eq. u_tensor: out[c][p] = sum_n u_c[elem_p][n] Phi_n(r_p) (direct
 * sum over nodes); 0 for NOT_FOUND points.                                   */
int or_eval(const double* field, int nc, int dr, int N, int64_t NE, const int32_t* code,
            const int32_t* elem, const double* r, int64_t n, double* out) {
  double z[OR_MAXN];
  if (or_gll_nodes(N, z)) return -1;
  const int ne = nodes_per_elem(N, dr);
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p) {
    if (code[p] == 2 || elem[p] < 0 || elem[p] >= NE) {
      for (int c = 0; c < nc; ++c) out[(int64_t)c * n + p] = 0.0;
      continue;
    }
    double phi[3][OR_MAXN];
    for (int j = 0; j < dr; ++j) or_lagrange(N, z, r[p * dr + j], phi[j], NULL, NULL);
    for (int c = 0; c < nc; ++c) {
      double s = 0.0;
      for (int q = 0; q < ne; ++q) {
        double B = 1.0;
        int idx[3] = {q % N, (q / N) % N, q / (N * N)};
        for (int j = 0; j < dr; ++j) B *= phi[j][idx[j]];
        s += field[((int64_t)c * NE + elem[p]) * ne + q] * B;
      }
      out[(int64_t)c * n + p] = s;
    }
  }
  return 0;
}

/* Eq. x: x = x_e(r) for given (elem, r) pairs, and optionally the Jacobian
 * jac[p][c][j] = dx_c/dr_j (used by tests to build off-surface points). */
int or_forward_map(const double* coords, int d, int dr, int N, int64_t NE,
                   const int32_t* elem, const double* r, int64_t n, double* x, double* jac) {
  double z[OR_MAXN];
  if (or_gll_nodes(N, z)) return -1;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p) {
    double G[9];
    eval_map(coords, d, dr, N, NE, elem[p], z, r + p * dr, x + p * d, jac ? G : NULL, NULL);
    if (jac)
      for (int q = 0; q < d * dr; ++q) jac[p * d * dr + q] = G[q];
  }
  return 0;
}

int or_num_threads(void) { return omp_get_max_threads(); }

/* Sets the OpenMP thread count of later calls (n >= 1). */
void or_set_num_threads(int n) {
  if (n >= 1) omp_set_num_threads(n);
}
