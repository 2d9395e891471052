// Setup (Sec. 3.1): element boxes and the process-local map Psi_L, on the GPU.
//
// Host side: the per-order constant tables (GLL nodes, barycentric and
// quadrature weights, Chebyshev points, piecewise-linear basis bounds and
// their pairwise products).  Device side: one CTA per element computes its
// AABB and OBB (k_boxes); four small kernels build Psi_L in CSR form.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "fp_basis.cuh"
#include "fp_common.cuh"

namespace fp {

namespace {

constexpr int kMaxM = 32;

// ---- host tables ----------------------------------------------------------

// P_n(x) and P'_n(x) by the three-term recurrence.
void legendre_host(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    *P = 1.0;
    *dP = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  // (1 - x^2) P'_n = n (P_{n-1} - x P_n), valid away from +-1
  *dP = (fabs(x) < 1.0) ? n * (p0 - x * p1) / (1.0 - x * x) : 0.5 * n * (n + 1) * pow(x, n + 1);
}

// GLL nodes: +-1 and the extrema of P_{N-1}, by Newton on P'_{N-1} with
// P'' taken from Legendre's equation (1-x^2) P'' = 2x P' - n(n+1) P.
// Also the GLL quadrature weights 2 / (n (n+1) P_n(z)^2).
void gll_host(int N, double* z, double* wq) {
  const int n = N - 1;
  z[0] = -1.0;
  z[N - 1] = 1.0;
  for (int j = 1; j < N - 1; ++j) {
    double x = -cos(M_PI * j / n);
    for (int it = 0; it < 60; ++it) {
      double P, dP;
      legendre_host(n, x, &P, &dP);
      const double d2P = (2.0 * x * dP - n * (n + 1.0) * P) / (1.0 - x * x);
      const double step = dP / d2P;
      x -= step;
      if (fabs(step) < 1e-17) break;
    }
    z[j] = x;
  }
  for (int j = 0; j < N; ++j) {
    double P, dP;
    legendre_host(n, z[j], &P, &dP);
    wq[j] = 2.0 / (n * (n + 1.0) * P * P);
  }
}

// phi_i(x) and phi'_i(x) with barycentric weights wb (product form).
void lagrange_host(int N, const double* z, const double* wb, double x, double* phi, double* dphi) {
  for (int i = 0; i < N; ++i) {
    double p = 1.0, dp = 0.0;
    for (int m = 0; m < N; ++m) {
      if (m == i) continue;
      dp = dp * (x - z[m]) + p;
      p = p * (x - z[m]);
    }
    phi[i] = wb[i] * p;
    dphi[i] = wb[i] * dp;
  }
}

}  // namespace

int host_basis_tab(int N, BasisTab* tab) {
  if (N < 2 || N > FP_MAX_N) return FP_EUNSUPPORTED;
  double z[FP_MAX_N], wq[FP_MAX_N];
  gll_host(N, z, wq);
  // exact symmetry about 0, which the symmetric form of the basis relies on
  for (int i = 0; i < N / 2; ++i) {
    const double a = 0.5 * (z[N - 1 - i] - z[i]);
    z[i] = -a;
    z[N - 1 - i] = a;
  }
  if (N % 2) z[N / 2] = 0.0;
  memset(tab, 0, sizeof(*tab));
  const double sigma = (N % 2) ? 1.0 : -1.0;  // (-1)^(N-1)
  for (int i = 0; i < N; ++i) {
    double p = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != i) p *= (z[i] - z[m]);
    tab->z[i] = z[i];
    tab->w[i] = (i >= (N + 1) / 2) ? sigma * tab->w[N - 1 - i] : 1.0 / p;
  }
  for (int i = 0; i < N; ++i) {
    tab->w2[i] = 2.0 * tab->w[i];
    tab->zf[i] = (float)tab->z[i];
    tab->wf[i] = (float)tab->w[i];
    tab->w2f[i] = 2.0f * tab->wf[i];
  }
  for (int m = 0; m < N / 2; ++m) {
    tab->z2[m] = tab->z[m] * tab->z[m];
    tab->z2f[m] = tab->zf[m] * tab->zf[m];
    tab->z2h[m] = (float)tab->z2[m];
    tab->z2l[m] = (float)(tab->z2[m] - (double)tab->z2h[m]);
  }
  for (int i = 0; i < N; ++i) {
    tab->zl[i] = (float)(tab->z[i] - (double)tab->zf[i]);
    tab->wl[i] = (float)(tab->w[i] - (double)tab->wf[i]);
  }
  // phi_m'(z_i) = (w_m / w_i) / (z_i - z_m) for m != i (differentiate the
  // product form of phi_m at a root of its other factors); the diagonal is
  // minus the row's other entries, since the derivative of sum_m phi_m = 1
  // vanishes.
  for (int i = 0; i < N; ++i) {
    double diag = 0.0;
    for (int m = 0; m < N; ++m) {
      if (m == i) continue;
      const double v = (tab->w[m] / tab->w[i]) / (z[i] - z[m]);
      tab->dn[i * N + m] = v;
      diag -= v;
    }
    tab->dn[i * N + i] = diag;
  }
  return FP_OK;
}

namespace {

// Sums of |phi_i^(k)(r)| over the N Lagrange bases, maximised over r in
// [-1, 1] by dense sampling (20001 points, 2% added for the sampling), for
// k = 0, 1, 2 (Ls[0] is the Lebesgue constant of the nodes).
void basis_sums(int N, double Ls[3]) {
  double z[FP_MAX_N], wq[FP_MAX_N], w[FP_MAX_N];
  gll_host(N, z, wq);
  for (int i = 0; i < N; ++i) {
    double p = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != i) p *= (z[i] - z[m]);
    w[i] = 1.0 / p;
  }
  for (int q = 0; q < 3; ++q) Ls[q] = 0.0;
  const int S = 20001;
  for (int k = 0; k < S; ++k) {
    const double x = -1.0 + 2.0 * k / (S - 1);
    double a[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < N; ++i) {
      // value, first and second derivative of prod_{m != i} (x - z_m)
      double p = 1.0, dp = 0.0, d2p = 0.0;
      for (int m = 0; m < N; ++m) {
        if (m == i) continue;
        const double t = x - z[m];
        d2p = d2p * t + 2.0 * dp;
        dp = dp * t + p;
        p = p * t;
      }
      a[0] += fabs(w[i] * p);
      a[1] += fabs(w[i] * dp);
      a[2] += fabs(w[i] * d2p);
    }
    for (int q = 0; q < 3; ++q) Ls[q] = std::max(Ls[q], a[q]);
  }
  for (int q = 0; q < 3; ++q) Ls[q] *= 1.02;
}

// The factor K such that, for an element whose nodal values deviate by at
// most dev from an affine function of r, every second-derivative sum over
// (j, k) of |d^2 x_c / dr_j dr_k| is at most dev * K:
// dr * L2 L0^(dr-1) (j = k) + dr (dr - 1) * L1^2 L0^(dr-2) (j != k).  This
// cruder bound serves the mixed path's certified refinement, whose
// acceptance threshold was chosen with it.
double curvature_factor(int N, int dr) {
  double L[3];
  basis_sums(N, L);
  const double pure = L[2] * pow(L[0], dr - 1), mixed = dr > 1 ? L[1] * L[1] * pow(L[0], dr - 2) : 0.0;
  return dr * pure + dr * (dr - 1) * mixed;
}

// Per-element doubles that k_boxes hands to k_box32: x(0) (3), the OBB frame
// T (9), the curvature bound (1).
constexpr int kLin = 16;

// Device table layout (doubles) for the box kernel.
struct TabLayout {
  int N, M;
  int c0, c1, eta, vlo, vhi, pmin, pmax, total;
  __host__ __device__ TabLayout(int N_, int M_) : N(N_), M(M_) {
    c0 = 0;
    c1 = c0 + N;
    eta = c1 + N;
    vlo = eta + M;
    vhi = vlo + N * M;
    pmin = vhi + N * M;
    pmax = pmin + M * M * N * N;
    total = pmax + M * M * N * N;
  }
};

// Sec. 3.1.1 tables for (N, M):
//  c0, c1: a_l = sum_i c_l[i] u_i, the (2l+1)/2-scaled Legendre projections,
//    from GLL quadrature (exact: phi_i P_l has degree <= N <= 2N-3 for N >= 3;
//    closed form for N = 2);
//  eta: Chebyshev points (Eq. chebyshev);
//  vlo, vhi [i][j]: basis bounds of Eq. 1D_bases_bounds, tangents at the
//    interval midpoints evaluated at their distance from eta_j;
//  pmin, pmax [k][l][b][a]: min / max of the four products of the bound
//    values of basis a at eta_k and basis b at eta_l, so that the four-term
//    min of Eq. 2D_function_bound_1 is w * pmin when w >= 0, w * pmax else.
std::vector<double> bound_tables(int N, int M) {
  TabLayout L(N, M);
  std::vector<double> t(L.total, 0.0);
  double z[FP_MAX_N], wq[FP_MAX_N], wb[FP_MAX_N];
  gll_host(N, z, wq);
  for (int i = 0; i < N; ++i) {
    double p = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != i) p *= (z[i] - z[m]);
    wb[i] = 1.0 / p;
  }
  for (int i = 0; i < N; ++i) {
    t[L.c0 + i] = 0.5 * wq[i];
    t[L.c1 + i] = (N == 2) ? (i == 0 ? -0.5 : 0.5) : 1.5 * wq[i] * z[i];
  }
  double eta[kMaxM];
  for (int j = 0; j < M; ++j) eta[j] = -cos(M_PI * (double)j / (double)(M - 1));
  for (int j = 0; j < M; ++j) t[L.eta + j] = eta[j];
  for (int j = 0; j < M; ++j) {
    double phi[FP_MAX_N], dphi[FP_MAX_N], pm[FP_MAX_N], dpm[FP_MAX_N], pp[FP_MAX_N], dpp[FP_MAX_N];
    if (j == 0 || j == M - 1) {
      for (int i = 0; i < N; ++i) {
        const double v = (j == 0) ? (i == 0) : (i == N - 1);
        t[L.vlo + i * M + j] = v;
        t[L.vhi + i * M + j] = v;
      }
      continue;
    }
    const double xm = 0.5 * (eta[j - 1] + eta[j]), xp = 0.5 * (eta[j] + eta[j + 1]);
    lagrange_host(N, z, wb, eta[j], phi, dphi);
    lagrange_host(N, z, wb, xm, pm, dpm);
    lagrange_host(N, z, wb, xp, pp, dpp);
    for (int i = 0; i < N; ++i) {
      const double cand[3] = {phi[i], pm[i] + (eta[j] - xm) * dpm[i], pp[i] - (xp - eta[j]) * dpp[i]};
      t[L.vlo + i * M + j] = std::min(cand[0], std::min(cand[1], cand[2]));
      t[L.vhi + i * M + j] = std::max(cand[0], std::max(cand[1], cand[2]));
    }
  }
  for (int k = 0; k < M; ++k)
    for (int l = 0; l < M; ++l)
      for (int b = 0; b < N; ++b)
        for (int a = 0; a < N; ++a) {
          const double A[2] = {t[L.vlo + a * M + k], t[L.vhi + a * M + k]};
          const double B[2] = {t[L.vlo + b * M + l], t[L.vhi + b * M + l]};
          double mn = A[0] * B[0], mx = mn;
          for (int x = 0; x < 2; ++x)
            for (int y = 0; y < 2; ++y) {
              mn = std::min(mn, A[x] * B[y]);
              mx = std::max(mx, A[x] * B[y]);
            }
          const int idx = ((k * M + l) * N + b) * N + a;
          t[L.pmin + idx] = mn;
          t[L.pmax + idx] = mx;
        }
  return t;
}

// ---- device: boxes ----------------------------------------------------------

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

constexpr int kBoxThreads = 128;

// Box expansion (Sec. 3.1.1, 10% by default; Sec. 4.1 for zero extents):
// extent L grows to (1+tol) L about the centre; an extent <= 1e-12 of the
// largest one is padded by tol * (smallest other extent) instead.
__device__ void expand(int d, const double* lo, const double* hi, double tol, double* mid, double* hw) {
  double Lmax = 0.0;
  for (int c = 0; c < d; ++c) Lmax = fmax(Lmax, hi[c] - lo[c]);
  double Lmin = INFINITY;
  for (int c = 0; c < d; ++c) {
    const double L = hi[c] - lo[c];
    if (L > 1e-12 * Lmax && L < Lmin) Lmin = L;
  }
  for (int c = 0; c < d; ++c) {
    const double L = hi[c] - lo[c];
    double pad = (L > 1e-12 * Lmax) ? 0.5 * tol * L : 0.5 * tol * Lmin;
    if (!isfinite(pad)) pad = 0.0;
    mid[c] = 0.5 * (lo[c] + hi[c]);
    hw[c] = 0.5 * L + pad;
  }
}

// The rotation R taking the unit tangent u = t/|t| of a line element to the
// x axis (Sec. 4.2, Rodrigues' formula): in 2D the plane rotation with rows
// (u0, u1), (-u1, u0); in 3D R = I + sin K + (1 - cos) K^2 with K the
// cross-product matrix of the unit axis u x e1 and cos = u0 (a tangent
// along -e1 turns by pi about e3).  Row-major, D x D.
template <int D>
__device__ void line_rotation(const double* t, double* R) {
  double nt = 0.0;
  for (int c = 0; c < D; ++c) nt += t[c] * t[c];
  nt = sqrt(nt);
  double u[3] = {0.0, 0.0, 0.0};
  for (int c = 0; c < D; ++c) u[c] = t[c] / nt;
  if (D == 2) {
    R[0] = u[0];
    R[1] = u[1];
    R[2] = -u[1];
    R[3] = u[0];
    return;
  }
  const double ax1 = u[2], ax2 = -u[1];  // u x e1 = (0, u2, -u1)
  const double sn = sqrt(ax1 * ax1 + ax2 * ax2), cs = u[0];
  for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
  if (sn == 0.0) {
    R[0] = cs > 0.0 ? 1.0 : -1.0;
    R[4] = cs > 0.0 ? 1.0 : -1.0;
    return;
  }
  const double k[3] = {0.0, ax1 / sn, ax2 / sn};
  const double K[9] = {0.0, -k[2], k[1], k[2], 0.0, -k[0], -k[1], k[0], 0.0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double k2 = 0.0;
      for (int m = 0; m < 3; ++m) k2 += K[i * 3 + m] * K[m * 3 + j];
      R[i * 3 + j] += sn * K[i * 3 + j] + (1.0 - cs) * k2;
    }
}

// One CTA per element.  AABB: bounds of each coordinate over the element's
// boundary pieces (quad edges, hex faces) or over the element itself
// (surface quads, lines), Eqs. 1D_bound_final / 2D_function_bound.  OBB: the
// same bounds of the nodes mapped by T = J_c^{-1} (volumes, Eq.
// OBB_transformation), T = [t1 t2 n]^{-1} (surface quads; this is the
// paper's R2 R1 of Sec. 4.2 written as one inverse: R1 is a rotation taking
// n to e3, and R2 R1 maps t1, t2, n to e1, e2, e3) or the Rodrigues
// rotation of line_rotation (lines).
template <int N, int D, int DR>
__global__ void __launch_bounds__(kBoxThreads)
    k_boxes(const double* __restrict__ coords, int64_t NE, const double* __restrict__ tab, int M,
            BasisTab B, double tol, double curv_factor, double* __restrict__ aabb,
            double* __restrict__ obb_c, double* __restrict__ obb_A, double* __restrict__ linmap,
            int* status) {
  constexpr int NN = ipow(N, DR);
  // bounding pieces: the 6 faces of a hex, the 4 edges of a quad, the
  // element itself for a surface quad or a line
  constexpr int NPIECE = (DR == 3) ? 6 : ((D == 2 && DR == 2) ? 4 : 1);
  constexpr int PIECE = (DR == 3 || (D == 3 && DR == 2)) ? N * N : N;  // values per piece
  const TabLayout L(N, M);
  __shared__ double X[D * NN];
  __shared__ double Xt[D * NN];
  __shared__ double uu[2 * D * PIECE];
  __shared__ unsigned char upos[2 * D * PIECE];
  __shared__ double lin[2 * D][3];
  __shared__ double rows[2 * D][N][2];
  __shared__ double rlo[kBoxThreads], rhi[kBoxThreads];
  __shared__ double T[9], Ti[9], xc[3], tlin[3];
  __shared__ double red[2][kBoxThreads / 32];
  __shared__ double sums[kBoxThreads / 32][12];
  __shared__ double blo[2][3], bhi[2][3];
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  for (int idx = tid; idx < D * NN; idx += blockDim.x) {
    const int c = idx / NN, n = idx % NN;
    X[idx] = coords[((int64_t)c * NE + e) * NN + n];
  }
  __syncthreads();
  {
    // centre x(0) and Jacobian J_c = G(0): sums over all nodes, split over
    // the threads (one lane doing them alone costs a full warp instruction
    // of the FP64 pipe per product), then reduced over the warps
    double ph[N], dph[N];
    lagrange<N, double>(B.z, B.w, 0.0, ph, dph);
    double part[3 + 9];
#pragma unroll
    for (int q = 0; q < 12; ++q) part[q] = 0.0;
    for (int n = tid; n < NN; n += blockDim.x) {
      const int i = n % N, j = (n / N) % N, k = n / (N * N);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const double v = X[c * NN + n];
        if (DR == 3) {
          part[c] += v * ph[i] * ph[j] * ph[k];
          part[3 + c * 3 + 0] += v * dph[i] * ph[j] * ph[k];
          part[3 + c * 3 + 1] += v * ph[i] * dph[j] * ph[k];
          part[3 + c * 3 + 2] += v * ph[i] * ph[j] * dph[k];
        } else if (DR == 2) {
          part[c] += v * ph[i] * ph[j];
          part[3 + c * 3 + 0] += v * dph[i] * ph[j];
          part[3 + c * 3 + 1] += v * ph[i] * dph[j];
        } else {
          part[c] += v * ph[i];
          part[3 + c * 3 + 0] += v * dph[i];
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      double v = part[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((tid & 31) == 0) sums[tid >> 5][q] = v;
    }
  }
  __syncthreads();
  if (tid == 0) {
    double J[9];
    for (int c = 0; c < D; ++c) {
      double xv = 0.0, g[3] = {0.0, 0.0, 0.0};
      for (int w = 0; w < kBoxThreads / 32; ++w) {
        xv += sums[w][c];
        for (int j = 0; j < DR; ++j) g[j] += sums[w][3 + c * 3 + j];
      }
      xc[c] = xv;
      for (int j = 0; j < DR; ++j) J[c * DR + j] = g[j];
    }
    double Mx[9];
    if (DR == D) {
      for (int q = 0; q < D * D; ++q) Mx[q] = J[q];
    } else if (DR == 1) {
      // lines (Sec. 4.2): R = the Rodrigues rotation taking t/|t| to e1;
      // Mx = R^T, so that T = Mx^{-1} = R
      double R[9], tt = 0.0;
      line_rotation<D>(J, R);
      for (int q = 0; q < D; ++q) tt += J[q] * J[q];
      for (int q = 0; q < D; ++q) tlin[q] = J[q] / tt;
      for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) Mx[a * D + b] = R[b * D + a];
    } else {  // [t1 t2 n/|n|] as columns
      const double t1[3] = {J[0], J[2], J[4]}, t2[3] = {J[1], J[3], J[5]};
      double n[3] = {t1[1] * t2[2] - t1[2] * t2[1], t1[2] * t2[0] - t1[0] * t2[2],
                     t1[0] * t2[1] - t1[1] * t2[0]};
      const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      for (int c = 0; c < 3; ++c) {
        Mx[c * 3 + 0] = t1[c];
        Mx[c * 3 + 1] = t2[c];
        Mx[c * 3 + 2] = n[c] / nn;
      }
    }
    double det;
    if (D == 2) {
      det = Mx[0] * Mx[3] - Mx[1] * Mx[2];
      T[0] = Mx[3] / det; T[1] = -Mx[1] / det;
      T[2] = -Mx[2] / det; T[3] = Mx[0] / det;
    } else {
      const double c00 = Mx[4] * Mx[8] - Mx[5] * Mx[7];
      const double c01 = Mx[5] * Mx[6] - Mx[3] * Mx[8];
      const double c02 = Mx[3] * Mx[7] - Mx[4] * Mx[6];
      det = Mx[0] * c00 + Mx[1] * c01 + Mx[2] * c02;
      T[0] = c00 / det;
      T[1] = (Mx[2] * Mx[7] - Mx[1] * Mx[8]) / det;
      T[2] = (Mx[1] * Mx[5] - Mx[2] * Mx[4]) / det;
      T[3] = c01 / det;
      T[4] = (Mx[0] * Mx[8] - Mx[2] * Mx[6]) / det;
      T[5] = (Mx[2] * Mx[3] - Mx[0] * Mx[5]) / det;
      T[6] = c02 / det;
      T[7] = (Mx[1] * Mx[6] - Mx[0] * Mx[7]) / det;
      T[8] = (Mx[0] * Mx[4] - Mx[1] * Mx[3]) / det;
    }
    if (!(det != 0.0) || !isfinite(det)) record_status(status, FP_DEV_DEGENERATE);
    for (int q = 0; q < D * D; ++q) Ti[q] = Mx[q];
  }
  __syncthreads();
  for (int idx = tid; idx < D * NN; idx += blockDim.x) {
    const int c = idx / NN, n = idx % NN;
    double s = 0.0;
    for (int q = 0; q < D; ++q) s += T[c * D + q] * (X[q * NN + n] - xc[q]);
    Xt[idx] = s;
  }
  if (DR == D) {
    // volumes: the nodes' largest distance from the tangent map x(0) + J_c r
    // at their reference coordinates (Ti holds J_c), for the curvature bound
    // of the mixed path's certified refinement
    double dv = 0.0;
    for (int idx = tid; idx < D * NN; idx += blockDim.x) {
      const int c = idx / NN, n = idx % NN;
      const int id[3] = {n % N, (n / N) % N, n / (N * N)};
      double a = X[idx] - xc[c];
      for (int q = 0; q < DR; ++q) a -= Ti[c * D + q] * B.z[id[q]];
      dv = fmax(dv, fabs(a));
    }
    dv = warp_max(dv);
    if ((tid & 31) == 0) red[0][tid >> 5] = dv;
  }
  __syncthreads();
  if (DR == D && tid == 0) {
    double dv = red[0][0];
    for (int w = 1; w < kBoxThreads / 32; ++w) dv = fmax(dv, red[0][w]);
    linmap[e * kLin + 12] = dv * curv_factor * (1.0 + 1e-6);
  }
  __syncthreads();
  const double* c0 = tab + L.c0;
  const double* c1 = tab + L.c1;
  const double* eta = tab + L.eta;
  // Every (box kind, coordinate) combination of a piece at once: thread t
  // works on combination t % NC at grid points t / NC, t / NC + PER, ...,
  // so the 2 D bounds of a piece share its barriers (one piece gather,
  // the compactions side by side) and nearly every thread is busy.
  constexpr int NC = 2 * D;
  constexpr int PER = kBoxThreads / NC;
  const int kc = tid % NC, slot = tid / NC;
  double tlo = INFINITY, thi = -INFINITY;
  for (int piece = 0; piece < NPIECE; ++piece) {
    // gather the piece's nodal values of every combination
    for (int idx = tid; idx < NC * PIECE; idx += blockDim.x) {
      const int q = idx / PIECE, a0 = idx % PIECE;
      int n;
      if (DR == 3) {
        const int a = a0 % N, b = a0 / N, fixed = piece / 2;
        const int val = (piece % 2) ? N - 1 : 0;
        const int i = fixed == 0 ? val : a;
        const int j = fixed == 0 ? a : (fixed == 1 ? val : b);
        const int k = fixed == 2 ? val : b;
        n = i + N * (j + N * k);
      } else if (D == 3 || DR == 1) {
        n = a0;
      } else {
        const int a = a0;
        int i, j;
        if (piece == 0) { i = a; j = 0; }
        else if (piece == 1) { i = a; j = N - 1; }
        else if (piece == 2) { i = 0; j = a; }
        else { i = N - 1; j = a; }
        n = i + N * j;
      }
      uu[idx] = (q / D ? Xt : X)[(q % D) * NN + n];
    }
    __syncthreads();
    // the linear Legendre part of every combination
    if (PIECE == N) {
      if (tid < NC) {
        const double* u = uu + tid * PIECE;
        double a00 = 0.0, a10 = 0.0;
        for (int a = 0; a < N; ++a) {
          a00 += c0[a] * u[a];
          a10 += c1[a] * u[a];
        }
        lin[tid][0] = a00;
        lin[tid][1] = a10;
        lin[tid][2] = 0.0;
      }
    } else {
      // one thread per (combination, row b) sums over a, then one per
      // combination over b
      if (tid < NC * N) {
        const int q = tid / N, b = tid % N;
        const double* u = uu + q * PIECE + N * b;
        double s0 = 0.0, s1 = 0.0;
        for (int a = 0; a < N; ++a) {
          s0 += c0[a] * u[a];
          s1 += c1[a] * u[a];
        }
        rows[q][b][0] = s0;
        rows[q][b][1] = s1;
      }
      __syncthreads();
      if (tid < NC) {
        double a00 = 0.0, a10 = 0.0, a01 = 0.0;
        for (int b = 0; b < N; ++b) {
          a00 += c0[b] * rows[tid][b][0];
          a10 += c0[b] * rows[tid][b][1];
          a01 += c1[b] * rows[tid][b][0];
        }
        lin[tid][0] = a00;
        lin[tid][1] = a10;
        lin[tid][2] = a01;
      }
    }
    __syncthreads();
    for (int idx = tid; idx < NC * PIECE; idx += blockDim.x) {
      const int q = idx / PIECE, a0 = idx % PIECE;
      const int a = a0 % N, b = a0 / N;
      const double v = uu[idx] - (lin[q][0] + lin[q][1] * B.z[a] + (PIECE == N ? 0.0 : lin[q][2] * B.z[b]));
      uu[idx] = v;
      upos[idx] = v >= 0.0;  // the sign decides which product bound is the lower one
    }
    __syncthreads();
    if (slot < PER) {
      const double* u = uu + kc * PIECE;
      const double* ln = lin[kc];
      if (PIECE == N) {
        const double* vlo = tab + L.vlo;
        const double* vhi = tab + L.vhi;
        for (int j = slot; j < M; j += PER) {
          double l = ln[0] + ln[1] * eta[j], h = l;
          for (int a = 0; a < N; ++a) {
            const double p = u[a] * vlo[a * M + j], q = u[a] * vhi[a * M + j];
            l += fmin(p, q);
            h += fmax(p, q);
          }
          tlo = fmin(tlo, l);
          thi = fmax(thi, h);
        }
      } else {
        const double* pmin = tab + L.pmin;
        const double* pmax = tab + L.pmax;
        const unsigned char* pos = upos + kc * PIECE;
        for (int g = slot; g < M * M; g += PER) {
          const int k = g / M, l = g % M;
          double lo = ln[0] + ln[1] * eta[k] + ln[2] * eta[l], hi = lo;
          const double* pn = pmin + (size_t)g * N * N;
          const double* px = pmax + (size_t)g * N * N;
          for (int ab = 0; ab < N * N; ++ab) {
            const double w = u[ab];
            const double pl = __ldg(pn + ab), ph = __ldg(px + ab);
            const bool nonneg = pos[ab];
            lo = fma(w, nonneg ? pl : ph, lo);
            hi = fma(w, nonneg ? ph : pl, hi);
          }
          tlo = fmin(tlo, lo);
          thi = fmax(thi, hi);
        }
      }
    }
    __syncthreads();
  }
  rlo[tid] = tlo;
  rhi[tid] = thi;
  __syncthreads();
  if (tid < NC) {
    double a = INFINITY, b = -INFINITY;
    for (int s2 = 0; s2 < PER; ++s2) {
      a = fmin(a, rlo[s2 * NC + tid]);
      b = fmax(b, rhi[s2 * NC + tid]);
    }
    blo[tid / D][tid % D] = a;
    bhi[tid / D][tid % D] = b;
  }
  __syncthreads();
  if (tid == 0) {
    double mid[3], hw[3];
    expand(D, blo[0], bhi[0], tol, mid, hw);
    for (int c = 0; c < D; ++c) {
      aabb[e * 2 * D + c] = mid[c] - hw[c];
      aabb[e * 2 * D + D + c] = mid[c] + hw[c];
    }
    for (int c = 0; c < D; ++c) {
      linmap[e * kLin + c] = xc[c];
      for (int q = 0; q < D; ++q) linmap[e * kLin + 3 + c * 3 + q] = T[c * D + q];
    }
    if (DR == 1)  // the linear start of a line: r = t.(x - x_c) / |t|^2
      for (int q = 0; q < D; ++q) linmap[e * kLin + 3 + q] = tlin[q];
    if (DR != D) linmap[e * kLin + 12] = 0.0;
    expand(D, blo[1], bhi[1], tol, mid, hw);
    for (int c = 0; c < D; ++c) {
      double s = xc[c];
      for (int q = 0; q < D; ++q) s += Ti[c * D + q] * mid[q];
      obb_c[e * D + c] = s;
      for (int q = 0; q < D; ++q) obb_A[(e * D + c) * D + q] = T[c * D + q] / hw[c];
    }
  }
}

// ---- device: Psi_L ------------------------------------------------------------

__global__ void k_grid_bounds(const double* __restrict__ aabb, int64_t NE, int d, double* out) {
  __shared__ double s[2][3][32];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t e = threadIdx.x; e < NE; e += blockDim.x)
    for (int c = 0; c < d; ++c) {
      lo[c] = fmin(lo[c], aabb[e * 2 * d + c]);
      hi[c] = fmax(hi[c], aabb[e * 2 * d + d + c]);
    }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int c = 0; c < d; ++c) {
    lo[c] = warp_min(lo[c]);
    hi[c] = warp_max(hi[c]);
    if (l == 0) {
      s[0][c][w] = lo[c];
      s[1][c][w] = hi[c];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int c = 0; c < d; ++c) {
      double a = s[0][c][0], b = s[1][c][0];
      for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
        a = fmin(a, s[0][c][q]);
        b = fmax(b, s[1][c][q]);
      }
      out[c] = a;
      out[3 + c] = b;
    }
}

struct GridView {
  double lo[3], scale[3];
  int NL, d;
};

__device__ __forceinline__ void cell_range(const GridView& g, const double* box, int* c0, int* c1) {
  for (int c = 0; c < 3; ++c) {
    c0[c] = 0;
    c1[c] = 0;
  }
  for (int c = 0; c < g.d; ++c) {
    c0[c] = cell_coord(box[c], g.lo[c], g.scale[c], g.NL);
    c1[c] = cell_coord(box[g.d + c], g.lo[c], g.scale[c], g.NL);
  }
}

// MODE 0: count entries per cell; MODE 1: place element ids.
template <int MODE>
__global__ void k_grid_scatter(const double* __restrict__ aabb, int64_t NE, GridView g,
                               int* __restrict__ counter, const int* __restrict__ start,
                               int* __restrict__ elems) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < NE;
       e += (int64_t)gridDim.x * blockDim.x) {
    int c0[3], c1[3];
    cell_range(g, aabb + e * 2 * g.d, c0, c1);
    for (int k = c0[2]; k <= c1[2]; ++k)
      for (int j = c0[1]; j <= c1[1]; ++j)
        for (int i = c0[0]; i <= c1[0]; ++i) {
          const int64_t cell = i + (int64_t)g.NL * (j + (int64_t)g.NL * k);
          const int pos = atomicAdd(&counter[cell], 1);
          if (MODE == 1) elems[start[cell] + pos] = (int)e;
        }
  }
}

// Ascending element ids within each cell (insertion sort; lists are short).
__global__ void k_grid_sort(const int* __restrict__ start, int64_t ncell, int* __restrict__ elems) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int b = start[c], en = start[c + 1];
    for (int i = b + 1; i < en; ++i) {
      const int v = elems[i];
      int j = i - 1;
      while (j >= b && elems[j] > v) {
        elems[j + 1] = elems[j];
        --j;
      }
      elems[j + 1] = v;
    }
  }
}

// coords32[c][e][n] = fl32(coords[c][e][n] - x_ref(e)_c)
__global__ void k_coords32(const double* __restrict__ x, const double* __restrict__ aabb, int d,
                           int64_t NE, int ne, float* __restrict__ y) {
  const int64_t total = (int64_t)d * NE * ne;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ce = i / ne;
    const int c = (int)(ce / NE);
    const int64_t e = ce % NE;
    y[i] = (float)(x[i] - elem_ref(aabb, d, e, c));
  }
}

// coords32p[c][e][row P + i] = coords32[c][e][row N + i] for i < N, 0 in the
// pad i = N..P-1 (P = pitch32(N), rows = N^(dr-1)).
__global__ void k_coords32p(const float* __restrict__ x32, int64_t nce, int N, int rows,
                            float* __restrict__ y) {
  const int P = pitch32(N);
  const int ne = N * rows, ne32p = P * rows;
  const int64_t total = nce * ne32p;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ce = o / ne32p;
    const int q = (int)(o - ce * ne32p);
    const int row = q / P, i = q - row * P;
    y[o] = (i < N) ? x32[ce * ne + row * N + i] : 0.f;
  }
}

// FP32 record per element (layout fp::BOX32): lo[3] hi[3] c[3] A[3][3] Xrel
// pad xc[3] T[3][3], rounded to nearest (the certified FP32 tests carry
// their own margins); Xrel = largest AABB half-width, slightly enlarged,
// bounds |x - x_ref| over the element; xc = x(0) - x_ref; T the OBB frame.
// Volumes: the element's bound L >= max over the element of
// sum_jk |d^2 x_c / dr_j dr_k| for every component c (the curvature term of
// the FP64 kernel's certified stop).  Each second derivative of x_c
// is a polynomial of degree < N in every direction, so its values at the
// GLL nodes, obtained exactly (up to rounding) by applying the GLL
// differentiation matrix dn along r_j and then along r_k, bound it on the
// whole element through the Lebesgue constant: |d_jk x_c| <= Lambda^dr
// max_nodes |d_jk x_c|.  The rounding of the two N-term sums is covered by
// an absolute slack, rslack max_n |x_c| (rslack = 2N u S^2 Lambda^dr dr^2,
// S the largest absolute row sum of dn).  One CTA per element, one component
// at a time: x_c, then its first derivatives along each r_j, in shared
// memory.
template <int N, int D>
__global__ void __launch_bounds__(kBoxThreads)
    k_curvature(const double* __restrict__ coords, int64_t NE, BasisTab B, double lam_dr, double rslack,
                float* __restrict__ curv) {
  constexpr int NN = ipow(N, D);
  constexpr int NPAIR = D * (D + 1) / 2;
  __shared__ double xs[NN];
  __shared__ double g1[D][NN];
  __shared__ double red[kBoxThreads / 32][NPAIR + 1];
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  const int st[3] = {1, N, N * N};
  double Lmax = 0.0;
  for (int c = 0; c < D; ++c) {
    for (int n = tid; n < NN; n += blockDim.x) xs[n] = coords[((int64_t)c * NE + e) * NN + n];
    __syncthreads();
    for (int idx = tid; idx < D * NN; idx += blockDim.x) {
      const int j = idx / NN, n = idx % NN;
      const int ij = (n / st[j]) % N;
      const double* line = xs + (n - ij * st[j]);
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < N; ++m) s = fma(B.dn[ij * N + m], line[m * st[j]], s);
      g1[j][n] = s;
    }
    __syncthreads();
    double mxv[NPAIR + 1];
#pragma unroll
    for (int q = 0; q <= NPAIR; ++q) mxv[q] = 0.0;
    for (int n = tid; n < NN; n += blockDim.x) {
      mxv[NPAIR] = fmax(mxv[NPAIR], fabs(xs[n]));
      int q = 0;
#pragma unroll
      for (int j = 0; j < D; ++j)
#pragma unroll
        for (int k = j; k < D; ++k, ++q) {
          const int ik = (n / st[k]) % N;
          const double* line = &g1[j][n - ik * st[k]];
          double s = 0.0;
#pragma unroll
          for (int m = 0; m < N; ++m) s = fma(B.dn[ik * N + m], line[m * st[k]], s);
          mxv[q] = fmax(mxv[q], fabs(s));
        }
    }
#pragma unroll
    for (int q = 0; q <= NPAIR; ++q) {
      double v = mxv[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
      if ((tid & 31) == 0) red[tid >> 5][q] = v;
    }
    __syncthreads();
    if (tid == 0) {
      double Lc = 0.0;
      int q = 0;
      for (int j = 0; j < D; ++j)
        for (int k = j; k < D; ++k, ++q) {
          double v = red[0][q];
          for (int w = 1; w < kBoxThreads / 32; ++w) v = fmax(v, red[w][q]);
          Lc += (j == k ? 1.0 : 2.0) * v;
        }
      double xm = red[0][NPAIR];
      for (int w = 1; w < kBoxThreads / 32; ++w) xm = fmax(xm, red[w][NPAIR]);
      Lmax = fmax(Lmax, lam_dr * Lc + rslack * xm);
    }
    __syncthreads();
  }
  // rounded to FP32 upwards by the widening (FP32 rounding is below 1e-7)
  if (tid == 0) curv[e] = (float)(Lmax * (1.0 + 1e-6));
}

__global__ void k_box32(const double* __restrict__ aabb, const double* __restrict__ obb_c,
                        const double* __restrict__ obb_A, const double* __restrict__ lin, int64_t NE,
                        int d, float* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < NE;
       e += (int64_t)gridDim.x * blockDim.x) {
    float* o = out + e * BOX32;
    for (int i = 0; i < BOX32; ++i) o[i] = 0.f;
    double X = 0.0;
    for (int c = 0; c < d; ++c) {
      o[c] = (float)aabb[e * 2 * d + c];
      o[3 + c] = (float)aabb[e * 2 * d + d + c];
      o[6 + c] = (float)obb_c[e * d + c];
      X = fmax(X, 0.5 * (aabb[e * 2 * d + d + c] - aabb[e * 2 * d + c]));
      for (int k = 0; k < d; ++k) o[9 + c * 3 + k] = (float)obb_A[(e * d + c) * d + k];
    }
    o[18] = (float)(X * (1.0 + 1e-6));
    o[19] = (float)(lin[e * kLin + 12] * (1.0 + 1e-6));
    for (int c = 0; c < d; ++c) {
      o[20 + c] = (float)(lin[e * kLin + c] - elem_ref(aabb, d, e, c));
      for (int q = 0; q < d; ++q) o[23 + c * 3 + q] = (float)lin[e * kLin + 3 + c * 3 + q];
    }
  }
}

template <typename T>
int dev_alloc(T** p, size_t count, size_t* bytes) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return FP_ENOMEM;
  }
  *bytes += count * sizeof(T);
  return FP_OK;
}

void free_mesh_memory(fp_mesh_s* m) {
  timer_free(m);
  cudaFree(m->coords);
  cudaFree(m->coords32);
  cudaFree(m->coords32p);
  cudaFree(m->aabb);
  cudaFree(m->obb_c);
  cudaFree(m->obb_A);
  cudaFree(m->box32);
  cudaFree(m->curv);
  cudaFree(m->cell_start);
  cudaFree(m->cell_elems);
  cudaFree(m->status);
}

int build_boxes_and_grid(fp_mesh_s* m, cudaStream_t st);

}  // namespace
}  // namespace fp

fp::DevMesh fp_mesh_s::view() const {
  fp::DevMesh v;
  v.coords = coords;
  v.coords32 = coords32;
  v.coords32p = coords32p;
  v.aabb = aabb;
  v.obb_c = obb_c;
  v.obb_A = obb_A;
  v.box32 = box32;
  v.curv = curv;
  v.cell_start = cell_start;
  v.cell_elems = cell_elems;
  v.NE = NE;
  v.cstride = NE * (int64_t)ne;
  v.cstride32p = NE * (int64_t)(fp::pitch32(N) * fp::ipow(N, dr - 1));
  for (int c = 0; c < 3; ++c) {
    v.lo[c] = lo[c];
    v.hi[c] = hi[c];
    v.scale[c] = scale[c];
  }
  v.NL = NL;
  v.max_iter = opts.max_iter;
  v.newton_tol = opts.newton_tol;
  v.dist_tol = opts.dist_tol;
  v.status = status;
  return v;
}

namespace fp {
namespace {

int build_boxes_and_grid(fp_mesh_s* m, cudaStream_t st) {
  // element boxes
  const std::vector<double> htab = bound_tables(m->N, m->M);
  double* dtab = nullptr;
  double* dlin = nullptr;  // per element x(0) and the OBB frame T, for box32
  FP_CUDA_TRY(cudaMalloc(&dtab, htab.size() * sizeof(double)));
  if (cudaMalloc(&dlin, sizeof(double) * kLin * m->NE) != cudaSuccess) {
    cudaFree(dtab);
    return FP_ENOMEM;
  }
  int rc = FP_OK;
  // setup timing (fp_mesh_info): k_boxes, and the Psi_L build
  cudaEvent_t ev[4] = {};
  bool timed = true;
  for (auto& e : ev) timed &= cudaEventCreate(&e) == cudaSuccess;
  do {
    if (cudaMemcpyAsync(dtab, htab.data(), htab.size() * sizeof(double), cudaMemcpyHostToDevice, st) !=
        cudaSuccess) {
      rc = FP_ELAUNCH;
      break;
    }
    if (timed) cudaEventRecord(ev[0], st);
    rc = dispatch_shape(m->N, m->d, m->dr, [&](auto Nc, auto Dc, auto DRc) -> int {
      constexpr int N = decltype(Nc)::value, D = decltype(Dc)::value, DR = decltype(DRc)::value;
      k_boxes<N, D, DR><<<(unsigned)m->NE, kBoxThreads, 0, st>>>(
          m->coords, m->NE, dtab, m->M, m->basis, m->opts.bbox_tol, curvature_factor(N, DR), m->aabb,
          m->obb_c, m->obb_A, dlin, m->status);
      return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ELAUNCH;
    });
    if (rc != FP_OK) break;
    if (timed) cudaEventRecord(ev[1], st);
    // volumes: the curvature bound of the FP64 certified stop (after the timed k_boxes)
    if (m->d == m->dr) {
      double Ls[3];
      basis_sums(m->N, Ls);
      const double lam = Ls[0];
      double S = 0.0;
      for (int i = 0; i < m->N; ++i) {
        double a = 0.0;
        for (int k = 0; k < m->N; ++k) a += fabs(m->basis.dn[i * m->N + k]);
        S = std::max(S, a);
      }
      const double lam_dr = pow(lam, m->dr);
      const double rslack = 2.0 * m->N * 1.1102230246251565e-16 * S * S * lam_dr * m->dr * m->dr;
      rc = dispatch_shape(m->N, m->d, m->dr, [&](auto Nc, auto Dc, auto DRc) -> int {
        constexpr int N = decltype(Nc)::value, D = decltype(Dc)::value, DR = decltype(DRc)::value;
        if constexpr (D == DR) {
          k_curvature<N, D><<<(unsigned)m->NE, kBoxThreads, 0, st>>>(m->coords, m->NE, m->basis, lam_dr,
                                                                     rslack, m->curv);
          return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ELAUNCH;
        }
        return FP_OK;
      });
      if (rc != FP_OK) break;
    }
    // grid bounds = union of the expanded AABBs
    double* dbounds = nullptr;
    if (cudaMalloc(&dbounds, 6 * sizeof(double)) != cudaSuccess) {
      rc = FP_ENOMEM;
      break;
    }
    if (timed) cudaEventRecord(ev[2], st);
    k_grid_bounds<<<1, 1024, 0, st>>>(m->aabb, m->NE, m->d, dbounds);
    double hb[6];
    cudaError_t ce = cudaMemcpyAsync(hb, dbounds, sizeof(hb), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    cudaFree(dbounds);
    if (ce != cudaSuccess) {
      rc = FP_ELAUNCH;
      break;
    }
    int NL = m->opts.n_grid;
    if (NL <= 0) {
      NL = 1;
      while (true) {
        int64_t p = 1;
        for (int c = 0; c < m->d; ++c) p *= NL;
        if (p >= m->NE) break;
        ++NL;
      }
    }
    int64_t ncell = 1;
    for (int c = 0; c < m->d; ++c) ncell *= NL;
    if (ncell > (int64_t)1 << 28) {
      rc = FP_EINVAL;
      break;
    }
    m->NL = NL;
    m->ncell = ncell;
    GridView g;
    g.NL = NL;
    g.d = m->d;
    for (int c = 0; c < 3; ++c) {
      m->lo[c] = (c < m->d) ? hb[c] : 0.0;
      m->hi[c] = (c < m->d) ? hb[3 + c] : 0.0;
      const double ext = m->hi[c] - m->lo[c];
      m->scale[c] = (c < m->d && ext > 0.0) ? (double)NL / ext : 0.0;
      g.lo[c] = m->lo[c];
      g.scale[c] = m->scale[c];
    }
    int* counts = nullptr;
    if ((rc = dev_alloc(&m->cell_start, ncell + 1, &m->bytes)) != FP_OK) break;
    if (cudaMalloc(&counts, ncell * sizeof(int)) != cudaSuccess) {
      rc = FP_ENOMEM;
      break;
    }
    const int eb = grid_for(m->NE, 256, 148 * 16);
    cudaMemsetAsync(counts, 0, ncell * sizeof(int), st);
    k_grid_scatter<0><<<eb, 256, 0, st>>>(m->aabb, m->NE, g, counts, nullptr, nullptr);
    k_scan<<<1, 1024, 0, st>>>(counts, ncell, m->cell_start);
    int nnz = 0;
    ce = cudaMemcpyAsync(&nnz, m->cell_start + ncell, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess || nnz < 0) {
      cudaFree(counts);
      rc = ce != cudaSuccess ? FP_ELAUNCH : FP_ENOMEM;
      break;
    }
    m->nnz = nnz;
    if ((rc = dev_alloc(&m->cell_elems, (size_t)nnz, &m->bytes)) != FP_OK) {
      cudaFree(counts);
      break;
    }
    cudaMemsetAsync(counts, 0, ncell * sizeof(int), st);
    k_grid_scatter<1><<<eb, 256, 0, st>>>(m->aabb, m->NE, g, counts, m->cell_start, m->cell_elems);
    k_grid_sort<<<grid_for(ncell, 256, 148 * 16), 256, 0, st>>>(m->cell_start, ncell, m->cell_elems);
    if (timed) cudaEventRecord(ev[3], st);
    if ((rc = dev_alloc(&m->box32, (size_t)m->NE * BOX32, &m->bytes)) != FP_OK) {
      cudaFree(counts);
      break;
    }
    k_box32<<<grid_for(m->NE, 256, 148 * 16), 256, 0, st>>>(m->aabb, m->obb_c, m->obb_A, dlin, m->NE,
                                                            m->d, m->box32);
    ce = cudaStreamSynchronize(st);
    cudaFree(counts);
    if (ce != cudaSuccess) rc = FP_ELAUNCH;
  } while (0);
  cudaStreamSynchronize(st);
  if (timed && rc == FP_OK) {
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, ev[0], ev[1]) == cudaSuccess) m->setup_ms[0] = a;
    if (cudaEventElapsedTime(&b, ev[2], ev[3]) == cudaSuccess) m->setup_ms[1] = b;
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  cudaFree(dtab);
  cudaFree(dlin);
  return rc;
}

}  // namespace
}  // namespace fp

extern "C" void fp_opts_default(fp_opts* o) {
  if (!o) return;
  o->bbox_tol = 0.1;
  o->M = 0;
  o->n_grid = 0;
  o->newton_tol = 1e-10;
  o->max_iter = 50;
  o->dist_tol = 1e-10;
  o->precision = FP_F64;
  o->point_order = FP_ORDER_CELL;
}

namespace {

// Find calls take their scratch (the cell order, the mixed path's queue,
// the host path's buffers) from the device's default stream-ordered pool;
// by default the pool hands freed memory back at every synchronisation, so
// each call would pay a fresh allocation.  Keeping up to 1 GiB of freed
// scratch in the pool (per process, per device) lets calls reuse it.
void keep_pool_memory() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = (uint64_t)1 << 30;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  done[dev] = true;
}

}  // namespace

extern "C" int fp_setup(const double* coords_dev, int d, int dr, int order, int64_t NE,
                        const fp_opts* opts, void* stream, fp_mesh* out) {
  using namespace fp;
  if (!out) return FP_EINVAL;
  keep_pool_memory();
  *out = nullptr;
  if (!coords_dev || NE <= 0 || NE > INT32_MAX) return FP_EINVAL;
  if (!((d == 2 && dr == 2) || (d == 3 && dr == 3) || (d == 3 && dr == 2) || (dr == 1 && (d == 2 || d == 3))))
    return FP_EINVAL;
  const int N = order + 1;
  if (order < 1) return FP_EINVAL;
  if (N > FP_MAX_N) return FP_EUNSUPPORTED;
  fp_opts o;
  fp_opts_default(&o);
  if (opts) o = *opts;
  if (o.M == 0) o.M = 2 * N;
  if (o.M < 2 || o.M > kMaxM || !(o.bbox_tol >= 0.0) || o.max_iter < 1 || !(o.newton_tol > 0.0) ||
      o.n_grid < 0 || (o.precision != FP_F64 && o.precision != FP_MIXED) ||
      (o.point_order != FP_ORDER_GIVEN && o.point_order != FP_ORDER_CELL))
    return FP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  fp_mesh_s* m = (fp_mesh_s*)calloc(1, sizeof(fp_mesh_s));
  if (!m) return FP_ENOMEM;
  m->d = d;
  m->dr = dr;
  m->N = N;
  m->ne = ipow(N, dr);
  m->M = o.M;
  m->NE = NE;
  m->opts = o;
  m->precision = o.precision;
  host_basis_tab(N, &m->basis);
  const size_t nc = (size_t)d * NE * m->ne;
  const size_t nc32p = (size_t)d * NE * (pitch32(N) * ipow(N, dr - 1));
  int rc = FP_OK;
  do {
    if ((rc = dev_alloc(&m->coords, nc, &m->bytes)) != FP_OK) break;
    if ((rc = dev_alloc(&m->coords32, nc, &m->bytes)) != FP_OK) break;
    if ((rc = dev_alloc(&m->coords32p, nc32p, &m->bytes)) != FP_OK) break;
    if ((rc = dev_alloc(&m->aabb, (size_t)NE * 2 * d, &m->bytes)) != FP_OK) break;
    if ((rc = dev_alloc(&m->obb_c, (size_t)NE * d, &m->bytes)) != FP_OK) break;
    if ((rc = dev_alloc(&m->obb_A, (size_t)NE * d * d, &m->bytes)) != FP_OK) break;
    if ((rc = dev_alloc(&m->status, 1, &m->bytes)) != FP_OK) break;
    if ((rc = dev_alloc(&m->curv, (size_t)NE, &m->bytes)) != FP_OK) break;
    if (cudaMemsetAsync(m->status, 0, sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(m->curv, 0, (size_t)NE * sizeof(float), st) != cudaSuccess ||
        cudaMemcpyAsync(m->coords, coords_dev, nc * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess) {
      rc = FP_ELAUNCH;
      break;
    }
    if ((rc = build_boxes_and_grid(m, st)) != FP_OK) break;
    k_coords32<<<grid_for((int64_t)nc, 256, 148 * 16), 256, 0, st>>>(m->coords, m->aabb, d, NE, m->ne,
                                                                    m->coords32);
    k_coords32p<<<grid_for((int64_t)nc32p, 256, 148 * 16), 256, 0, st>>>(m->coords32, (int64_t)d * NE, N,
                                                                        ipow(N, dr - 1), m->coords32p);
    int hstat = 0;
    if (cudaMemcpyAsync(&hstat, m->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = FP_ELAUNCH;
      break;
    }
    if (hstat != 0) rc = FP_EINVAL;  // a degenerate element (singular J at its centre)
  } while (0);
  if (rc != FP_OK) {
    cudaStreamSynchronize(st);
    free_mesh_memory(m);
    free(m);
    return rc;
  }
  *out = m;
  return FP_OK;
}

extern "C" int fp_free(fp_mesh m) {
  if (!m) return FP_EINVAL;
  cudaDeviceSynchronize();
  fp::free_mesh_memory(m);
  free(m);
  return FP_OK;
}

extern "C" int fp_get_info(fp_mesh m, fp_mesh_info* info) {
  if (!m || !info) return FP_EINVAL;
  memset(info, 0, sizeof(*info));
  info->d = m->d;
  info->dr = m->dr;
  info->N = m->N;
  info->M = m->M;
  info->n_grid = m->NL;
  info->NE = m->NE;
  info->n_cells = m->ncell;
  info->n_cell_entries = m->nnz;
  for (int c = 0; c < 3; ++c) {
    info->grid_lo[c] = m->lo[c];
    info->grid_hi[c] = m->hi[c];
  }
  info->device_bytes = m->bytes;
  info->setup_boxes_ms = m->setup_ms[0];
  info->setup_grid_ms = m->setup_ms[1];
  return FP_OK;
}

extern "C" int fp_get_boxes(fp_mesh m, double* aabb, double* obb_c, double* obb_A, void* stream) {
  if (!m) return FP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t d = m->d;
  if (aabb) FP_CUDA_TRY(cudaMemcpyAsync(aabb, m->aabb, m->NE * 2 * d * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (obb_c) FP_CUDA_TRY(cudaMemcpyAsync(obb_c, m->obb_c, m->NE * d * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (obb_A) FP_CUDA_TRY(cudaMemcpyAsync(obb_A, m->obb_A, m->NE * d * d * sizeof(double), cudaMemcpyDeviceToDevice, st));
  FP_CUDA_TRY(cudaStreamSynchronize(st));
  return FP_OK;
}

namespace {
__global__ void k_get_curvature(const float* __restrict__ curv, int64_t NE, double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < NE; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (double)curv[e];
}
}  // namespace

extern "C" int fp_get_curvature(fp_mesh m, double* curv_dev, void* stream) {
  if (!m || !curv_dev) return FP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  k_get_curvature<<<fp::grid_for(m->NE, 256, 148 * 8), 256, 0, st>>>(m->curv, m->NE, curv_dev);
  FP_CUDA_TRY(cudaGetLastError());
  FP_CUDA_TRY(cudaStreamSynchronize(st));
  return FP_OK;
}

extern "C" int fp_get_grid(fp_mesh m, int32_t* cell_start, int32_t* cell_elems, void* stream) {
  if (!m) return FP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cell_start)
    FP_CUDA_TRY(cudaMemcpyAsync(cell_start, m->cell_start, (m->ncell + 1) * sizeof(int), cudaMemcpyDeviceToDevice, st));
  if (cell_elems && m->nnz > 0)
    FP_CUDA_TRY(cudaMemcpyAsync(cell_elems, m->cell_elems, m->nnz * sizeof(int), cudaMemcpyDeviceToDevice, st));
  FP_CUDA_TRY(cudaStreamSynchronize(st));
  return FP_OK;
}

extern "C" int fp_device_status(fp_mesh m, int* status, void* stream) {
  if (!m || !status) return FP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  FP_CUDA_TRY(cudaMemcpyAsync(status, m->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  FP_CUDA_TRY(cudaMemsetAsync(m->status, 0, sizeof(int), st));
  FP_CUDA_TRY(cudaStreamSynchronize(st));
  return FP_OK;
}

extern "C" const char* fp_status_string(int s) {
  switch (s) {
    case FP_OK: return "ok";
    case FP_EINVAL: return "invalid argument";
    case FP_ENOMEM: return "out of device memory or over budget";
    case FP_ELAUNCH: return "kernel launch or CUDA runtime failure";
    case FP_EDEVICE: return "a kernel recorded a device error";
    case FP_ETIMEDOUT: return "timed out";
    case FP_EBUSY: return "busy";
    case FP_EUNSUPPORTED: return "element type or order not supported";
    case FP_ECANCELED: return "request cancelled";
    default: return "unknown status";
  }
}
