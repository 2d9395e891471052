// Find (Sec. 3.2): cell lookup in Psi_L, AABB + OBB filter, trust-region
// Newton (Sec. 3.2.1) in each candidate, selection of the result.
//
// FP64 path: one thread per point.  On this GPU the FP64 FMA pipe (about
// 1.1 TFLOP/s, 1/62 of FP32) bounds the kernel, and an inactive lane costs
// the same issue slot as an active one, so the contractions are
// sum-factorised and every step mirrors the FP64 definition exactly (same
// decisions, same order).
#include <math.h>

#include "fp_basis.cuh"
#include "fp_common.cuh"

namespace fp {

constexpr int kFindThreads = 128;

// Solves H_FF s_F = -g_F on the free coordinates (held ones get s = 0): the
// held rows and columns are replaced by the identity, which leaves the free
// block's leading minors unchanged.
template <int DR, typename T>
__device__ __forceinline__ bool masked_solve(const T (&H)[DR][DR], const bool (&held)[DR],
                                             const T (&g)[DR], T (&s)[DR]) {
  T A[DR][DR], b[DR];
#pragma unroll
  for (int j = 0; j < DR; ++j) {
#pragma unroll
    for (int k = 0; k < DR; ++k)
      A[j][k] = (held[j] || held[k]) ? (j == k ? T(1) : T(0)) : H[j][k];
    b[j] = held[j] ? T(0) : -g[j];
  }
  if (!spd_solve<DR, T>(A, b, s)) return false;
#pragma unroll
  for (int j = 0; j < DR; ++j)
    if (held[j]) s[j] = T(0);
  return true;
}

// Per-thread counters: [0] candidates, [1] iterations, [2] rejected steps,
// [3] beta = 1 iterations, [4] FP64 iterations (mixed), [5] FP64 rechecks.
struct Counters {
  unsigned v[6];
  __device__ Counters() {
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = 0;
  }
  __device__ void flush(unsigned long long* stats) {
    if (!stats) return;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      unsigned x = v[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) == 0 && x) atomicAdd(stats + i, (unsigned long long)x);
    }
  }
};

// Trust-region Newton of Sec. 3.2.1 for point xs in the element whose data
// starts at X (component c at X + c*cs).  The steps, in order:
//  r_0 = the closest GLL node (squared distances in non-contracted FP64,
//        ties to the lowest node index);
//  each iteration: gradient g = -G^T dx; Hessian G^T G, minus
//        sum_c dx_c d2x_c/dr dr when beta = 1 (l > 0 and r on the boundary);
//        coordinates at a bound whose gradient points outwards are held;
//        solve on the free block (beta = 0 block if the beta = 1 block is not
//        positive definite; no step if neither is); clip to [-alpha, alpha];
//        project on [-1,1]; stop once |dr|_inf < tol (that step is taken and
//        x(r*) evaluated); stop if the predicted decrease
//        -2 g.dr - dr^T H dr is not positive; ratio test 0.9 / 0.01 with
//        alpha x2 / kept / /4 and reject; a full-length step whose predicted
//        decrease is below 1e-12 X |dx| (the rounding level of the measured
//        decrease) is accepted.
// Returns the iteration count; r and F = |dx|^2 at the final point.
template <int N, int D, int DR>
__device__ int newton_f64(const double* __restrict__ X, int64_t cs, const BasisTab& B,
                          const double (&xs)[D], double xscale, double tol, int max_iter,
                          double (&r)[DR], double& Fout, Counters& cnt) {
  constexpr int NN = (DR == 3) ? N * N * N : N * N;
  double best = INFINITY;
  int nb = 0;
#pragma unroll 5
  for (int n = 0; n < NN; ++n) {
    double dd = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const double t = __dsub_rn(xs[c], ldg(X + c * cs + n));
      dd = __dadd_rn(dd, __dmul_rn(t, t));
    }
    if (dd < best) {
      best = dd;
      nb = n;
    }
  }
  {
    const int idx[3] = {nb % N, (nb / N) % N, nb / (N * N)};
#pragma unroll
    for (int j = 0; j < DR; ++j) {
      double v = 0.0;
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i == idx[j]) v = B.z[i];
      r[j] = v;
    }
  }
  double alpha = 1.0;
  double ph[DR][N], dph[DR][N];
  double x[D], G[D * DR], dx[D], F = 0.0;
#pragma unroll
  for (int j = 0; j < DR; ++j) lagrange<N, double>(B.z, B.w, r[j], ph[j], dph[j]);
  map_eval<N, DR, D, true, double>(X, cs, ph, dph, x, G);
#pragma unroll
  for (int c = 0; c < D; ++c) {
    dx[c] = xs[c] - x[c];
    F += dx[c] * dx[c];
  }
  int it = 0;
  for (int l = 0; l < max_iter; ++l) {
    bool at_bound = false;
#pragma unroll
    for (int j = 0; j < DR; ++j) at_bound |= (r[j] == -1.0 || r[j] == 1.0);
    const bool beta = (l > 0) && at_bound;
    double g[DR];
    bool held[DR];
#pragma unroll
    for (int j = 0; j < DR; ++j) {
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c) s -= G[c * DR + j] * dx[c];
      g[j] = s;
      held[j] = (r[j] == -1.0 && s > 0.0) || (r[j] == 1.0 && s < 0.0);
    }
    double HGN[DR][DR], H[DR][DR];
#pragma unroll
    for (int j = 0; j < DR; ++j)
#pragma unroll
      for (int k = 0; k < DR; ++k) {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) s += G[c * DR + j] * G[c * DR + k];
        HGN[j][k] = s;
        H[j][k] = s;
      }
    if (beta) {
      double d2[DR][N], S[D * DR * DR];
#pragma unroll
      for (int j = 0; j < DR; ++j) lagrange2<N, double>(B.z, B.w, r[j], ph[j], dph[j], d2[j]);
      map_hess<N, DR, D, double>(X, cs, ph, dph, d2, S);
#pragma unroll
      for (int j = 0; j < DR; ++j)
#pragma unroll
        for (int k = 0; k < DR; ++k) {
          double s = 0.0;
#pragma unroll
          for (int c = 0; c < D; ++c) s += dx[c] * S[(c * DR + j) * DR + k];
          H[j][k] -= s;
        }
    }
    double step[DR];
    bool used_beta = beta;
    bool ok = masked_solve<DR, double>(H, held, g, step);
    if (!ok && beta) {
      used_beta = false;
      ok = masked_solve<DR, double>(HGN, held, g, step);
    }
    if (!ok) {
      used_beta = false;
#pragma unroll
      for (int j = 0; j < DR; ++j) step[j] = 0.0;
    }
    double rn[DR], ds[DR], mx = 0.0;
    bool clipped = false;
#pragma unroll
    for (int j = 0; j < DR; ++j) {
      double s = step[j];
      if (s > alpha) {
        s = alpha;
        clipped = true;
      }
      if (s < -alpha) {
        s = -alpha;
        clipped = true;
      }
      double v = r[j] + s;
      if (v > 1.0) v = 1.0;
      if (v < -1.0) v = -1.0;
      rn[j] = v;
      ds[j] = v - r[j];
      mx = fmax(mx, fabs(ds[j]));
    }
    if (mx < tol) {
      ++it;
      ++cnt.v[1];
#pragma unroll
      for (int j = 0; j < DR; ++j) {
        r[j] = rn[j];
        lagrange<N, double>(B.z, B.w, r[j], ph[j], dph[j]);
      }
      map_eval<N, DR, D, false, double>(X, cs, ph, dph, x, nullptr);
      F = 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const double t = xs[c] - x[c];
        F += t * t;
      }
      break;
    }
    double lin = 0.0, quad = 0.0;
#pragma unroll
    for (int j = 0; j < DR; ++j) lin += g[j] * ds[j];
    if (used_beta) {
#pragma unroll
      for (int j = 0; j < DR; ++j)
#pragma unroll
        for (int k = 0; k < DR; ++k) quad += ds[j] * H[j][k] * ds[k];
    } else {
#pragma unroll
      for (int c = 0; c < D; ++c) {
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < DR; ++j) t += G[c * DR + j] * ds[j];
        quad += t * t;
      }
    }
    const double pred = -2.0 * lin - quad;
    if (!(pred > 0.0)) break;
    ++it;
    ++cnt.v[1];
    if (beta) ++cnt.v[3];
    double xn[D], Gn[D * DR], dxn[D], Fn = 0.0;
#pragma unroll
    for (int j = 0; j < DR; ++j) lagrange<N, double>(B.z, B.w, rn[j], ph[j], dph[j]);
    map_eval<N, DR, D, true, double>(X, cs, ph, dph, xn, Gn);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      dxn[c] = xs[c] - xn[c];
      Fn += dxn[c] * dxn[c];
    }
    const double decr = F - Fn;
    const double tau = 1e-12 * xscale * sqrt(F);
    bool accept;
    if (!clipped && pred < tau) {
      accept = true;
    } else if (decr >= 0.9 * pred) {
      alpha *= 2.0;
      accept = true;
    } else if (decr >= 0.01 * pred) {
      accept = true;
    } else {
      alpha *= 0.25;
      accept = false;
      ++cnt.v[2];
    }
    if (accept) {
#pragma unroll
      for (int j = 0; j < DR; ++j) r[j] = rn[j];
#pragma unroll
      for (int c = 0; c < D; ++c) dx[c] = dxn[c];
#pragma unroll
      for (int q = 0; q < D * DR; ++q) G[q] = Gn[q];
      F = Fn;
    }
  }
  Fout = F;
  return it;
}

// Eq. AABB_test (as lo <= x <= hi) and Eq. OBB_test on the expanded boxes,
// with the same rounded operations as the FP64 definition.
template <int D>
__device__ __forceinline__ bool in_boxes_f64(const DevMesh& m, int64_t e, const double (&xs)[D]) {
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const double lo = __ldg(m.aabb + e * 2 * D + c), hi = __ldg(m.aabb + e * 2 * D + D + c);
    if (!(xs[c] >= lo && xs[c] <= hi)) return false;
  }
#pragma unroll
  for (int c = 0; c < D; ++c) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < D; ++q)
      s = __dadd_rn(s, __dmul_rn(__ldg(m.obb_A + (e * D + c) * D + q),
                                 __dsub_rn(xs[q], __ldg(m.obb_c + e * D + q))));
    if (!(fabs(s) <= 1.0)) return false;
  }
  return true;
}

template <int D>
__device__ __forceinline__ double aabb_scale(const DevMesh& m, int64_t e) {
  double X = 0.0;
#pragma unroll
  for (int c = 0; c < 2 * D; ++c) X = fmax(X, fabs(__ldg(m.aabb + e * 2 * D + c)));
  return X;
}

// Psi_L cell of x, or -1 when x lies outside the grid (then outside every
// AABB) or has a non-finite coordinate.
template <int D>
__device__ __forceinline__ int64_t point_cell(const DevMesh& m, const double (&xs)[D]) {
  int64_t cell = 0, mul = 1;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    if (!(xs[c] >= m.lo[c] && xs[c] <= m.hi[c])) return -1;
    cell += mul * cell_coord(xs[c], m.lo[c], m.scale[c], m.NL);
    mul *= m.NL;
  }
  return cell;
}

template <int N, int D, int DR>
__global__ void __launch_bounds__(kFindThreads)
    k_find_f64(const DevMesh m, const BasisTab B, const double* __restrict__ pts, int64_t n,
               int* __restrict__ code, int* __restrict__ elem, double* __restrict__ rout,
               double* __restrict__ dist2, unsigned long long* stats) {
  constexpr int NN = (DR == 3) ? N * N * N : N * N;
  Counters cnt;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    double xs[D];
#pragma unroll
    for (int c = 0; c < D; ++c) xs[c] = __ldg(pts + p * D + c);
    int bcode = FP_NOT_FOUND, be = -1;
    double br[DR], bd = INFINITY;
#pragma unroll
    for (int j = 0; j < DR; ++j) br[j] = 0.0;
    const int64_t cell = point_cell<D>(m, xs);
    if (cell >= 0) {
      const int q0 = __ldg(m.cell_start + cell), q1 = __ldg(m.cell_start + cell + 1);
      for (int q = q0; q < q1; ++q) {
        const int e = __ldg(m.cell_elems + q);
        if (e < 0 || e >= m.NE) {
          record_status(m.status, FP_DEV_BAD_ELEM);
          continue;
        }
        if (!in_boxes_f64<D>(m, e, xs)) continue;
        ++cnt.v[0];
        double rr[DR], dd;
        newton_f64<N, D, DR>(m.coords + (int64_t)e * NN, m.cstride, B, xs, aabb_scale<D>(m, e),
                             m.newton_tol, m.max_iter, rr, dd, cnt);
        bool inside = true;
#pragma unroll
        for (int j = 0; j < DR; ++j) inside &= fabs(rr[j]) < 1.0;
        if (DR < D) inside &= dd < m.dist_tol;
        if (inside) {
          bcode = FP_INTERIOR;
          be = e;
          bd = dd;
#pragma unroll
          for (int j = 0; j < DR; ++j) br[j] = rr[j];
          break;
        }
        if (dd < bd) {
          bcode = FP_BORDER;
          be = e;
          bd = dd;
#pragma unroll
          for (int j = 0; j < DR; ++j) br[j] = rr[j];
        }
      }
    }
    code[p] = bcode;
    elem[p] = be;
#pragma unroll
    for (int j = 0; j < DR; ++j) rout[p * DR + j] = br[j];
    dist2[p] = bd;
  }
  cnt.flush(stats);
}

int find_f64(const fp_mesh_s* m, const double* pts, int64_t n, int* code, int* elem, double* r,
             double* dist2, unsigned long long* stats, cudaStream_t st) {
  const DevMesh v = m->view();
  return dispatch_shape(m->N, m->d, m->dr, [&](auto Nc, auto Dc, auto DRc) -> int {
    constexpr int N = decltype(Nc)::value, D = decltype(Dc)::value, DR = decltype(DRc)::value;
    const int blocks = grid_for(n, kFindThreads, 148 * 64);
    k_find_f64<N, D, DR><<<blocks, kFindThreads, 0, st>>>(v, m->basis, pts, n, code, elem, r, dist2, stats);
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ELAUNCH;
  });
}

int find_mixed(const fp_mesh_s* m, const double* pts, int64_t n, int* code, int* elem, double* r,
               double* dist2, unsigned long long* stats, cudaStream_t st);

}  // namespace fp

// Nothing extra to prepare until the mixed path lands.
int fp_mixed_prepare(fp_mesh_s* m, cudaStream_t st) {
  (void)m;
  (void)st;
  return FP_OK;
}

int fp::find_mixed(const fp_mesh_s* m, const double* pts, int64_t n, int* code, int* elem, double* r,
                   double* dist2, unsigned long long* stats, cudaStream_t st) {
  return find_f64(m, pts, n, code, elem, r, dist2, stats, st);
}

static int findpts_impl(fp_mesh m, const double* pts, int64_t n, int32_t* code, int32_t* elem,
                        double* r, double* dist2, uint64_t* stats, void* stream) {
  if (!m || n < 0) return FP_EINVAL;
  if (n == 0) return FP_OK;
  if (!pts || !code || !elem || !r || !dist2) return FP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  auto* s = reinterpret_cast<unsigned long long*>(stats);
  if (m->precision == FP_MIXED) return fp::find_mixed(m, pts, n, code, elem, r, dist2, s, st);
  return fp::find_f64(m, pts, n, code, elem, r, dist2, s, st);
}

extern "C" int fp_findpts(fp_mesh m, const double* pts, int64_t n, int32_t* code, int32_t* elem,
                          double* r, double* dist2, void* stream) {
  return findpts_impl(m, pts, n, code, elem, r, dist2, nullptr, stream);
}

extern "C" int fp_findpts_stats(fp_mesh m, const double* pts, int64_t n, int32_t* code,
                                int32_t* elem, double* r, double* dist2, uint64_t* stats,
                                void* stream) {
  if (!stats) return FP_EINVAL;
  return findpts_impl(m, pts, n, code, elem, r, dist2, stats, stream);
}

extern "C" int fp_set_precision(fp_mesh m, int precision) {
  if (!m || (precision != FP_F64 && precision != FP_MIXED)) return FP_EINVAL;
  m->precision = precision;
  return FP_OK;
}
