// x(r) and G(r) of hex elements computed by the whole warp for the few lanes
// that need them (the tail of a launch, a follow-up over few points).
//
// A launch ends with the slowest points of its last warps, each round of
// which is a full evaluation (about 1,200 FP64 instructions at N = 5) that
// costs the FP64 pipe the same time with one lane active as with 32.  When
// at most kCoopLanes lanes of a warp need an evaluation, the warp takes
// them one at a time and splits each: lane l forms the i-sums of the (j, k)
// row pairs l, l + 32, ..., lane k then the j-sums of row k, and every lane
// the k-sums, with the rows passed by shuffles.  Each sum is the same chain
// of FMAs, in the same order, as in map_eval_rolled, so the result is
// bit-identical to the lane's own evaluation (the outputs do not depend on
// which path ran).  About 45 FP64 instructions per component, plus one
// basis evaluation (three lanes, one direction each), instead of
// N^2 (2N + 3) + 4N per component.
#pragma once
#include "fp_basis.cuh"

namespace fp {

constexpr int kCoopLanes = 6;

template <int N, int D>
__device__ __forceinline__ void coop_eval_hex(bool want, const double* __restrict__ X, int64_t cs,
                                              const BasisTab& B, const double (&re)[3], double (&xo)[D],
                                              double (&Go)[D * 3]) {
  constexpr unsigned kAll = 0xffffffffu;
  constexpr int NP = N * N;             // (j, k) row pairs
  constexpr int NS = (NP + 31) / 32;    // pairs per lane
  const int lane = threadIdx.x & 31;
  unsigned mask = __ballot_sync(kAll, want);
  while (mask) {
    const int src = __ffs(mask) - 1;
    mask &= mask - 1;
    const double* Xs = reinterpret_cast<const double*>(
        __shfl_sync(kAll, reinterpret_cast<unsigned long long>(X), src));
    const int64_t css = __shfl_sync(kAll, (long long)cs, src);
    // lane d < 3 evaluates the basis along direction d at the owner's r_d
    // (the same basis call as the owner's own evaluation); the others
    // take the values by shuffles
    double rd = __shfl_sync(kAll, re[0], src);
    const double r1 = __shfl_sync(kAll, re[1], src), r2 = __shfl_sync(kAll, re[2], src);
    if (lane == 1) rd = r1;
    if (lane == 2) rd = r2;
    double bph[N], bdph[N];
    lagrange_sym<N, double>(B, rd, bph, bdph);
    const int kl = lane < N ? lane : 0;  // the row k whose j-sums this lane forms
#pragma unroll 1
    for (int c = 0; c < D; ++c) {
      const double* xe = Xs + c * css;
      double a[NS], b[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) a[s] = b[s] = 0.0;
      // the shuffles are executed by every lane, outside the guarded loads
      // (a warp collective must not sit in a branch that only some lanes take)
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const double pi = __shfl_sync(kAll, bph[i], 0), qi = __shfl_sync(kAll, bdph[i], 0);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          const int q = lane + 32 * s;
          if (q < NP) {
            const int j = q % N, k = q / N;
            const double v = __ldg(xe + (k * N + j) * N + i);
            a[s] = fma(v, pi, a[s]);
            b[s] = fma(v, qi, b[s]);
          }
        }
      }
      double ak = 0.0, bk = 0.0, ck = 0.0;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const int q = j + N * kl;
        double aj = __shfl_sync(kAll, a[0], q & 31), bj = __shfl_sync(kAll, b[0], q & 31);
#pragma unroll
        for (int s = 1; s < NS; ++s) {
          const double as = __shfl_sync(kAll, a[s], q & 31), bs = __shfl_sync(kAll, b[s], q & 31);
          if ((q >> 5) == s) {
            aj = as;
            bj = bs;
          }
        }
        const double p1 = __shfl_sync(kAll, bph[j], 1), q1 = __shfl_sync(kAll, bdph[j], 1);
        ak = fma(aj, p1, ak);
        bk = fma(bj, p1, bk);
        ck = fma(aj, q1, ck);
      }
      double xv = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const double akk = __shfl_sync(kAll, ak, k), bkk = __shfl_sync(kAll, bk, k),
                     ckk = __shfl_sync(kAll, ck, k);
        const double tk = __shfl_sync(kAll, bph[k], 2), dtk = __shfl_sync(kAll, bdph[k], 2);
        xv = fma(akk, tk, xv);
        g0 = fma(bkk, tk, g0);
        g1 = fma(ckk, tk, g1);
        g2 = fma(akk, dtk, g2);
      }
      if (lane == src) {
#pragma unroll
        for (int cc = 0; cc < D; ++cc)
          if (cc == c) {
            xo[cc] = xv;
            Go[cc * 3 + 0] = g0;
            Go[cc * 3 + 1] = g1;
            Go[cc * 3 + 2] = g2;
          }
      }
    }
  }
}

}  // namespace fp
