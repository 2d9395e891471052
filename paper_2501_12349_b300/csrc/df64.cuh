// Double-float arithmetic on the FP32 pipe: a value is an unevaluated pair
// hi + lo of floats, |lo| <= ulp(hi) / 2, carrying about 48 significant bits.
// On this GPU the FP32 pipe issues about 64 times the FP64 pipe's operations,
// so a double-float multiply-add (about 12 FP32 operations) costs a fifth of
// an FP64 one.  The error-free transformations used (Knuth's two-sum, the
// FMA two-product, Dekker's fast two-sum for |a| >= |b|) and the compensated
// dot product built from them (Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26 (2005), Algorithm Dot2 with the
// products' low parts added) are written with the _rn intrinsics so that the
// compiler neither contracts nor reorders them.
#pragma once
#include "fp_common.cuh"

namespace fp {

struct df {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  return fast_two_sum(p, e);
}

// (two_sum, not fast_two_sum, renormalises: after cancellation the error
// term can exceed the sum)
__device__ __forceinline__ df df_add(df a, df b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  float h, l;
  two_sum(s, e, h, l);
  return df{h, l};
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.h, -a.l}; }

// A double split exactly into hi = fl32(x) and lo = fl32(x - hi): x - hi is
// exact in FP64, so |x - (hi + lo)| <= 2^-48 |x| for x in the FP32 normal
// range.
__device__ __forceinline__ df df_from(double x) {
  const float h = __double2float_rn(x);
  return df{h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double df_to(df a) { return (double)a.h + (double)a.l; }

// Compensated accumulation of sum_i x_i y_i: s the running FP32 sum, c the
// FP32 sum of the rounding errors of the products and of the additions.
struct DfAcc {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(df x, df y) {
    const float p = __fmul_rn(x.h, y.h);
    float pe = __fmaf_rn(x.h, y.h, -p);
    pe = __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, pe));
    float s2, se;
    two_sum(s, p, s2, se);
    s = s2;
    c = __fadd_rn(c, __fadd_rn(pe, se));
  }
  __device__ __forceinline__ df get() const {
    float h, l;
    two_sum(s, c, h, l);
    return df{h, l};
  }
};

// The Lagrange bases on the GLL nodes in double-float arithmetic, values
// only, in the symmetric form of lagrange_sym_values (s = r^2, pairs
// f_m = s - z_m^2): the table's double-float forms of z, w and z^2.
template <int N>
__device__ __forceinline__ void lagrange_sym_values_df(const BasisTab& B, df r, df* phi) {
  constexpr int K = N / 2;
  constexpr bool kOdd = (N % 2) != 0;
  const df s = df_mul(r, r);
  df f[K];
#pragma unroll
  for (int m = 0; m < K; ++m) f[m] = df_add(s, df{-B.z2h[m], -B.z2l[m]});
  df L[K];
  if constexpr (K == 1) {
    L[0] = df{1.f, 0.f};
  } else if constexpr (K == 2) {
    L[0] = f[1];
    L[1] = f[0];
  } else {
    df pre[K], suf[K];
    pre[1] = f[0];
#pragma unroll
    for (int i = 2; i < K; ++i) pre[i] = df_mul(pre[i - 1], f[i - 1]);
    suf[K - 2] = f[K - 1];
#pragma unroll
    for (int i = K - 3; i >= 0; --i) suf[i] = df_mul(suf[i + 1], f[i + 1]);
    L[0] = suf[0];
    L[K - 1] = pre[K - 1];
#pragma unroll
    for (int i = 1; i < K - 1; ++i) L[i] = df_mul(pre[i], suf[i]);
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const df w{B.wf[i], B.wl[i]}, z{B.zf[i], B.zl[i]};
    df Q = (K == 1) ? w : df_mul(w, L[i]);
    if constexpr (kOdd) Q = df_mul(Q, r);
    phi[i] = df_mul(Q, df_add(r, z));
    const df pm = df_mul(Q, df_add(r, df_neg(z)));
    phi[N - 1 - i] = kOdd ? pm : df_neg(pm);
  }
  if constexpr (kOdd) {
    const df w{B.wf[K], B.wl[K]};
    phi[K] = df_mul(w, (K == 1) ? f[0] : df_mul(L[0], f[0]));
  }
}

}  // namespace fp
