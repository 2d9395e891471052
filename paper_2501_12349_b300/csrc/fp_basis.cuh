// Device arithmetic of the element map (Sec. 2, Eqs. x_tensor, u_tensor,
// jacobian): Lagrange bases on the GLL nodes and sum-factorised contractions
// of an element's nodal data.  Templated on the element size N, the reference
// dimension DR, the physical dimension D and the arithmetic type T (double
// for the FP64 path, float for the FP32 phase of the mixed path).
#pragma once
#include "fp_common.cuh"

namespace fp {

template <typename T>
__device__ __forceinline__ T ldg(const T* p) {
  return __ldg(p);
}

template <typename T>
struct TabOf;
template <>
struct TabOf<double> {
  static __device__ __forceinline__ const double* z(const BasisTab& b) { return b.z; }
  static __device__ __forceinline__ const double* w(const BasisTab& b) { return b.w; }
  static __device__ __forceinline__ const double* z2(const BasisTab& b) { return b.z2; }
  static __device__ __forceinline__ const double* w2(const BasisTab& b) { return b.w2; }
};
template <>
struct TabOf<float> {
  static __device__ __forceinline__ const float* z(const BasisTab& b) { return b.zf; }
  static __device__ __forceinline__ const float* w(const BasisTab& b) { return b.wf; }
  static __device__ __forceinline__ const float* z2(const BasisTab& b) { return b.z2f; }
  static __device__ __forceinline__ const float* w2(const BasisTab& b) { return b.w2f; }
};

// phi_i(r) = w_i prod_{m != i} (r - z_m) and its derivative, from prefix and
// suffix products of (r - z_m) carried with their derivatives.
template <int N, typename T>
__device__ __forceinline__ void lagrange(const T* z, const T* w, T r, T* phi, T* dphi) {
  T d[N], p[N], dp[N];
#pragma unroll
  for (int m = 0; m < N; ++m) d[m] = r - z[m];
  p[0] = T(1);
  dp[0] = T(0);
#pragma unroll
  for (int i = 1; i < N; ++i) {
    dp[i] = fma(dp[i - 1], d[i - 1], p[i - 1]);
    p[i] = p[i - 1] * d[i - 1];
  }
  T s = T(1), ds = T(0);
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    phi[i] = w[i] * (p[i] * s);
    dphi[i] = w[i] * fma(dp[i], s, p[i] * ds);
    ds = fma(ds, d[i], s);
    s = s * d[i];
  }
}

// The same bases by the symmetry of the GLL nodes (z_{N-1-i} = -z_i): with
// s = r^2 and f_m = s - z_m^2 for the K = N/2 pairs, (r - z_i)(r + z_i) = f_i,
// so the node polynomial is [r] prod_m f_m ([r] only for odd N) and
//   phi_i = Q_i (r + z_i),  phi_{N-1-i} = sigma Q_i (r - z_i),
//   Q_i = w_i [r] L_i,  L_i = prod_{m != i} f_m  (i < K),
// with sigma = (-1)^(N-1) the sign relating mirrored weights; for odd N the
// middle basis is phi_K = w_K prod_m f_m.  Derivatives by the product rule
// (df_m/dr = 2r, dL_i/ds = sum over m != i of the products without f_i, f_m).
// Every factor is a difference of nearby exact quantities, as in the product
// form, and at a node r = z_j (s = z_j^2 rounded as in the table, f_j = 0)
// every basis but phi_j vanishes exactly.  At N = 5: 26 operations for
// values and derivatives against 46 for the product form.
template <int N, typename T>
__device__ __forceinline__ void sym_leave_one_out(const T (&f)[N / 2], T (&L)[N / 2], T (&dL)[N / 2]) {
  constexpr int K = N / 2;
  if constexpr (K == 1) {
    L[0] = T(1);
    dL[0] = T(0);
  } else if constexpr (K == 2) {
    L[0] = f[1];
    L[1] = f[0];
    dL[0] = dL[1] = T(1);
  } else {
    T pre[K], dpre[K], suf[K], dsuf[K];
    pre[1] = f[0];
    dpre[1] = T(1);
#pragma unroll
    for (int i = 2; i < K; ++i) {
      dpre[i] = fma(dpre[i - 1], f[i - 1], pre[i - 1]);
      pre[i] = pre[i - 1] * f[i - 1];
    }
    suf[K - 2] = f[K - 1];
    dsuf[K - 2] = T(1);
#pragma unroll
    for (int i = K - 3; i >= 0; --i) {
      dsuf[i] = fma(dsuf[i + 1], f[i + 1], suf[i + 1]);
      suf[i] = suf[i + 1] * f[i + 1];
    }
    L[0] = suf[0];
    dL[0] = dsuf[0];
    L[K - 1] = pre[K - 1];
    dL[K - 1] = dpre[K - 1];
#pragma unroll
    for (int i = 1; i < K - 1; ++i) {
      L[i] = pre[i] * suf[i];
      dL[i] = fma(dpre[i], suf[i], pre[i] * dsuf[i]);
    }
  }
}

template <int N, typename T>
__device__ __forceinline__ void lagrange_sym(const BasisTab& B, T r, T* phi, T* dphi) {
  constexpr int K = N / 2;
  constexpr bool kOdd = (N % 2) != 0;
  const T* z = TabOf<T>::z(B);
  const T* w = TabOf<T>::w(B);
  const T* z2 = TabOf<T>::z2(B);
  const T* w2 = TabOf<T>::w2(B);
  const T s = r * r;
  T f[K], L[K], dL[K];
#pragma unroll
  for (int m = 0; m < K; ++m) f[m] = s - z2[m];
  sym_leave_one_out<N, T>(f, L, dL);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    T Q, dQ;
    if constexpr (kOdd) {
      const T wl = (K == 1) ? w[i] : w[i] * L[i];
      Q = wl * r;
      // dQ = w_i (L_i + 2 s dL_i)
      if constexpr (K == 1) dQ = w[i];
      else if constexpr (K == 2) dQ = fma(w2[i], s, wl);
      else dQ = w[i] * fma(s + s, dL[i], L[i]);
    } else {
      Q = (K == 1) ? w[i] : w[i] * L[i];
      // dQ = 2 w_i r dL_i
      if constexpr (K == 1) dQ = T(0);
      else if constexpr (K == 2) dQ = w2[i] * r;
      else dQ = (w2[i] * r) * dL[i];
    }
    const T rp = r + z[i], rm = r - z[i];
    phi[i] = Q * rp;
    if constexpr (kOdd) {
      phi[N - 1 - i] = Q * rm;
    } else {
      phi[N - 1 - i] = (-Q) * rm;
    }
    if constexpr (!kOdd && K == 1) {
      dphi[i] = Q;
      dphi[N - 1 - i] = -Q;
    } else if constexpr (kOdd) {
      dphi[i] = fma(dQ, rp, Q);
      dphi[N - 1 - i] = fma(dQ, rm, Q);
    } else {
      dphi[i] = fma(dQ, rp, Q);
      dphi[N - 1 - i] = fma(-dQ, rm, -Q);
    }
  }
  if constexpr (kOdd) {
    // phi_K = w_K prod_m f_m, dphi_K = 2 w_K r sum_m L_m
    const T P = (K == 1) ? f[0] : L[0] * f[0];
    phi[K] = w[K] * P;
    T sL = L[0];
#pragma unroll
    for (int m = 1; m < K; ++m) sL += L[m];
    dphi[K] = (K == 1) ? w2[K] * r : (w2[K] * r) * sL;
  }
}

// Values only, in the symmetric form (at N = 5: 17 operations against 23).
template <int N, typename T>
__device__ __forceinline__ void lagrange_sym_values(const BasisTab& B, T r, T* phi) {
  constexpr int K = N / 2;
  constexpr bool kOdd = (N % 2) != 0;
  const T* z = TabOf<T>::z(B);
  const T* w = TabOf<T>::w(B);
  const T* z2 = TabOf<T>::z2(B);
  const T s = r * r;
  T f[K], L[K], dL[K];
#pragma unroll
  for (int m = 0; m < K; ++m) f[m] = s - z2[m];
  sym_leave_one_out<N, T>(f, L, dL);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    T Q = (K == 1) ? w[i] : w[i] * L[i];
    if constexpr (kOdd) Q = Q * r;
    phi[i] = Q * (r + z[i]);
    if constexpr (kOdd) {
      phi[N - 1 - i] = Q * (r - z[i]);
    } else {
      phi[N - 1 - i] = (-Q) * (r - z[i]);
    }
  }
  if constexpr (kOdd) phi[K] = w[K] * ((K == 1) ? f[0] : L[0] * f[0]);
}

// One row of element data (N r-nodes from xe) contracted with the r-basis:
// a += sum_i v_i phi_i and, if WANT_G, b += sum_i v_i phi_i', FMAs in
// ascending i.  With kVec (FP32 rows padded to a multiple of 4 floats, so
// xe is 16-byte aligned) the row first loads as float4s, then a float2 or
// float for the rest: one or two load requests where N scalar loads would
// be N; otherwise each value loads beside its FMAs.
template <int N, bool kVec, bool WANT_G, typename T>
__device__ __forceinline__ void row_dot(const T* __restrict__ xe, const T (&ph)[N], const T (&dph)[N], T& a,
                                        T& b) {
  if constexpr (kVec) {
    static_assert(sizeof(T) == 4, "vector rows hold floats");
    constexpr int kQ = (N % 4 == 3) ? (N + 3) / 4 : N / 4;  // float4s (a 3-rest takes one too)
    T v[N];
    const float4* q = reinterpret_cast<const float4*>(xe);
#pragma unroll
    for (int k = 0; k < kQ; ++k) {
      const float4 f = __ldg(q + k);
      const float t4[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (4 * k + t < N) v[4 * k + t] = t4[t];
    }
    if constexpr (N % 4 == 2) {
      const float2 f = __ldg(reinterpret_cast<const float2*>(xe) + 2 * kQ);
      v[N - 2] = f.x;
      v[N - 1] = f.y;
    } else if constexpr (N % 4 == 1) {
      v[N - 1] = __ldg(reinterpret_cast<const float*>(xe) + N - 1);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
      a = fma(v[i], ph[i], a);
      if (WANT_G) b = fma(v[i], dph[i], b);
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const T v = ldg(xe + i);
      a = fma(v, ph[i], a);
      if (WANT_G) b = fma(v, dph[i], b);
    }
  }
}

// x_c = sum u_ijk phi_i(r) phi_j(s) phi_k(t) for the D components of element
// data X (component c at X + c*cs, rows of N r-nodes at pitch P) and, if
// WANT_G, G[c*DR + j] = dx_c/dr_j.  Contraction order: r (the contiguous
// index) first, then s, then t, so a component costs N^2 (2N + 3) + 4N FMA
// with G (N^3 + N^2 + N without).
template <int N, int DR, int D, bool WANT_G, typename T, int P = N>
__device__ __forceinline__ void map_eval(const T* __restrict__ X, int64_t cs, const T (&ph)[DR][N],
                                         const T (&dph)[DR][N], T* x, T* G) {
  // vector rows for FP32 lines, and quads up to N = 5 (beyond it the
  // unrolled contraction's rows, loaded ahead, spill)
  constexpr bool kVec = sizeof(T) == 4 && P % 4 == 0 && (DR == 1 || (DR == 2 && N <= 5));
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const T* xe = X + c * cs;
    T xv = T(0), g0 = T(0), g1 = T(0), g2 = T(0);
    if constexpr (DR == 3) {
#pragma unroll
      for (int k = 0; k < N; ++k) {
        T ak = T(0), bk = T(0), ck = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          T a = T(0), b = T(0);
          row_dot<N, false, WANT_G, T>(xe + (k * N + j) * P, ph[0], dph[0], a, b);
          ak = fma(a, ph[1][j], ak);
          if (WANT_G) {
            bk = fma(b, ph[1][j], bk);
            ck = fma(a, dph[1][j], ck);
          }
        }
        xv = fma(ak, ph[2][k], xv);
        if (WANT_G) {
          g0 = fma(bk, ph[2][k], g0);
          g1 = fma(ck, ph[2][k], g1);
          g2 = fma(ak, dph[2][k], g2);
        }
      }
    } else if constexpr (DR == 2) {
#pragma unroll
      for (int j = 0; j < N; ++j) {
        T a = T(0), b = T(0);
        row_dot<N, kVec, WANT_G, T>(xe + j * P, ph[0], dph[0], a, b);
        xv = fma(a, ph[1][j], xv);
        if (WANT_G) {
          g0 = fma(b, ph[1][j], g0);
          g1 = fma(a, dph[1][j], g1);
        }
      }
    } else {  // line elements
      row_dot<N, kVec, WANT_G, T>(xe, ph[0], dph[0], xv, g0);
    }
    x[c] = xv;
    if (WANT_G) {
      G[c * DR + 0] = g0;
      if constexpr (DR >= 2) G[c * DR + 1] = g1;
      if constexpr (DR == 3) G[c * DR + 2] = g2;
    }
  }
}

// Per-thread slots in shared memory, column-major ([slot][blockDim.x]) so
// that a warp reading slot k touches consecutive words.
template <typename T>
struct Slots {
  T* base;
  int stride;
  __device__ __forceinline__ T& operator()(int k) const { return base[k * stride + threadIdx.x]; }
};

// As map_eval for hexes (DR == 3, rows at pitch P), with the outer t-loop
// rolled: the t-basis values come from shared-memory slots pt(k) = phi_k(t),
// dpt(k) = phi_k'(t), so the contraction inlines as one N^2 body instead of
// N^3 (a much smaller kernel: the FP64 find kernels were instruction-fetch
// bound unrolled).  FP32 rows at a pitch that is a multiple of 4 load as
// vectors.
template <int N, int D, bool WANT_G, typename T, int P = N>
__device__ __forceinline__ void map_eval_rolled(const T* __restrict__ X, int64_t cs,
                                                const T (&ph)[3][N], const T (&dph)[3][N],
                                                const Slots<T>& pt, const Slots<T>& dpt, T* x, T* G) {
  constexpr bool kVec = sizeof(T) == 4 && P % 4 == 0;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const T* xe = X + c * cs;
    T xv = T(0), g0 = T(0), g1 = T(0), g2 = T(0);
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
      T ak = T(0), bk = T(0), ck = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        T a = T(0), b = T(0);
        row_dot<N, kVec, WANT_G, T>(xe + (k * N + j) * P, ph[0], dph[0], a, b);
        ak = fma(a, ph[1][j], ak);
        if (WANT_G) {
          bk = fma(b, ph[1][j], bk);
          ck = fma(a, dph[1][j], ck);
        }
      }
      const T tk = pt(k);
      xv = fma(ak, tk, xv);
      if (WANT_G) {
        g0 = fma(bk, tk, g0);
        g1 = fma(ck, tk, g1);
        g2 = fma(ak, dpt(k), g2);
      }
    }
    x[c] = xv;
    if (WANT_G) {
      G[c * 3 + 0] = g0;
      G[c * 3 + 1] = g1;
      G[c * 3 + 2] = g2;
    }
  }
}

// Order tests from the bit patterns, on the integer pipe (the FP64 one is
// the find kernels' bound) and exact for every value: for IEEE values of one sign the integer order of the bit
// patterns is the value order, and a NaN fails every test, as it fails the
// floating-point comparison.
template <typename T>
struct FBits;
template <>
struct FBits<double> {
  using I = long long;
  static constexpr I kAbs = 0x7fffffffffffffffLL, kInf = 0x7ff0000000000000LL;
  static __device__ __forceinline__ I of(double v) { return __double_as_longlong(v); }
  static __device__ __forceinline__ double from(I i) { return __longlong_as_double(i); }
};
template <>
struct FBits<float> {
  using I = int;
  static constexpr I kAbs = 0x7fffffff, kInf = 0x7f800000;
  static __device__ __forceinline__ I of(float v) { return __float_as_int(v); }
  static __device__ __forceinline__ float from(I i) { return __int_as_float(i); }
};
// (For float the plain comparisons are kept: the FP32 pipe is not the bound
// of the FP32 phase, and the integer forms only add ALU instructions.)
// v > 0
template <typename T>
__device__ __forceinline__ bool is_pos(T v) {
  if constexpr (std::is_same_v<T, float>) return v > 0.0f;
  const auto i = FBits<T>::of(v);
  return i > 0 && i <= FBits<T>::kInf;
}
// v < 0
template <typename T>
__device__ __forceinline__ bool is_neg(T v) {
  if constexpr (std::is_same_v<T, float>) return v < 0.0f;
  const auto i = FBits<T>::of(v);
  const auto a = i & FBits<T>::kAbs;
  return i < 0 && a != 0 && a <= FBits<T>::kInf;
}
// v > c for c >= +0 (c not NaN)
template <typename T>
__device__ __forceinline__ bool above_nonneg(T v, T c) {
  if constexpr (std::is_same_v<T, float>) return v > c;
  const auto i = FBits<T>::of(v);
  return i > FBits<T>::of(c) && i <= FBits<T>::kInf;
}
// a < b for a >= +0 and b >= +0, either of them possibly a NaN
template <typename T>
__device__ __forceinline__ bool below_nonneg(T a, T b) {
  if constexpr (std::is_same_v<T, float>) return a < b;
  const auto ia = FBits<T>::of(a), ib = FBits<T>::of(b);
  return ia >= 0 && ia < ib && ib <= FBits<T>::kInf;
}

// Solves A s = b for a symmetric DR x DR matrix by cofactors when A is
// positive definite (all leading principal minors > 0, the same sign test as
// the pivots of a Cholesky factorisation); returns false otherwise.
template <int DR, typename T>
__device__ __forceinline__ bool spd_solve(const T (&A)[DR][DR], const T (&b)[DR], T (&s)[DR]) {
  if constexpr (DR == 1) {
    if (!(A[0][0] > T(0))) return false;
    s[0] = b[0] / A[0][0];
    return true;
  } else if constexpr (DR == 2) {
    const T det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    if (!is_pos(A[0][0]) || !is_pos(det)) return false;
    const T inv = T(1) / det;
    s[0] = (A[1][1] * b[0] - A[0][1] * b[1]) * inv;
    s[1] = (A[0][0] * b[1] - A[1][0] * b[0]) * inv;
    return true;
  } else {
    const T m2 = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    const T c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    const T c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    const T c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    const T det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
    if (!is_pos(A[0][0]) || !is_pos(m2) || !is_pos(det)) return false;
    const T c11 = A[0][0] * A[2][2] - A[0][2] * A[2][0];
    const T c12 = A[0][2] * A[1][0] - A[0][0] * A[1][2];
    const T c22 = m2;
    const T inv = T(1) / det;
    // symmetric adjugate
    s[0] = (c00 * b[0] + c01 * b[1] + c02 * b[2]) * inv;
    s[1] = (c01 * b[0] + c11 * b[1] + c12 * b[2]) * inv;
    s[2] = (c02 * b[0] + c12 * b[1] + c22 * b[2]) * inv;
    return true;
  }
}

}  // namespace fp
