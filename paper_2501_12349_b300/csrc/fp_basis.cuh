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
};
template <>
struct TabOf<float> {
  static __device__ __forceinline__ const float* z(const BasisTab& b) { return b.zf; }
  static __device__ __forceinline__ const float* w(const BasisTab& b) { return b.wf; }
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

// Values only: phi_i(r) = w_i (prefix product)_i (suffix product)_i.
template <int N, typename T>
__device__ __forceinline__ void lagrange_values(const T* z, const T* w, T r, T* phi) {
  T d[N], p[N];
#pragma unroll
  for (int m = 0; m < N; ++m) d[m] = r - z[m];
  p[0] = T(1);
#pragma unroll
  for (int i = 1; i < N; ++i) p[i] = p[i - 1] * d[i - 1];
  T s = T(1);
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    phi[i] = w[i] * (p[i] * s);
    s = s * d[i];
  }
}

// Values, first and second derivatives.
template <int N, typename T>
__device__ __forceinline__ void lagrange2(const T* z, const T* w, T r, T* phi, T* dphi, T* d2phi) {
  T d[N], p[N], dp[N], d2p[N];
#pragma unroll
  for (int m = 0; m < N; ++m) d[m] = r - z[m];
  p[0] = T(1);
  dp[0] = T(0);
  d2p[0] = T(0);
#pragma unroll
  for (int i = 1; i < N; ++i) {
    d2p[i] = fma(d2p[i - 1], d[i - 1], T(2) * dp[i - 1]);
    dp[i] = fma(dp[i - 1], d[i - 1], p[i - 1]);
    p[i] = p[i - 1] * d[i - 1];
  }
  T s = T(1), ds = T(0), d2s = T(0);
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    phi[i] = w[i] * (p[i] * s);
    dphi[i] = w[i] * fma(dp[i], s, p[i] * ds);
    d2phi[i] = w[i] * fma(d2p[i], s, fma(T(2) * dp[i], ds, p[i] * d2s));
    d2s = fma(d2s, d[i], T(2) * ds);
    ds = fma(ds, d[i], s);
    s = s * d[i];
  }
}

// x_c = sum u_ijk phi_i(r) phi_j(s) phi_k(t) for the D components of element
// data X (component c at X + c*cs) and, if WANT_G, G[c*DR + j] = dx_c/dr_j.
// Contraction order: r (the contiguous index) first, then s, then t, so a
// component costs N^2 (2N + 3) + 4N FMA with G (N^3 + N^2 + N without).
template <int N, int DR, int D, bool WANT_G, typename T>
__device__ __forceinline__ void map_eval(const T* __restrict__ X, int64_t cs, const T (&ph)[DR][N],
                                         const T (&dph)[DR][N], T* x, T* G) {
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
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const T v = ldg(xe + (k * N + j) * N + i);
            a = fma(v, ph[0][i], a);
            if (WANT_G) b = fma(v, dph[0][i], b);
          }
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
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const T v = ldg(xe + j * N + i);
          a = fma(v, ph[0][i], a);
          if (WANT_G) b = fma(v, dph[0][i], b);
        }
        xv = fma(a, ph[1][j], xv);
        if (WANT_G) {
          g0 = fma(b, ph[1][j], g0);
          g1 = fma(a, dph[1][j], g1);
        }
      }
    } else {  // line elements
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const T v = ldg(xe + i);
        xv = fma(v, ph[0][i], xv);
        if (WANT_G) g0 = fma(v, dph[0][i], g0);
      }
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

// As map_eval for hexes (DR == 3), with the outer t-loop rolled: the t-basis
// values come from shared-memory slots pt(k) = phi_k(t), dpt(k) = phi_k'(t),
// so the contraction inlines as one N^2 body instead of N^3 (a much smaller
// kernel: the FP64 find kernels were instruction-fetch bound unrolled).
template <int N, int D, bool WANT_G, typename T>
__device__ __forceinline__ void map_eval_rolled(const T* __restrict__ X, int64_t cs,
                                                const T (&ph)[3][N], const T (&dph)[3][N],
                                                const Slots<T>& pt, const Slots<T>& dpt, T* x, T* G) {
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
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const T v = ldg(xe + (k * N + j) * N + i);
          a = fma(v, ph[0][i], a);
          if (WANT_G) b = fma(v, dph[0][i], b);
        }
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
    if (!(A[0][0] > T(0)) || !(det > T(0))) return false;
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
    if (!(A[0][0] > T(0)) || !(m2 > T(0)) || !(det > T(0))) return false;
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
