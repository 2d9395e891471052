// The double-float interpolation (FP_MIXED) shared by fp_eval, the batch
// plans and the server: the field split into (hi, lo) pairs after an exact
// power-of-two scaling per component, and the sum-factorised contraction of
// Eq. u_tensor (Sec. 3.3) as compensated dot products in double-float
// arithmetic on the FP32 pipe (df64.cuh).  Error: about 2^-48 relative per
// split and operation, at most about N u^2 of the |terms| per compensated
// N-term sum (u = 2^-24), so within about 1e-13 of the element's nodal scale
// at N <= 8.  The points are visited in an element-grouped order (the lanes
// of a warp then read one element's values; in the given order each lane's
// gather is a cache line of its own, and that, not arithmetic, bounds it).
#pragma once
#include "df64.cuh"
#include "find_common.cuh"

namespace fp {

// One component of one field to split: per values at src, pairs to dst, the
// component's largest biased exponent to *exp (caller-zeroed).
struct SplitJob {
  const double* src;
  int64_t per;
  float2* dst;
  int* exp;
};

// The jobs of a call: the table tab[blockIdx.y], or, with tab == nullptr, the
// nc components of one field (component c at field + c per, pairs at
// out + c per, exponent at exp + c).
struct SplitJobs {
  const SplitJob* tab;
  const double* field;
  int64_t per;
  float2* out;
  int* exp;
  __device__ __forceinline__ SplitJob get(int j) const {
    if (tab) return tab[j];
    return SplitJob{field + (int64_t)j * per, per, out + (int64_t)j * per, exp + j};
  }
};

// 2^(1023 - e) for a biased exponent e in [1, 2046], else 1 (an all-zero
// component, or one holding an infinity or NaN, which propagates as in FP64).
__device__ __forceinline__ double df_unscale_of(int e) {
  return (e >= 1 && e <= 2046) ? __longlong_as_double((long long)(2046 - e) << 52) : 1.0;
}
__device__ __forceinline__ double df_scale_of(int e) {
  return (e >= 1 && e <= 2046) ? __longlong_as_double((long long)e << 52) : 1.0;
}

template <int kUnused = 0>
__global__ void k_split_exp(SplitJobs jobs) {
  const SplitJob jb = jobs.get(blockIdx.y);
  int m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < jb.per; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (int)((__double_as_longlong(jb.src[i]) >> 52) & 0x7ff));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(jb.exp, m);
}

template <int kUnused = 0>
__global__ void k_split(SplitJobs jobs) {
  const SplitJob jb = jobs.get(blockIdx.y);
  const double s = df_unscale_of(*jb.exp);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < jb.per; i += (int64_t)gridDim.x * blockDim.x) {
    const df v = df_from(jb.src[i] * s);  // exact scaling by a power of two
    jb.dst[i] = make_float2(v.h, v.l);
  }
}

// Launches the two passes over njobs jobs of at most max_per values (the
// exponents must be zero beforehand).
inline int split_fields(const SplitJobs& jobs, int njobs, int64_t max_per, cudaStream_t st) {
  if (njobs <= 0 || max_per <= 0) return FP_OK;
  const dim3 g((unsigned)grid_for(max_per, 256, 148 * 8), (unsigned)njobs);
  k_split_exp<<<g, 256, 0, st>>>(jobs);
  k_split<<<g, 256, 0, st>>>(jobs);
  return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ELAUNCH;
}

// sum_ijk x_ijk phi_i phi_j phi_k (and the 2D, 1D forms) of one element's
// split values, each sum-factorised stage a compensated dot product.
template <int N, int DR>
__device__ __forceinline__ df contract_df(const float2* __restrict__ x, const df (&ph)[DR][N]) {
  auto ld = [&](int q) {
    const float2 v = __ldg(x + q);
    return df{v.x, v.y};
  };
  DfAcc acc;
  if constexpr (DR == 3) {
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
      df pk = ph[2][0];
#pragma unroll
      for (int q = 1; q < N; ++q)
        if (q == k) pk = ph[2][q];
      DfAcc bk;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        DfAcc a;
#pragma unroll
        for (int i = 0; i < N; ++i) a.add(ld((k * N + j) * N + i), ph[0][i]);
        bk.add(a.get(), ph[1][j]);
      }
      acc.add(bk.get(), pk);
    }
  } else if constexpr (DR == 2) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      DfAcc a;
#pragma unroll
      for (int i = 0; i < N; ++i) a.add(ld(j * N + i), ph[0][i]);
      acc.add(a.get(), ph[1][j]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) acc.add(ld(i), ph[0][i]);
  }
  return acc.get();
}

// Interpolation over a table of batch items (one element shape) in double
// float: thread t takes the global point order[t] (or t), the item holding
// it by binary search over the items' starts; an item's split field and
// exponents are fs and fexp ([nc][NE][N^dr] pairs, [nc]).
template <int N, int DR>
__global__ void __launch_bounds__(128)
    k_eval_items_df(const BatchItem* __restrict__ items, int nitems, int64_t total, const int* __restrict__ order,
                    const BasisTab B) {
  constexpr int NN = ipow(N, DR);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = order ? (int64_t)__ldg(order + t) : t;
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].start <= g) lo = mid;
      else hi = mid - 1;
    }
    const BatchItem& it = items[lo];
    if (it.fs == nullptr || it.nc <= 0) continue;
    const int64_t p = g - it.start;
    const int c0 = it.code[p], e = it.elem[p];
    const int64_t NE = it.m.NE;
    if (c0 == FP_NOT_FOUND || e < 0 || e >= NE) {
      if (c0 != FP_NOT_FOUND) record_status(it.m.status, FP_DEV_BAD_ELEM);
      for (int c = 0; c < it.nc; ++c) it.out[(int64_t)c * it.ld + p] = 0.0;
      continue;
    }
    df ph[DR][N];
#pragma unroll
    for (int j = 0; j < DR; ++j) lagrange_sym_values_df<N>(B, df_from(it.r[p * DR + j]), ph[j]);
    for (int c = 0; c < it.nc; ++c) {
      const df v = contract_df<N, DR>(it.fs + (c * NE + e) * NN, ph);
      it.out[(int64_t)c * it.ld + p] = df_to(v) * df_scale_of(__ldg(it.fexp + c));
    }
  }
}

}  // namespace fp
