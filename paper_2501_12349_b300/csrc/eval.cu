// Interpolate (Sec. 3.3, Eq. u_tensor): u(r*) in element e* for each found
// point, one thread per point, the contraction sum-factorised (N^3 + N^2 + N
// FMA per component for a hex).  FP64-pipe bound like find; with the mesh in
// mixed precision, the same contraction in double-float arithmetic on the
// FP32 pipe (below).
//
// The field's nodes per direction, N~, may differ from the mesh's N (Sec. 2,
// after Eq. u_tensor: a solution is often represented at another order than
// the coordinates); the kernel is the same with the GLL basis of N~ points.
#include <mutex>

#include "eval_df.cuh"
#include "fp_basis.cuh"
#include "fp_common.cuh"

namespace fp {

constexpr int kEvalThreads = 128;
constexpr int64_t kEvalOrderMin = 16384;  // FP_MIXED: the double-float path from this many points

template <int N, int DR>
__global__ void __launch_bounds__(kEvalThreads)
    k_eval_f64(const BasisTab B, const int* __restrict__ code, const int* __restrict__ elem,
               const double* __restrict__ r, int64_t n, const double* __restrict__ field, int nc,
               int64_t NE, double* __restrict__ out, int* status) {
  constexpr int NN = ipow(N, DR);
  const int64_t cs = NE * NN;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int c0 = __ldg(code + p), e = __ldg(elem + p);
    const bool valid = c0 != FP_NOT_FOUND && e >= 0 && e < NE;
    if (c0 != FP_NOT_FOUND && !valid) record_status(status, FP_DEV_BAD_ELEM);
    if (!valid) {
      for (int c = 0; c < nc; ++c) out[(int64_t)c * n + p] = 0.0;
      continue;
    }
    double ph[DR][N], dph[DR][N] = {};  // dph unused: values only
#pragma unroll
    for (int j = 0; j < DR; ++j) lagrange_sym_values<N, double>(B, __ldg(r + p * DR + j), ph[j]);
    for (int c = 0; c < nc; ++c) {
      double v;
      map_eval<N, DR, 1, false, double>(field + c * cs + (int64_t)e * NN, 0, ph, dph, &v, nullptr);
      out[(int64_t)c * n + p] = v;
    }
  }
}

// ---- FP_MIXED: the contraction in double-float arithmetic -----------------
//
// With the mesh in mixed precision, interpolation runs on the FP32 pipe: the
// field, scaled per component by an exact power of two so that its largest
// magnitude lies in [1, 2), is split once per call into double-float pairs
// (split_fields, eval_df.cuh), the bases are evaluated in double-float arithmetic from
// the split r, and each stage of the sum-factorised contraction is a
// compensated dot product of N terms (DfAcc).  Error: the input splits and
// each double-float operation contribute about 2^-48 relative, each N-term
// compensated sum at most about N u^2 of its sum of |terms| (u = 2^-24), so
// |u_df - u| <= about 1e-13 of the element's nodal scale (at N <= 8, with the
// Lebesgue constant's growth over the three stages), against the 1e-12 of
// the interpolation tolerance; in practice a few 1e-16.

// Points in element order for the double-float contraction: counts per
// element (bucket NE for the points not found), an exclusive scan, then
// each point placed in its element's range (order within an element
// arbitrary: every point's value is computed on its own).  The lanes of a
// warp then read the same element's values, where in the given order each
// lane's gather is a cache line of its own.
__global__ void k_elem_count(const int* __restrict__ code, const int* __restrict__ elem, int64_t n, int64_t NE,
                             int* __restrict__ counts) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int e = __ldg(elem + p);
    const int64_t b = (__ldg(code + p) != FP_NOT_FOUND && e >= 0 && e < NE) ? e : NE;
    atomicAdd(counts + b, 1);
  }
}

__global__ void k_elem_scatter(const int* __restrict__ code, const int* __restrict__ elem, int64_t n, int64_t NE,
                               int* __restrict__ next, int* __restrict__ perm) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int e = __ldg(elem + p);
    const int64_t b = (__ldg(code + p) != FP_NOT_FOUND && e >= 0 && e < NE) ? e : NE;
    perm[atomicAdd(next + b, 1)] = (int)p;
  }
}

template <int N, int DR>
__global__ void __launch_bounds__(kEvalThreads)
    k_eval_df(const BasisTab B, const int* __restrict__ code, const int* __restrict__ elem,
              const double* __restrict__ r, int64_t n, const int* __restrict__ perm,
              const float2* __restrict__ fs, const int* __restrict__ emax, int nc, int64_t NE,
              double* __restrict__ out, int* status) {
  constexpr int NN = ipow(N, DR);
  const int64_t cs = NE * NN;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = perm ? (int64_t)__ldg(perm + t) : t;
    const int c0 = __ldg(code + p), e = __ldg(elem + p);
    const bool valid = c0 != FP_NOT_FOUND && e >= 0 && e < NE;
    if (c0 != FP_NOT_FOUND && !valid) record_status(status, FP_DEV_BAD_ELEM);
    if (!valid) {
      for (int c = 0; c < nc; ++c) out[(int64_t)c * n + p] = 0.0;
      continue;
    }
    df ph[DR][N];
#pragma unroll
    for (int j = 0; j < DR; ++j) lagrange_sym_values_df<N>(B, df_from(__ldg(r + p * DR + j)), ph[j]);
    for (int c = 0; c < nc; ++c) {
      const df v = contract_df<N, DR>(fs + c * cs + (int64_t)e * NN, ph);
      out[(int64_t)c * n + p] = df_to(v) * df_scale_of(__ldg(emax + c));
    }
  }
}

}  // namespace fp

namespace fp {

// GLL basis tables of every supported N, built once per process.
const BasisTab* basis_of(int N) {
  static BasisTab tabs[FP_MAX_N + 1];
  static std::once_flag once;
  std::call_once(once, [] {
    for (int k = 2; k <= FP_MAX_N; ++k) host_basis_tab(k, &tabs[k]);
  });
  return (N >= 2 && N <= FP_MAX_N) ? &tabs[N] : nullptr;
}

// The double-float contraction pays once its per-point saving outweighs the
// per-call split of the field and the element sort: quads, hexes and
// surfaces, at least kEvalOrderMin points and 8 per element on average.
bool eval_uses_df(const fp_mesh_s* m, int64_t n) {
  return m->precision == FP_MIXED && m->dr >= 2 && n >= kEvalOrderMin && n >= 8 * m->NE;
}

int df_field_prepare(const fp_mesh_s* m, const double* field, int Nf, int nc, DfField* f, cudaStream_t st) {
  *f = DfField{};
  const int64_t per = m->NE * ipow(Nf, m->dr);
  const size_t vals = (size_t)nc * (size_t)per;
  if (cudaMallocAsync(&f->scratch, vals * sizeof(float2) + (size_t)nc * sizeof(int), st) != cudaSuccess) {
    f->scratch = nullptr;
    return FP_ENOMEM;
  }
  f->fs = (float2*)f->scratch;
  f->emax = (int*)(f->fs + vals);
  f->nc = nc;
  f->Nf = Nf;
  FP_CUDA_TRY(cudaMemsetAsync(f->emax, 0, (size_t)nc * sizeof(int), st));
  return split_fields(SplitJobs{nullptr, field, per, f->fs, f->emax}, nc, per, st);
}

int df_field_eval(const fp_mesh_s* m, const DfField& f, const int32_t* code, const int32_t* elem,
                  const double* r, int64_t n, double* out, cudaStream_t st) {
  if (n == 0) return FP_OK;
  const BasisTab* B = f.Nf == m->N ? &m->basis : basis_of(f.Nf);
  if (!B) return FP_EUNSUPPORTED;
  // the element order (from kEvalOrderMin points; the order changes no value)
  const bool ordered = n >= kEvalOrderMin;
  int* ints = nullptr;
  int* perm = nullptr;
  if (ordered) {
    if (cudaMallocAsync((void**)&ints, sizeof(int) * (size_t)(2 * m->NE + 3 + n), st) != cudaSuccess)
      return FP_ENOMEM;
    int* counts = ints;                 // [NE + 1]
    int* start = counts + (m->NE + 1);  // [NE + 2]
    perm = start + (m->NE + 2);
    if (cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)(m->NE + 1), st) != cudaSuccess) {
      cudaFreeAsync(ints, st);
      return FP_ELAUNCH;
    }
    const int pb = grid_for(n, 256, 148 * 8);
    k_elem_count<<<pb, 256, 0, st>>>(code, elem, n, m->NE, counts);
    // exclusive scan over the NE + 1 buckets (start[NE + 1] = n)
    k_scan<<<1, 1024, 0, st>>>(counts, m->NE + 1, start);
    k_elem_scatter<<<pb, 256, 0, st>>>(code, elem, n, m->NE, start, perm);
  }
  const int rc = dispatch_shape(f.Nf, m->d, m->dr, [&](auto Nc, auto Dc, auto DRc) -> int {
    constexpr int N = decltype(Nc)::value, DR = decltype(DRc)::value;
    (void)Dc;
    const int blocks = grid_for(n, kEvalThreads, 148 * 64);
    k_eval_df<N, DR><<<blocks, kEvalThreads, 0, st>>>(*B, code, elem, r, n, perm, f.fs, f.emax, f.nc, m->NE, out,
                                                       m->status);
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ELAUNCH;
  });
  if (ints) cudaFreeAsync(ints, st);
  return rc;
}

void df_field_release(DfField& f, cudaStream_t st) {
  if (f.scratch) cudaFreeAsync(f.scratch, st);
  f = DfField{};
}

}  // namespace fp

namespace {

int eval_impl(fp_mesh m, const int32_t* code, const int32_t* elem, const double* r, int64_t n,
              const double* field, int Nf, int nc, double* out, void* stream) {
  using namespace fp;
  if (!m || n < 0 || nc < 0) return FP_EINVAL;
  const BasisTab* B = Nf == m->N ? &m->basis : basis_of(Nf);
  if (!B) return FP_EUNSUPPORTED;
  if (n == 0 || nc == 0) return FP_OK;
  if (!code || !elem || !r || !field || !out) return FP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t t0 = timer_mark(m, st);
  int rc = FP_OK;
  if (eval_uses_df(m, n)) {
    DfField f;
    rc = df_field_prepare(m, field, Nf, nc, &f, st);
    if (rc == FP_OK) rc = df_field_eval(m, f, code, elem, r, n, out, st);
    df_field_release(f, st);
  } else {
    rc = dispatch_shape(Nf, m->d, m->dr, [&](auto Nc, auto Dc, auto DRc) -> int {
      constexpr int N = decltype(Nc)::value, DR = decltype(DRc)::value;
      (void)Dc;
      const int blocks = grid_for(n, kEvalThreads, 148 * 64);
      k_eval_f64<N, DR><<<blocks, kEvalThreads, 0, st>>>(*B, code, elem, r, n, field, nc, m->NE, out,
                                                          m->status);
      return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ELAUNCH;
    });
  }
  timer_span(m, FP_TIME_EVAL, t0, timer_mark(m, st));
  return rc;
}

}  // namespace

extern "C" int fp_eval(fp_mesh m, const int32_t* code, const int32_t* elem, const double* r,
                       int64_t n, const double* field, int nc, double* out, void* stream) {
  if (!m) return FP_EINVAL;
  return eval_impl(m, code, elem, r, n, field, m->N, nc, out, stream);
}

extern "C" int fp_eval_order(fp_mesh m, const int32_t* code, const int32_t* elem, const double* r,
                             int64_t n, const double* field, int field_order, int nc, double* out,
                             void* stream) {
  if (!m) return FP_EINVAL;
  if (field_order < 1 || field_order > FP_MAX_N - 1) return FP_EUNSUPPORTED;
  return eval_impl(m, code, elem, r, n, field, field_order + 1, nc, out, stream);
}
