// Interpolate (Sec. 3.3, Eq. u_tensor): u(r*) in element e* for each found
// point, one thread per point, the contraction sum-factorised (N^3 + N^2 + N
// FMA per component for a hex).  FP64-pipe bound like find.
//
// The field's nodes per direction, N~, may differ from the mesh's N (Sec. 2,
// after Eq. u_tensor: a solution is often represented at another order than
// the coordinates); the kernel is the same with the GLL basis of N~ points.
#include <mutex>

#include "fp_basis.cuh"
#include "fp_common.cuh"

namespace fp {

constexpr int kEvalThreads = 128;

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

}  // namespace fp

namespace {

// GLL basis tables of every supported N, built once per process.
const fp::BasisTab* basis_of(int N) {
  static fp::BasisTab tabs[FP_MAX_N + 1];
  static std::once_flag once;
  std::call_once(once, [] {
    for (int k = 2; k <= FP_MAX_N; ++k) fp::host_basis_tab(k, &tabs[k]);
  });
  return (N >= 2 && N <= FP_MAX_N) ? &tabs[N] : nullptr;
}

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
  const int rc = dispatch_shape(Nf, m->d, m->dr, [&](auto Nc, auto Dc, auto DRc) -> int {
    constexpr int N = decltype(Nc)::value, DR = decltype(DRc)::value;
    (void)Dc;
    const int blocks = grid_for(n, kEvalThreads, 148 * 64);
    k_eval_f64<N, DR><<<blocks, kEvalThreads, 0, st>>>(*B, code, elem, r, n, field, nc, m->NE, out,
                                                        m->status);
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ELAUNCH;
  });
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
