// Find (Sec. 3.2): entry points and the FP64 path's launch.  The kernels
// are in find_f64.cuh (FP64) and find_mixed.cu (FP_MIXED).
#include <math.h>

#include "find_f64.cuh"

namespace fp {

int find_f64(const fp_mesh_s* m, const double* pts, const int* pidx, int64_t n, int* code,
             int* elem, double* r, double* dist2, unsigned long long* stats, cudaStream_t st) {
  const DevMesh v = m->view();
  return dispatch_shape(m->N, m->d, m->dr, [&](auto Nc, auto Dc, auto DRc) -> int {
    constexpr int N = decltype(Nc)::value, D = decltype(Dc)::value, DR = decltype(DRc)::value;
    const int blocks = persistent_blocks(n, f64_ctas(N));
    k_find_f64<N, D, DR><<<blocks, kFindThreads, 0, st>>>(v, m->basis, pts, pidx, n, nullptr, code,
                                                          elem, r, dist2, 5, stats);
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ELAUNCH;
  });
}

}  // namespace fp

// Below this many points the counting sort of the cell order costs more
// than the locality it buys.
constexpr int64_t kOrderMinPoints = 1 << 14;

static int findpts_impl(fp_mesh m, const double* pts, int64_t n, int32_t* code, int32_t* elem,
                        double* r, double* dist2, uint64_t* stats, void* stream) {
  if (!m || n < 0 || n > INT32_MAX) return FP_EINVAL;
  if (n == 0) return FP_OK;
  if (!pts || !code || !elem || !r || !dist2) return FP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  auto* s = reinterpret_cast<unsigned long long*>(stats);
  const bool mixed = m->precision == FP_MIXED;
  const bool ordered = m->opts.point_order == FP_ORDER_CELL && n >= kOrderMinPoints;
  // scratch: the mixed path's queue (n entries + counter), then the order
  const int64_t nq = mixed ? n + 1 : 0;
  const int64_t ints = nq + (ordered ? fp::cell_order_ints(m, n) : 0);
  int* scratch = nullptr;
  if (ints > 0 && cudaMallocAsync((void**)&scratch, sizeof(int) * (size_t)ints, st) != cudaSuccess)
    return FP_ENOMEM;
  int* perm = nullptr;
  cudaEvent_t t0 = fp::timer_mark(m, st), t1 = nullptr, t2 = nullptr;
  int rc = ordered ? fp::cell_order(m, pts, n, scratch + nq, &perm, st) : FP_OK;
  if (rc == FP_OK) {
    if (mixed) {
      rc = cudaMemsetAsync(scratch + n, 0, sizeof(int), st) == cudaSuccess ? FP_OK : FP_ELAUNCH;
      t1 = fp::timer_mark(m, st);
      if (rc == FP_OK)
        rc = fp::launch_mixed_with_queue(m, pts, perm, n, code, elem, r, dist2, scratch, scratch + n, s, st,
                                         &t2);
    } else {
      t1 = fp::timer_mark(m, st);
      rc = fp::find_f64(m, pts, perm, n, code, elem, r, dist2, s, st);
    }
  }
  cudaEvent_t t3 = fp::timer_mark(m, st);
  if (ordered) fp::timer_span(m, FP_TIME_ORDER, t0, t1);
  fp::timer_span(m, FP_TIME_FIND, t1, mixed ? t2 : t3);
  if (mixed) fp::timer_span(m, FP_TIME_FOLLOW, t2, t3);
  if (scratch) cudaFreeAsync(scratch, st);
  return rc;
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

extern "C" int fp_set_point_order(fp_mesh m, int order) {
  if (!m || (order != FP_ORDER_GIVEN && order != FP_ORDER_CELL)) return FP_EINVAL;
  m->opts.point_order = order;
  return FP_OK;
}
