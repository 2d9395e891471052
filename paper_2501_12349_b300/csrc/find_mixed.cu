// Mixed-precision find (FP_MIXED): the kernels over one mesh and over a
// batch class, and their launches; the lane loop is in find_mixed.cuh.
#include "find_mixed.cuh"

namespace fp {
namespace {

template <int N, int D, int DR>
__global__ void __launch_bounds__(kFindThreads, mixed_ctas(N, D, DR))
    k_find_mixed(const __grid_constant__ DevMesh m, const BasisTab B, const double* __restrict__ pts,
                 const int* __restrict__ pidx, int64_t n, int* __restrict__ code, int* __restrict__ elem,
                 double* __restrict__ rout, double* __restrict__ dist2, int* __restrict__ queue,
                 int* __restrict__ qcount, unsigned long long* stats) {
  const SingleWork<D, DR> w{&m, pts, pidx, n, code, elem, rout, dist2, 5};
  __shared__ MixedShared<N, D, DR> sh;
  find_mixed_loop<N, D, DR>(w, B, queue, qcount, stats, sh);
}

template <int N, int D, int DR>
__global__ void __launch_bounds__(kFindThreads, mixed_ctas(N, D, DR))
    k_find_mixed_batch(const BatchItem* __restrict__ items, int nitems, int64_t total,
                       const int* __restrict__ gidx, const BasisTab B, int* __restrict__ queue,
                       int* __restrict__ qcount, int clog2, unsigned long long* stats) {
  const BatchWork<D, DR> w{items, nitems, gidx, total, clog2};
  __shared__ MixedShared<N, D, DR> sh;
  find_mixed_loop<N, D, DR>(w, B, queue, qcount, stats, sh);
}

}  // namespace

}  // namespace fp

namespace fp {

// The two launches of the mixed path with a caller-provided queue
// (capacity >= n entries) and zeroed counter; allocates nothing.
int launch_mixed_with_queue(const fp_mesh_s* m, const double* pts, const int* pidx, int64_t n, int* code,
                            int* elem, double* r, double* dist2, int* queue, int* qcount,
                            unsigned long long* stats, cudaStream_t st, cudaEvent_t* mid) {
  const DevMesh v = m->view();
  return dispatch_shape(m->N, m->d, m->dr, [&](auto Nc, auto Dc, auto DRc) -> int {
    constexpr int N = decltype(Nc)::value, D = decltype(Dc)::value, DR = decltype(DRc)::value;
    k_find_mixed<N, D, DR><<<persistent_blocks(n, mixed_ctas(N, D, DR)), kFindThreads, 0, st>>>(
        v, m->basis, pts, pidx, n, code, elem, r, dist2, queue, qcount, stats);
    if (mid) *mid = timer_mark(m, st);
    if (n <= kGroupMaxPoints)
      k_find_f64_group<N, D, DR><<<persistent_blocks(n, f64_ctas(N)), kFindThreads, 0, st>>>(
          v, m->basis, pts, queue, n, qcount, code, elem, r, dist2, fallback_stats(stats));
    else
      k_find_f64<N, D, DR><<<follow_blocks(), kFollowThreads, 0, st>>>(
          v, m->basis, pts, queue, n, qcount, code, elem, r, dist2, kFollowClog2, fallback_stats(stats));
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ELAUNCH;
  });
}

}  // namespace fp

namespace fp {

// One element shape of a batch: the mixed kernel over all items, then the
// FP64 kernel over the queued global indices (queue capacity >= total).
int launch_batch_class(const BatchItem* items, int nitems, int64_t total, int N, int d, int dr,
                       const BasisTab& B, int precision, int ctas_per_sm, int clog2, const int* order,
                       int* queue, int* qcount, unsigned long long* stats, cudaStream_t st) {
  return dispatch_shape(N, d, dr, [&](auto Nc, auto Dc, auto DRc) -> int {
    constexpr int NN = decltype(Nc)::value, D = decltype(Dc)::value, DR = decltype(DRc)::value;
    if (ctas_per_sm <= 0) ctas_per_sm = precision == FP_MIXED ? mixed_ctas(NN, D, DR) : f64_ctas(NN);
    const int blocks = persistent_blocks(total, ctas_per_sm);
    if (precision == FP_MIXED) {
      k_find_mixed_batch<NN, D, DR><<<blocks, kFindThreads, 0, st>>>(items, nitems, total, order, B, queue,
                                                                     qcount, clog2, stats);
      if (total <= kGroupMaxPoints)
        k_find_f64_group_batch<NN, D, DR><<<persistent_blocks(total, f64_ctas(NN)), kFindThreads, 0, st>>>(
            items, nitems, total, queue, qcount, B, fallback_stats(stats));
      else
        k_find_f64_batch<NN, D, DR><<<follow_blocks(), kFollowThreads, 0, st>>>(
            items, nitems, total, queue, qcount, B, kFollowClog2, fallback_stats(stats));
    } else {
      k_find_f64_batch<NN, D, DR><<<blocks, kFindThreads, 0, st>>>(items, nitems, total, order, nullptr, B,
                                                                   clog2, stats);
    }
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ELAUNCH;
  });
}

int launch_batch_follow(const BatchItem* items, int nitems, int64_t total, int N, int d, int dr,
                        const BasisTab& B, int* queue, int* qcount, cudaStream_t st) {
  return dispatch_shape(N, d, dr, [&](auto Nc, auto Dc, auto DRc) -> int {
    constexpr int NN = decltype(Nc)::value, D = decltype(Dc)::value, DR = decltype(DRc)::value;
    if (total <= kGroupMaxPoints)
      k_find_f64_group_batch<NN, D, DR><<<persistent_blocks(total, f64_ctas(NN)), kFindThreads, 0, st>>>(
          items, nitems, total, queue, qcount, B, nullptr);
    else
      k_find_f64_batch<NN, D, DR><<<follow_blocks(), kFollowThreads, 0, st>>>(items, nitems, total, queue, qcount,
                                                                              B, kFollowClog2, nullptr);
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ELAUNCH;
  });
}

}  // namespace fp
