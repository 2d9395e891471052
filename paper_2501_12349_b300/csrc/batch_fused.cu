// The fused form of a batch's find: every element shape of the plan in ONE
// persistent launch.  The plan's point sequences (one per element shape,
// each in its element order) are cut into tiles; each CTA pulls tiles from
// a global counter and, per tile, dispatches on the tile's shape (N, d, dr)
// to that shape's lane loop (FP64, or the mixed path's FP32 phase with its
// FP64 refinement), compiled once per shape as a separate device function.
// Shared memory is one dynamic buffer sized for the largest shape.  The
// kernel's register budget is set by the costliest shape, so every shape
// runs at that occupancy; batch.cu times this form against one persistent
// launch per shape and keeps the faster (fp_batch_set_fused).
#include "find_mixed.cuh"

namespace fp {

namespace {

// Shape index of (N, d, dr): N in 2..FP_MAX_N, (d, dr) one of the five.
__host__ __device__ constexpr int shape_index(int N, int d, int dr) {
  return (N - 2) * 5 + (d == 2 && dr == 2 ? 0 : d == 3 && dr == 3 ? 1 : d == 3 && dr == 2 ? 2 : d == 2 ? 3 : 4);
}

template <int N, int D, int DR, bool kMixed>
__device__ __noinline__ void fused_tile(const FusedClass& c, int64_t base, int64_t n, int clog2,
                                        unsigned char* smem) {
  const TileWork<D, DR> w{{c.items, c.nitems, c.order, n, clog2}, base};
  if constexpr (kMixed)
    find_mixed_loop<N, D, DR>(w, c.B, c.queue, c.qcount, nullptr, *reinterpret_cast<MixedShared<N, D, DR>*>(smem));
  else
    find_f64_loop<N, D, DR>(w, c.B, nullptr, *reinterpret_cast<F64Shared<N, D, DR>*>(smem));
}

#define FP_FUSED_CASES(NV)                                                                                 \
  case shape_index(NV, 2, 2): fused_tile<NV, 2, 2, kMixed>(c, tl.base, tl.n, clog2, smem); break;          \
  case shape_index(NV, 3, 3): fused_tile<NV, 3, 3, kMixed>(c, tl.base, tl.n, clog2, smem); break;          \
  case shape_index(NV, 3, 2): fused_tile<NV, 3, 2, kMixed>(c, tl.base, tl.n, clog2, smem); break;          \
  case shape_index(NV, 2, 1): fused_tile<NV, 2, 1, kMixed>(c, tl.base, tl.n, clog2, smem); break;          \
  case shape_index(NV, 3, 1): fused_tile<NV, 3, 1, kMixed>(c, tl.base, tl.n, clog2, smem); break;

template <bool kMixed>
__global__ void __launch_bounds__(kFindThreads, kFusedCtas)
    k_find_fused(const FusedClass* __restrict__ classes, const FusedTile* __restrict__ tiles, int ntiles,
                 int* __restrict__ counter, int clog2, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_tile;
  for (int guard = 0;; ++guard) {
    __syncthreads();  // every warp is done with the previous tile
    if (threadIdx.x == 0) s_tile = guard < ntiles + 1 ? atomicAdd(counter, 1) : ntiles;
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) break;
    const FusedTile tl = tiles[t];
    const FusedClass& c = classes[tl.cls];
    switch (c.shape) {
      FP_FUSED_CASES(2)
      FP_FUSED_CASES(3)
      FP_FUSED_CASES(4)
      FP_FUSED_CASES(5)
      FP_FUSED_CASES(6)
      FP_FUSED_CASES(7)
      FP_FUSED_CASES(8)
      default:
        if (threadIdx.x == 0) record_status(status, FP_DEV_BAD_ELEM);
    }
  }
}

#undef FP_FUSED_CASES

template <int N, int D, int DR>
constexpr size_t fused_smem_of(bool mixed) {
  return mixed ? sizeof(MixedShared<N, D, DR>) : sizeof(F64Shared<N, D, DR>);
}

size_t fused_smem(bool mixed) {
  size_t b = 0;
  for (int N = 2; N <= FP_MAX_N; ++N)
    for (int s = 0; s < 5; ++s) {
      const int d = (s == 0 || s == 3) ? 2 : 3, dr = s == 0 ? 2 : s == 1 ? 3 : s == 2 ? 2 : 1;
      dispatch_shape(N, d, dr, [&](auto Nc, auto Dc, auto DRc) -> int {
        b = std::max(b, fused_smem_of<decltype(Nc)::value, decltype(Dc)::value, decltype(DRc)::value>(mixed));
        return FP_OK;
      });
    }
  return b;
}

}  // namespace

int shape_of(int N, int d, int dr) { return shape_index(N, d, dr); }

int launch_fused(const FusedClass* classes, const FusedTile* tiles, int ntiles, int* counter, int precision,
                 int* status, cudaStream_t st) {
  const bool mixed = precision == FP_MIXED;
  const size_t smem = fused_smem(mixed);
  const int blocks = sm_count() * kFusedCtas;
  if (mixed) {
    if (cudaFuncSetAttribute(k_find_fused<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return FP_ELAUNCH;
    k_find_fused<true><<<blocks, kFindThreads, smem, st>>>(classes, tiles, ntiles, counter, 5, status);
  } else {
    if (cudaFuncSetAttribute(k_find_fused<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return FP_ELAUNCH;
    k_find_fused<false><<<blocks, kFindThreads, smem, st>>>(classes, tiles, ntiles, counter, 5, status);
  }
  return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ELAUNCH;
}

}  // namespace fp
