// fp_findpts_mixed_noalloc: the mixed-precision find without any device
// allocation.  The paper has no counterpart; this entry point exists for
// callers that cannot let a library allocate GPU memory (see findpts.h).
//
// The mixed path's only scratch memory is its queue of points handed from
// the FP32 kernel to the FP64 kernel (one int per point plus a counter).
// Here that queue is a file-scope device array of fixed size: every GPU
// that loads this library holds it (4 MiB) until the process exits.
#include <mutex>

#include "find_common.cuh"

namespace {

// Queue entries [0, FP_NOALLOC_MAX_POINTS) and the counter at the end.
static __device__ __align__(256) int g_noalloc_queue[FP_NOALLOC_MAX_POINTS + 1];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
int* g_queue_on_device[kMaxDevices] = {};

// The device address of g_noalloc_queue on the current device.  In host
// code the array's name is only a host-side stand-in, so the address is
// looked up once per device (with that device current) and cached.
int queue_on_current_device(int** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FP_ELAUNCH;
  if (dev < 0 || dev >= kMaxDevices) return FP_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_queue_on_device[dev] == nullptr) {
    int* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_queue);
    if (e != cudaSuccess || p == nullptr) return FP_ELAUNCH;
    g_queue_on_device[dev] = p;
  }
  *out = g_queue_on_device[dev];
  return FP_OK;
}

}  // namespace

extern "C" int fp_findpts_mixed_noalloc(fp_mesh m, const double* pts, int64_t n, int32_t* code,
                                        int32_t* elem, double* r, double* dist2, void* stream) {
  if (!m || n < 0) return FP_EINVAL;
  if (n > FP_NOALLOC_MAX_POINTS) return FP_EINVAL;  // beyond the fixed scratch size
  if (n == 0) return FP_OK;
  if (!pts || !code || !elem || !r || !dist2) return FP_EINVAL;
  int* queue = nullptr;
  FP_TRY(queue_on_current_device(&queue));
  cudaStream_t st = (cudaStream_t)stream;
  int* qcount = queue + FP_NOALLOC_MAX_POINTS;
  // the counter must start at zero; queue entries are only read below it
  FP_CUDA_TRY(cudaMemsetAsync(qcount, 0, sizeof(int), st));
  return fp::launch_mixed_with_queue(m, pts, nullptr, n, code, elem, r, dist2, queue, qcount, nullptr, st);
}
