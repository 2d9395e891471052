// Per-kernel CUDA-event timing of a mesh's find and eval calls
// (fp_set_timing / fp_kernel_times): the events are recorded on the
// caller's stream between the kernels of each call, so a benchmark can
// divide a kernel's algorithmic work by that kernel's own duration.
#include <mutex>
#include <set>
#include <vector>

#include "fp_common.cuh"

namespace fp {

struct KernelTimer {
  struct Span {
    int stage;
    cudaEvent_t a, b;
  };
  std::mutex mu;
  bool on = false;
  std::vector<cudaEvent_t> spare;  // events whose intervals have been read
  std::vector<cudaEvent_t> used;   // events recorded since the last read
  std::vector<Span> spans;
  static constexpr size_t kMaxSpans = 65536;
};

cudaEvent_t timer_mark(const fp_mesh_s* m, cudaStream_t st) {
  KernelTimer* t = m->timer;
  if (!t) return nullptr;
  std::lock_guard<std::mutex> lk(t->mu);
  if (!t->on || t->spans.size() >= KernelTimer::kMaxSpans) return nullptr;
  cudaEvent_t ev = nullptr;
  if (!t->spare.empty()) {
    ev = t->spare.back();
    t->spare.pop_back();
  } else if (cudaEventCreate(&ev) != cudaSuccess) {
    return nullptr;
  }
  if (cudaEventRecord(ev, st) != cudaSuccess) {
    t->spare.push_back(ev);
    return nullptr;
  }
  t->used.push_back(ev);
  return ev;
}

void timer_span(const fp_mesh_s* m, int stage, cudaEvent_t a, cudaEvent_t b) {
  KernelTimer* t = m->timer;
  if (!t || !a || !b || stage < 0 || stage >= FP_NTIMES) return;
  std::lock_guard<std::mutex> lk(t->mu);
  t->spans.push_back({stage, a, b});
}

void timer_free(fp_mesh_s* m) {
  KernelTimer* t = m->timer;
  if (!t) return;
  for (cudaEvent_t ev : t->spare) cudaEventDestroy(ev);
  for (cudaEvent_t ev : t->used) cudaEventDestroy(ev);  // released once complete
  delete t;
  m->timer = nullptr;
}

}  // namespace fp

extern "C" int fp_set_timing(fp_mesh m, int on) {
  if (!m) return FP_EINVAL;
  if (!m->timer) {
    if (!on) return FP_OK;
    m->timer = new (std::nothrow) fp::KernelTimer();
    if (!m->timer) return FP_ENOMEM;
  }
  std::lock_guard<std::mutex> lk(m->timer->mu);
  m->timer->on = on != 0;
  return FP_OK;
}

extern "C" int fp_kernel_times(fp_mesh m, double* ms, int64_t* calls) {
  if (!m || !ms) return FP_EINVAL;
  for (int s = 0; s < FP_NTIMES; ++s) {
    ms[s] = 0.0;
    if (calls) calls[s] = 0;
  }
  fp::KernelTimer* t = m->timer;
  if (!t) return FP_OK;
  std::lock_guard<std::mutex> lk(t->mu);
  int rc = FP_OK;
  for (const auto& sp : t->spans) {
    float v = 0.f;
    if (cudaEventSynchronize(sp.b) != cudaSuccess || cudaEventElapsedTime(&v, sp.a, sp.b) != cudaSuccess) {
      rc = FP_ELAUNCH;
      continue;
    }
    ms[sp.stage] += v;
    if (calls) ++calls[sp.stage];
  }
  for (cudaEvent_t ev : t->used) cudaEventSynchronize(ev);
  t->spare.insert(t->spare.end(), t->used.begin(), t->used.end());
  t->used.clear();
  t->spans.clear();
  return rc;
}
