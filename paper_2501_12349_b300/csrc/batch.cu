// Batched find + eval over many meshes in one graph launch.
//
// A plan groups the caller's (mesh, points, outputs[, field]) items by
// element shape (N, d, dr).  Per shape it uploads the item table once and
// runs one persistent find launch over all its items (lanes pull points from
// the whole shape's point sequence, so many small meshes fill the GPU
// together), plus one eval launch.  The launches of all shapes are captured
// once into a CUDA graph on forked streams; fp_batch_run replays it.  The
// launch shape of each class (CTAs per SM, points per CTA chunk) is picked
// by fp_batch_autotune, which times the candidates on the batch's own data.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "eval_df.cuh"
#include "find_common.cuh"

namespace fp {


namespace {

constexpr int kEvalThreads = 128;

// Eval (Sec. 3.3) for every point of every item that carries a field.
template <int N, int DR>
__global__ void __launch_bounds__(kEvalThreads)
    k_eval_batch(const BatchItem* __restrict__ items, int nitems, int64_t total, const BasisTab B) {
  constexpr int NN = ipow(N, DR);
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].start <= g) lo = mid;
      else hi = mid - 1;
    }
    const BatchItem& it = items[lo];
    if (it.field == nullptr || it.nc <= 0) continue;
    const int64_t p = g - it.start;
    const int c0 = it.code[p], e = it.elem[p];
    const int64_t NE = it.m.NE;
    if (c0 == FP_NOT_FOUND || e < 0 || e >= NE) {
      if (c0 != FP_NOT_FOUND) record_status(it.m.status, FP_DEV_BAD_ELEM);
      for (int c = 0; c < it.nc; ++c) it.out[(int64_t)c * it.ld + p] = 0.0;
      continue;
    }
    double ph[DR][N], dph[DR][N] = {};  // dph unused: values only
#pragma unroll
    for (int j = 0; j < DR; ++j) lagrange_sym_values<N, double>(B, it.r[p * DR + j], ph[j]);
    for (int c = 0; c < it.nc; ++c) {
      double v;
      map_eval<N, DR, 1, false, double>(it.field + (c * NE + e) * NN, 0, ph, dph, &v, nullptr);
      it.out[(int64_t)c * it.ld + p] = v;
    }
  }
}

int launch_eval_class(const BatchItem* items, int nitems, int64_t total, int N, int d, int dr,
                      const BasisTab& B, cudaStream_t st) {
  return dispatch_shape(N, d, dr, [&](auto Nc, auto Dc, auto DRc) -> int {
    constexpr int NN = decltype(Nc)::value, DR = decltype(DRc)::value;
    (void)Dc;
    const int blocks = grid_for(total, kEvalThreads, sm_count() * 16);
    k_eval_batch<NN, DR><<<blocks, kEvalThreads, 0, st>>>(items, nitems, total, B);
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ELAUNCH;
  });
}

struct Tuning {
  int ctas_per_sm = 0;  // 0: the kernel's own (mixed_ctas(N, d, dr) mixed; f64_ctas(N) FP64)
  int clog2 = 5;
  float ms = -1.f;  // measured time of the chosen shape, -1 if untuned
};

// Process-wide cache of tuned shapes: (N, d, dr, precision, log2 points).
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int, int>, Tuning> g_tune_cache;

int log2_bucket(int64_t n) {
  int b = 0;
  while ((int64_t(1) << (b + 1)) <= n) ++b;
  return b;
}

struct ClassPlan {
  int N, d, dr;
  BasisTab B;
  std::vector<BatchItem> items;
  int64_t total = 0;
  BatchItem* d_items = nullptr;
  int* d_queue = nullptr;  // total + 1 ints: mixed-path queue and its counter
  int* d_order = nullptr;  // cell-order scratch (NULL: points as given)
  int64_t buckets = 0;     // sum over items of (Psi_L cells + 1)
  bool unordered = false;  // some item's mesh takes its points as given
  bool has_field = false;
  // FP_MIXED: double-float interpolation (the items' fields split on every
  // run, in the point order), where it pays (see df_pays)
  bool df = false;
  float2* d_fs = nullptr;
  int* d_fexp = nullptr;
  SplitJob* d_jobs = nullptr;
  int njobs = 0;
  int64_t max_per = 0;
  Tuning tune;
  cudaStream_t side = nullptr;
  cudaEvent_t join = nullptr;
};

}  // namespace
}  // namespace fp

struct fp_batch_s {
  std::vector<fp::ClassPlan> classes;
  int precision = FP_F64;
  // the fused form (one persistent find launch over all shapes)
  bool fused = false;
  fp::FusedClass* d_fclasses = nullptr;
  fp::FusedTile* d_tiles = nullptr;
  int ntiles = 0;
  int* d_counter = nullptr;
  int* status = nullptr;  // the first item's mesh status word
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;  // the plan's own stream: the caller's may be
                               // the legacy default stream, which cannot be captured
  int64_t total_points = 0;
};

namespace fp {
namespace {

// The eval of one class: the double-float contraction over the class's
// point order after splitting its fields (FP_MIXED, where it pays), else
// the FP64 one in the items' order.
int enqueue_eval(ClassPlan& c, cudaStream_t st) {
  if (!c.has_field) return FP_OK;
  if (!c.df) return launch_eval_class(c.d_items, (int)c.items.size(), c.total, c.N, c.d, c.dr, c.B, st);
  FP_CUDA_TRY(cudaMemsetAsync(c.d_fexp, 0, sizeof(int) * (size_t)c.njobs, st));
  FP_TRY(split_fields(SplitJobs{c.d_jobs, nullptr, 0, nullptr, nullptr}, c.njobs, c.max_per, st));
  return dispatch_shape(c.N, c.d, c.dr, [&](auto Nc, auto Dc, auto DRc) -> int {
    constexpr int NN = decltype(Nc)::value, DR = decltype(DRc)::value;
    (void)Dc;
    k_eval_items_df<NN, DR><<<grid_for(c.total, 128, sm_count() * 16), 128, 0, st>>>(
        c.d_items, (int)c.items.size(), c.total, c.d_order, c.B);
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ELAUNCH;
  });
}

// Enqueues one class: counter reset, find launch(es), eval launch.
int enqueue_class(ClassPlan& c, int precision, const Tuning& t, cudaStream_t st) {
  if (c.total == 0) return FP_OK;
  int* qcount = c.d_queue + c.total;
  if (precision == FP_MIXED) FP_CUDA_TRY(cudaMemsetAsync(qcount, 0, sizeof(int), st));
  int* order = nullptr;
  if (c.d_order)
    FP_TRY(batch_cell_order(c.d_items, (int)c.items.size(), c.total, c.d, c.buckets, c.d_order, &order, st));
  FP_TRY(launch_batch_class(c.d_items, (int)c.items.size(), c.total, c.N, c.d, c.dr, c.B, precision,
                            t.ctas_per_sm, t.clog2, order, c.d_queue, qcount, nullptr, st));
  return enqueue_eval(c, st);
}

void destroy_graph(fp_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Points per tile of the fused launch: 32 per thread of a CTA.
constexpr int kFusedTile = 32 * kFindThreads;

// The fused form's class and tile tables: the classes' tiles, costliest
// shape first (its points take longest), each class's tiles in its point
// order (costly cost classes first).
int build_fused_tables(fp_batch_s* b, cudaStream_t st) {
  std::vector<FusedClass> fc;
  std::vector<int> ids;
  for (size_t i = 0; i < b->classes.size(); ++i) {
    const ClassPlan& c = b->classes[i];
    FusedClass f;
    memset(&f, 0, sizeof(f));
    f.items = c.d_items;
    f.nitems = (int)c.items.size();
    f.shape = shape_of(c.N, c.d, c.dr);
    f.order = c.d_order;  // batch_cell_order puts the permutation at the scratch start
    f.queue = c.d_queue;
    f.qcount = c.d_queue ? c.d_queue + c.total : nullptr;
    f.B = c.B;
    fc.push_back(f);
    if (c.total > 0) ids.push_back((int)i);
  }
  auto cost = [&](int i) {
    const ClassPlan& c = b->classes[i];
    return (double)ipow(c.N, c.dr) * (2 * c.N + 3) * c.d;
  };
  std::stable_sort(ids.begin(), ids.end(), [&](int a, int x) { return cost(a) > cost(x); });
  std::vector<FusedTile> tiles;
  for (int i : ids)
    for (int64_t g = 0; g < b->classes[i].total; g += kFusedTile)
      tiles.push_back({i, (int)std::min<int64_t>(kFusedTile, b->classes[i].total - g), g});
  b->ntiles = (int)tiles.size();
  if (fc.empty() || tiles.empty()) return FP_OK;
  if (cudaMalloc(&b->d_fclasses, sizeof(FusedClass) * fc.size()) != cudaSuccess ||
      cudaMalloc(&b->d_tiles, sizeof(FusedTile) * tiles.size()) != cudaSuccess ||
      cudaMalloc(&b->d_counter, sizeof(int)) != cudaSuccess)
    return FP_ENOMEM;
  FP_CUDA_TRY(cudaMemcpyAsync(b->d_fclasses, fc.data(), sizeof(FusedClass) * fc.size(), cudaMemcpyHostToDevice, st));
  FP_CUDA_TRY(cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(FusedTile) * tiles.size(), cudaMemcpyHostToDevice, st));
  return FP_OK;
}

// The fused form: per class (forked) the point order and the queue counter,
// then one persistent find launch over every class's tiles, then per class
// (forked) the FP64 follow-up of FP_MIXED and the eval.
int capture_fused(fp_batch_s* b) {
  cudaStream_t st = b->cap;
  FP_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int rc = FP_OK;
  auto fork_classes = [&](auto&& body) {
    if (rc == FP_OK && cudaEventRecord(b->fork, st) != cudaSuccess) rc = FP_ELAUNCH;
    for (auto& c : b->classes) {
      if (rc != FP_OK) break;
      if (c.total == 0) continue;
      if (cudaStreamWaitEvent(c.side, b->fork, 0) != cudaSuccess) {
        rc = FP_ELAUNCH;
        break;
      }
      rc = body(c);
      if (rc == FP_OK && (cudaEventRecord(c.join, c.side) != cudaSuccess ||
                          cudaStreamWaitEvent(st, c.join, 0) != cudaSuccess))
        rc = FP_ELAUNCH;
    }
  };
  fork_classes([&](ClassPlan& c) -> int {
    if (b->precision == FP_MIXED) FP_CUDA_TRY(cudaMemsetAsync(c.d_queue + c.total, 0, sizeof(int), c.side));
    int* order = nullptr;
    if (c.d_order)
      FP_TRY(batch_cell_order(c.d_items, (int)c.items.size(), c.total, c.d, c.buckets, c.d_order, &order, c.side));
    return FP_OK;
  });
  if (rc == FP_OK && cudaMemsetAsync(b->d_counter, 0, sizeof(int), st) != cudaSuccess) rc = FP_ELAUNCH;
  if (rc == FP_OK) rc = launch_fused(b->d_fclasses, b->d_tiles, b->ntiles, b->d_counter, b->precision, b->status, st);
  fork_classes([&](ClassPlan& c) -> int {
    if (b->precision == FP_MIXED)
      FP_TRY(launch_batch_follow(c.d_items, (int)c.items.size(), c.total, c.N, c.d, c.dr, c.B, c.d_queue,
                                 c.d_queue + c.total, c.side));
    return enqueue_eval(c, c.side);
  });
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  if (rc != FP_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rc != FP_OK ? rc : FP_ELAUNCH;
  }
  b->graph = g;
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    destroy_graph(b);
    return FP_ELAUNCH;
  }
  return FP_OK;
}

// Captures every class's work, each on its own forked stream, into b->exec
// (the fused form: capture_fused).
int capture(fp_batch_s* b) {
  cudaStream_t st = b->cap;
  destroy_graph(b);
  if (b->fused) return capture_fused(b);
  FP_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int rc = FP_OK;
  if (cudaEventRecord(b->fork, st) != cudaSuccess) rc = FP_ELAUNCH;
  for (auto& c : b->classes) {
    if (rc != FP_OK) break;
    if (c.total == 0) continue;
    if (cudaStreamWaitEvent(c.side, b->fork, 0) != cudaSuccess) {
      rc = FP_ELAUNCH;
      break;
    }
    rc = enqueue_class(c, b->precision, c.tune, c.side);
    if (rc == FP_OK && (cudaEventRecord(c.join, c.side) != cudaSuccess ||
                        cudaStreamWaitEvent(st, c.join, 0) != cudaSuccess))
      rc = FP_ELAUNCH;
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  if (rc != FP_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rc != FP_OK ? rc : FP_ELAUNCH;
  }
  b->graph = g;
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    destroy_graph(b);
    return FP_ELAUNCH;
  }
  return FP_OK;
}

void free_plan(fp_batch_s* b) {
  destroy_graph(b);
  for (auto& c : b->classes) {
    cudaFree(c.d_items);
    cudaFree(c.d_queue);
    cudaFree(c.d_order);
    cudaFree(c.d_fs);
    cudaFree(c.d_fexp);
    cudaFree(c.d_jobs);
    if (c.side) cudaStreamDestroy(c.side);
    if (c.join) cudaEventDestroy(c.join);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaFree(b->d_fclasses);
  cudaFree(b->d_tiles);
  cudaFree(b->d_counter);
}

}  // namespace
}  // namespace fp

extern "C" int fp_batch_create(const fp_mesh* meshes, int nm, const fp_batch_item* items,
                               int nitems, int precision, void* stream, fp_batch* out) {
  using namespace fp;
  if (!out) return FP_EINVAL;
  *out = nullptr;
  if (!meshes || nm <= 0 || !items || nitems <= 0) return FP_EINVAL;
  if (precision != FP_F64 && precision != FP_MIXED) return FP_EINVAL;
  for (int i = 0; i < nitems; ++i) {
    const fp_batch_item& it = items[i];
    if (it.mesh < 0 || it.mesh >= nm || !meshes[it.mesh] || it.n < 0 || it.n > INT32_MAX) return FP_EINVAL;
    if (it.n > 0 && (!it.pts || !it.code || !it.elem || !it.r || !it.dist2)) return FP_EINVAL;
    if (it.field && (it.nc <= 0 || !it.out)) return FP_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  fp_batch_s* b = new fp_batch_s();
  b->precision = precision;
  // group by element shape, items kept in the caller's order within a class
  std::map<std::tuple<int, int, int>, int> cls;
  for (int i = 0; i < nitems; ++i) {
    const fp_mesh_s* m = meshes[items[i].mesh];
    const auto key = std::make_tuple(m->N, m->d, m->dr);
    auto f = cls.find(key);
    int ci;
    if (f == cls.end()) {
      ci = (int)b->classes.size();
      cls[key] = ci;
      b->classes.emplace_back();
      ClassPlan& c = b->classes.back();
      c.N = m->N;
      c.d = m->d;
      c.dr = m->dr;
      c.B = m->basis;
    } else {
      ci = f->second;
    }
    ClassPlan& c = b->classes[ci];
    BatchItem bi;
    memset(&bi, 0, sizeof(bi));
    bi.m = m->view();
    bi.pts = items[i].pts;
    bi.n = items[i].n;
    bi.start = c.total;
    bi.code = items[i].code;
    bi.elem = items[i].elem;
    bi.r = items[i].r;
    bi.dist2 = items[i].dist2;
    bi.field = items[i].field;
    bi.nc = items[i].field ? items[i].nc : 0;
    bi.out = items[i].out;
    bi.ld = items[i].n;
    if (bi.field) c.has_field = true;
    if (bi.n > 0) {
      bi.key_base = c.buckets;
      c.buckets += order_keys(m);
      c.items.push_back(bi);
      c.total += bi.n;
      if (m->opts.point_order != FP_ORDER_CELL) c.unordered = true;
    }
  }
  int rc = FP_OK;
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
    rc = FP_ELAUNCH;
  for (auto& c : b->classes) {
    if (rc != FP_OK) break;
    b->total_points += c.total;
    if (c.total > INT32_MAX) {
      rc = FP_EINVAL;
      break;
    }
    if (c.items.empty()) continue;
    {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      auto f = g_tune_cache.find(std::make_tuple(c.N, c.d, c.dr, precision, log2_bucket(c.total)));
      if (f != g_tune_cache.end()) c.tune = f->second;
    }
    if (cudaMalloc(&c.d_items, sizeof(BatchItem) * c.items.size()) != cudaSuccess ||
        cudaMalloc(&c.d_queue, sizeof(int) * (size_t)(c.total + 1)) != cudaSuccess) {
      rc = FP_ENOMEM;
      break;
    }
    // the cell order (as for single-mesh calls of at least 16384 points)
    if (!c.unordered && c.total >= (1 << 14) && 4 * c.buckets + 1 < INT32_MAX &&
        cudaMalloc(&c.d_order, sizeof(int) * (size_t)batch_cell_order_ints(c.total, c.buckets)) != cudaSuccess) {
      rc = FP_ENOMEM;
      break;
    }
    // FP_MIXED double-float interpolation where it pays: quads, hexes and
    // surfaces in the point order, at least 8 points per element of the
    // items with a field (the fields are split on every run)
    if (precision == FP_MIXED && c.dr >= 2 && c.has_field && c.d_order) {
      int64_t vals = 0, ne_sum = 0;
      int nj = 0;
      const int NN = ipow(c.N, c.dr);
      for (const auto& it : c.items)
        if (it.field) {
          vals += (int64_t)it.nc * it.m.NE * NN;
          ne_sum += it.m.NE;
          nj += it.nc;
        }
      if (c.total >= 8 * ne_sum && nj > 0) {
        if (cudaMalloc(&c.d_fs, sizeof(float2) * (size_t)vals) != cudaSuccess ||
            cudaMalloc(&c.d_fexp, sizeof(int) * (size_t)nj) != cudaSuccess ||
            cudaMalloc(&c.d_jobs, sizeof(SplitJob) * (size_t)nj) != cudaSuccess) {
          rc = FP_ENOMEM;
          break;
        }
        std::vector<SplitJob> jobs;
        int64_t off = 0;
        int eo = 0;
        for (auto& it : c.items) {
          if (!it.field) continue;
          const int64_t per = it.m.NE * NN;
          it.fs = c.d_fs + off;
          it.fexp = c.d_fexp + eo;
          for (int q = 0; q < it.nc; ++q)
            jobs.push_back(SplitJob{it.field + q * per, per, c.d_fs + off + q * per, c.d_fexp + eo + q});
          off += (int64_t)it.nc * per;
          eo += it.nc;
          c.max_per = std::max(c.max_per, per);
        }
        c.njobs = nj;
        c.df = true;
        if (cudaMemcpy(c.d_jobs, jobs.data(), sizeof(SplitJob) * jobs.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
          rc = FP_ELAUNCH;
          break;
        }
      }
    }
    if (cudaMemcpyAsync(c.d_items, c.items.data(), sizeof(BatchItem) * c.items.size(),
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c.side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c.join, cudaEventDisableTiming) != cudaSuccess) {
      rc = FP_ELAUNCH;
      break;
    }
  }
  if (rc == FP_OK) {
    b->status = meshes[items[0].mesh]->status;
    rc = build_fused_tables(b, st);
  }
  if (rc == FP_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = FP_ELAUNCH;
  if (rc == FP_OK) rc = capture(b);
  if (rc != FP_OK) {
    cudaStreamSynchronize(st);
    free_plan(b);
    delete b;
    return rc;
  }
  *out = b;
  return FP_OK;
}

extern "C" int fp_batch_set_fused(fp_batch b, int on) {
  if (!b) return FP_EINVAL;
  b->fused = on != 0;
  return fp::capture(b);
}

extern "C" int fp_batch_run(fp_batch b, void* stream) {
  if (!b || !b->exec) return FP_EINVAL;
  FP_CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  return FP_OK;
}

extern "C" int fp_batch_autotune(fp_batch b, void* stream) {
  using namespace fp;
  if (!b) return FP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int clogs[3] = {5, 7, 9};
  cudaEvent_t e0, e1;
  FP_CUDA_TRY(cudaEventCreate(&e0));
  FP_CUDA_TRY(cudaEventCreate(&e1));
  int rc = FP_OK;
  for (auto& c : b->classes) {
    if (c.total == 0 || rc != FP_OK) continue;
    Tuning best;
    // CTAs per SM: the kernel's register-limited maximum and one fewer
    const int cmax = b->precision == FP_MIXED ? mixed_ctas(c.N, c.d, c.dr) : f64_ctas(c.N);
    const int ctas[2] = {cmax - 1, cmax};
    for (int a = 0; a < 2 && rc == FP_OK; ++a)
      for (int k = 0; k < 3 && rc == FP_OK; ++k) {
        Tuning t;
        t.ctas_per_sm = ctas[a];
        t.clog2 = clogs[k];
        float ms_best = 1e30f;
        for (int rep = 0; rep < 3 && rc == FP_OK; ++rep) {  // first rep warms up
          cudaEventRecord(e0, st);
          rc = enqueue_class(c, b->precision, t, st);
          cudaEventRecord(e1, st);
          if (cudaEventSynchronize(e1) != cudaSuccess) rc = FP_ELAUNCH;
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) ms_best = std::min(ms_best, ms);
        }
        t.ms = ms_best;
        if (best.ms < 0.f || t.ms < best.ms) best = t;
      }
    if (rc == FP_OK) {
      c.tune = best;
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      g_tune_cache[std::make_tuple(c.N, c.d, c.dr, b->precision, log2_bucket(c.total))] = best;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == FP_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = FP_ELAUNCH;
  if (rc == FP_OK) rc = capture(b);
  return rc;
}

extern "C" int fp_batch_describe(fp_batch b, int i, fp_batch_class_info* info) {
  if (!b || !info || i < 0 || i >= (int)b->classes.size()) return FP_EINVAL;
  const auto& c = b->classes[i];
  info->N = c.N;
  info->d = c.d;
  info->dr = c.dr;
  info->n_items = (int)c.items.size();
  info->n_points = c.total;
  info->ctas_per_sm = c.tune.ctas_per_sm > 0 ? c.tune.ctas_per_sm
                                             : (b->precision == FP_MIXED ? fp::mixed_ctas(c.N, c.d, c.dr)
                                                                          : fp::f64_ctas(c.N));
  info->chunk_points = 1 << c.tune.clog2;
  info->tuned_ms = c.tune.ms;
  return FP_OK;
}

extern "C" int fp_batch_num_classes(fp_batch b) { return b ? (int)b->classes.size() : FP_EINVAL; }

extern "C" int fp_batch_free(fp_batch b) {
  if (!b) return FP_EINVAL;
  cudaDeviceSynchronize();
  fp::free_plan(b);
  delete b;
  return FP_OK;
}
