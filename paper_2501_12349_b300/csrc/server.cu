// Continuous-batching server over resident meshes.
//
// Requests:
//   remap    — find the points, interpolate the mesh's resident field
//              (the remap of Sec. 6.4: Find once, Interpolate);
//   particle — K explicit-midpoint (RK2) steps through the mesh's resident
//              velocity field (the Find / Interpolate / Integrate loop of the
//              particle-tracking algorithm, Sec. 6.7), then a final find of
//              the end positions.  A particle that leaves the mesh is
//              NOT_FOUND, its interpolated velocity is 0 and it stays put.
// A scheduler thread runs ticks.  A tick takes tiles (contiguous ranges of
// points) of the current stage of the ready requests, those with the least
// work left in their stage first, up to a budget of points per tick, so a
// large request proceeds tile by tile while small ones pass it; it packs the
// tiles into batch tables grouped by element shape and issues one find launch
// per shape (FP64 or mixed) and one eval launch per shape, the shapes side by
// side on streams forked from the tick's stream (a small shape's launch is
// bound by its slowest points, not by the GPU, so shapes in sequence would
// add up their critical paths), then one particle-advance launch; up to two
// ticks are in flight, and a request's stage ends when all its tiles have
// finished.  Requests are admitted when a first-fit arena inside a fixed
// device-memory budget and a slot are free; host<->device copies run on an
// upload and a download stream of their own, so arriving requests' uploads
// and finished requests' downloads overlap the ticks and each other (the
// link's two directions).  Every device wait on the host is bounded (poll +
// sleep with a deadline); a tick that exceeds it fails its requests with
// FP_ETIMEDOUT.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "eval_df.cuh"
#include "find_common.cuh"

namespace fp {


namespace {

using Clock = std::chrono::steady_clock;

// ---- device: batched eval and particle advance --------------------------------

template <int N, int DR>
__global__ void __launch_bounds__(128)
    k_serve_eval(const BatchItem* __restrict__ items, int nitems, int64_t total, const BasisTab B) {
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

// One particle stage over a tile of a request's points: mode 0 (midpoint)
// xs = x + c u; mode 1 (full step) x = x + c u and xs = x.  u holds the
// stage's interpolated velocity, component k at u + k * ld.
struct AdvItem {
  double* x;
  double* xs;
  const double* u;
  int64_t n;
  int64_t ld;
  int64_t start;
  double c;
  int mode;
  int d;
};

__global__ void k_advance(const AdvItem* __restrict__ items, int nitems, int64_t total) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].start <= g) lo = mid;
      else hi = mid - 1;
    }
    const AdvItem& it = items[lo];
    const int64_t p = g - it.start;
    for (int c = 0; c < it.d; ++c) {
      const double v = it.x[p * it.d + c] + it.c * it.u[(int64_t)c * it.ld + p];
      if (it.mode == 0) {
        it.xs[p * it.d + c] = v;
      } else {
        it.x[p * it.d + c] = v;
        it.xs[p * it.d + c] = v;
      }
    }
  }
}

// ---- host: arena, requests, ticks ------------------------------------------------

// First-fit allocator over one device buffer (256-byte granules).
struct Arena {
  char* base = nullptr;
  size_t size = 0, used = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  bool init(size_t bytes) {
    size = (bytes + 255) & ~size_t(255);
    if (cudaMalloc(&base, size) != cudaSuccess) return false;
    free_[0] = size;
    return true;
  }
  void* alloc(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        used += bytes;
        return base + off;
      }
    }
    return nullptr;
  }
  void release(void* p, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    size_t off = (char*)p - base;
    used -= bytes;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
};

enum RState { R_QUEUED, R_UPLOADING, R_READY, R_DOWNLOADING, R_DONE };

struct Request {
  int64_t id;
  int mesh, kind, rk_steps;
  int64_t n;
  double dt;
  const double* pts_h;
  int32_t *code_h, *elem_h;
  double *r_h, *dist2_h, *out_h;
  RState state = R_QUEUED;
  int status = FP_OK;
  int stage = 0, nstages = 1;
  int64_t next = 0;  // first point of the current stage not yet given to a tick
  int64_t done = 0;  // points of the current stage finished
  int inflight = 0;  // tiles of this request in ticks on the GPU
  size_t bytes = 0;
  char* block = nullptr;
  double *x = nullptr, *xs = nullptr, *r = nullptr, *dist2 = nullptr, *u = nullptr;
  int32_t *code = nullptr, *elem = nullptr;
  int nc = 0;
  cudaEvent_t ev = nullptr;  // upload / download completion
  Clock::time_point t_submit, t_admit, t_done;
  int64_t born = 0;  // stage points the server had finished at submission
};

struct MeshEntry {
  fp_mesh_s* m;
  const double* remap_field;
  int nc_remap;
  const double* vel;
  // FP_MIXED, quads/hexes/surfaces: the fields as double-float pairs (split
  // at creation) and their components' scaling exponents
  float2* remap_fs = nullptr;
  int* remap_fexp = nullptr;
  float2* vel_fs = nullptr;
  int* vel_fexp = nullptr;
};

// The double-float copy of a resident field ([nc][NE][N^dr]): allocated and
// split on stream st.
int split_resident(const double* field, int nc, int64_t per, float2** fs, int** fexp, cudaStream_t st) {
  FP_CUDA_TRY(cudaMalloc(fs, sizeof(float2) * (size_t)nc * (size_t)per));
  FP_CUDA_TRY(cudaMalloc(fexp, sizeof(int) * (size_t)nc));
  FP_CUDA_TRY(cudaMemsetAsync(*fexp, 0, sizeof(int) * (size_t)nc, st));
  return split_fields(SplitJobs{nullptr, field, per, *fs, *fexp}, nc, per, st);
}

// A contiguous range of one request's points within one tick.
struct Tile {
  int64_t id, off, len;
};

constexpr int kTickForks = 6;

struct TickSlot {
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  bool timed_out = false;
  int fail_rc = 0;  // a launch of this tick failed: its requests fail at completion
  Clock::time_point started;
  std::vector<Tile> tiles;
  BatchItem* items_h = nullptr;  // pinned
  BatchItem* items_d = nullptr;
  AdvItem* adv_h = nullptr;
  AdvItem* adv_d = nullptr;
  int* queue = nullptr;
  int64_t queue_cap = 0;
  int* order = nullptr;  // cell-order scratch, carved into one range per shape
  int64_t order_cap = 0;
  // the shapes of a tick run side by side on these streams, forked from st
  // after the item tables are uploaded and joined back before the particle
  // advance and the tick's completion event
  cudaStream_t fork[kTickForks] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kTickForks] = {};
};

}  // namespace
}  // namespace fp

struct fp_server_s {
  std::vector<fp::MeshEntry> meshes;
  fp_server_opts opts;
  fp::Arena arena;
  cudaStream_t up = nullptr, down = nullptr;
  fp::TickSlot slot[2];
  int max_items = 0;
  int64_t tick_points = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> queued;
  std::unordered_map<int64_t, std::unique_ptr<fp::Request>> reqs;
  int64_t next_id = 1;
  int64_t served = 0;  // stage points finished (tiles of completed ticks)
  int active = 0;
  std::atomic<bool> stop{false};
  std::thread worker;
  fp_server_stats stats;
  int device = 0;
};

namespace fp {
namespace {

size_t request_bytes(const fp_server_s* s, int mesh, int kind, int64_t n) {
  const MeshEntry& me = s->meshes[mesh];
  const int d = me.m->d, dr = me.m->dr;
  const int nc = kind == FP_REQ_REMAP ? me.nc_remap : d;
  size_t b = 0;
  auto add = [&](size_t bytes) { b += (bytes + 255) & ~size_t(255); };
  add(sizeof(double) * n * d);       // x (points / positions)
  if (kind == FP_REQ_PARTICLE) add(sizeof(double) * n * d);  // stage positions
  add(sizeof(int32_t) * n * 2);      // code, elem
  add(sizeof(double) * n * dr);      // r
  add(sizeof(double) * n);           // dist2
  add(sizeof(double) * n * std::max(nc, 1));  // interpolated values
  return b;
}

void carve(fp_server_s* s, Request& q) {
  const MeshEntry& me = s->meshes[q.mesh];
  const int d = me.m->d, dr = me.m->dr;
  char* p = q.block;
  auto take = [&](size_t bytes) {
    char* r = p;
    p += (bytes + 255) & ~size_t(255);
    return r;
  };
  q.x = (double*)take(sizeof(double) * q.n * d);
  q.xs = q.kind == FP_REQ_PARTICLE ? (double*)take(sizeof(double) * q.n * d) : q.x;
  q.code = (int32_t*)take(sizeof(int32_t) * q.n * 2);
  q.elem = q.code + q.n;
  q.r = (double*)take(sizeof(double) * q.n * dr);
  q.dist2 = (double*)take(sizeof(double) * q.n);
  q.nc = q.kind == FP_REQ_REMAP ? me.nc_remap : d;
  q.u = (double*)take(sizeof(double) * q.n * std::max(q.nc, 1));
}

// Admission (lock held): first fit over the oldest queued requests.
void admit(fp_server_s* s) {
  int scanned = 0;
  for (auto it = s->queued.begin(); it != s->queued.end() && scanned < 32;) {
    ++scanned;
    if (s->active >= s->opts.max_active) break;
    Request& q = *s->reqs[*it];
    void* blk = s->arena.alloc(q.bytes);
    if (!blk) {
      ++it;
      continue;
    }
    q.block = (char*)blk;
    carve(s, q);
    const int d = s->meshes[q.mesh].m->d;
    cudaError_t e = cudaMemcpyAsync(q.x, q.pts_h, sizeof(double) * q.n * d, cudaMemcpyHostToDevice, s->up);
    if (e == cudaSuccess && q.kind == FP_REQ_PARTICLE)
      e = cudaMemcpyAsync(q.xs, q.x, sizeof(double) * q.n * d, cudaMemcpyDeviceToDevice, s->up);
    if (e == cudaSuccess) e = cudaEventRecord(q.ev, s->up);
    q.status = e == cudaSuccess ? FP_OK : FP_ELAUNCH;
    q.state = R_UPLOADING;
    q.t_admit = Clock::now();
    ++s->active;
    s->stats.admitted++;
    it = s->queued.erase(it);
  }
  s->stats.bytes_in_use = s->arena.used;
}

void finish(fp_server_s* s, Request& q, int status) {
  q.status = q.status != FP_OK ? q.status : status;
  q.state = R_DONE;
  q.t_done = Clock::now();
  if (q.block) {
    s->arena.release(q.block, q.bytes);
    q.block = nullptr;
  }
  --s->active;
  s->stats.completed++;
  s->stats.bytes_in_use = s->arena.used;
  s->cv_done.notify_all();
}

// Copies a request's results to its host buffers on the download stream.
void start_download(fp_server_s* s, Request& q) {
  const MeshEntry& me = s->meshes[q.mesh];
  const int d = me.m->d, dr = me.m->dr;
  cudaError_t e = cudaSuccess;
  auto cp = [&](void* h, const void* dv, size_t bytes) {
    if (h && e == cudaSuccess) e = cudaMemcpyAsync(h, dv, bytes, cudaMemcpyDeviceToHost, s->down);
  };
  cp(q.code_h, q.code, sizeof(int32_t) * q.n);
  cp(q.elem_h, q.elem, sizeof(int32_t) * q.n);
  cp(q.r_h, q.r, sizeof(double) * q.n * dr);
  cp(q.dist2_h, q.dist2, sizeof(double) * q.n);
  if (q.kind == FP_REQ_REMAP) cp(q.out_h, q.u, sizeof(double) * q.n * q.nc);
  else cp(q.out_h, q.x, sizeof(double) * q.n * d);
  if (e == cudaSuccess) e = cudaEventRecord(q.ev, s->down);
  if (e != cudaSuccess) q.status = FP_ELAUNCH;
  q.state = R_DOWNLOADING;
}

// (first item, items, points, queue offset, element shape, a mesh of the
// shape, cell-order buckets)
using TickLaunch = std::tuple<int, int, int64_t, int64_t, std::tuple<int, int, int>, const fp_mesh_s*, int64_t>;
int enqueue_tick(fp_server_s* s, TickSlot& t, const std::vector<TickLaunch>& launches, int ni, int na,
                 int64_t atotal);

// Builds one tick on slot t from the ready requests and launches it (lock
// held).  Returns 0 (nothing to do, or launched), or a negative status.
int launch_tick(fp_server_s* s, TickSlot& t) {
  t.tiles.clear();
  // tile-level interleaving: the requests in the policy's order, each takes
  // what the tick's point budget leaves (FP_SCHED_SRPT: least work left in
  // the current stage; FP_SCHED_SLACK: least slack, see findpts.h)
  std::vector<std::pair<double, int64_t>> cand;  // (key, id)
  for (auto& kv : s->reqs) {
    const Request& q = *kv.second;
    if (!(q.state == R_READY && q.status == FP_OK && q.next < q.n)) continue;
    double key = (double)(q.n - q.next);
    if (s->opts.policy == FP_SCHED_SLACK) {
      const double size = (double)q.n * q.nstages;
      const double left = (double)q.n * (q.nstages - q.stage) - (double)q.next;
      key = s->opts.slack_base + s->opts.slack_factor * size - (double)(s->served - q.born) - left;
    }
    cand.emplace_back(key, q.id);
  }
  if (cand.empty()) return 0;
  std::sort(cand.begin(), cand.end());
  int64_t budget = s->tick_points;
  for (auto& c : cand) {
    if (budget <= 0 || (int)t.tiles.size() >= s->max_items) break;
    const Request& q = *s->reqs[c.second];
    const int64_t len = std::min(q.n - q.next, budget);
    t.tiles.push_back({q.id, q.next, len});
    budget -= len;
  }
  // group by element shape
  std::map<std::tuple<int, int, int>, std::vector<int>> cls;
  for (int k = 0; k < (int)t.tiles.size(); ++k) {
    const Request& q = *s->reqs[t.tiles[k].id];
    const fp_mesh_s* m = s->meshes[q.mesh].m;
    cls[std::make_tuple(m->N, m->d, m->dr)].push_back(k);
  }
  int ni = 0, na = 0;
  int64_t qoff = 0, atotal = 0;
  std::vector<TickLaunch> launches;
  for (auto& kv : cls) {
    const int first = ni;
    int64_t total = 0;
    const fp_mesh_s* m0 = nullptr;
    // cell order: one range of buckets per mesh, shared by all its tiles,
    // so points of different requests in one cell are searched together
    std::map<int, int64_t> base;
    int64_t buckets = 0;
    for (int k : kv.second) {
      const Tile& tl = t.tiles[k];
      Request& q = *s->reqs[tl.id];
      const MeshEntry& me = s->meshes[q.mesh];
      const int d = me.m->d, dr = me.m->dr;
      if (!m0) m0 = me.m;
      if (!base.count(q.mesh)) {
        base[q.mesh] = buckets;
        buckets += order_keys(me.m);
      }
      BatchItem& bi = t.items_h[ni++];
      memset(&bi, 0, sizeof(bi));
      bi.m = me.m->view();
      bi.key_base = base[q.mesh];
      bi.pts = q.xs + tl.off * d;
      bi.n = tl.len;
      bi.start = total;
      bi.code = q.code + tl.off;
      bi.elem = q.elem + tl.off;
      bi.r = q.r + tl.off * dr;
      bi.dist2 = q.dist2 + tl.off;
      const bool last = q.stage == q.nstages - 1;
      if (q.kind == FP_REQ_REMAP) {
        bi.field = me.remap_field;
        bi.nc = me.remap_field ? me.nc_remap : 0;
        bi.fs = me.remap_fs;
        bi.fexp = me.remap_fexp;
      } else if (!last) {
        bi.field = me.vel;
        bi.nc = d;
        bi.fs = me.vel_fs;
        bi.fexp = me.vel_fexp;
      }
      bi.out = q.u + tl.off;
      bi.ld = q.n;
      total += tl.len;
      if (q.kind == FP_REQ_PARTICLE && !last) {
        AdvItem& a = t.adv_h[na++];
        a.x = q.x + tl.off * d;
        a.xs = q.xs + tl.off * d;
        a.u = q.u + tl.off;
        a.n = tl.len;
        a.ld = q.n;
        a.start = atotal;
        a.mode = (q.stage % 2 == 0) ? 0 : 1;
        a.c = (q.stage % 2 == 0) ? 0.5 * q.dt : q.dt;
        a.d = d;
        atotal += tl.len;
      }
    }
    launches.emplace_back(first, ni - first, total, qoff, kv.first, m0, buckets);
    qoff += total + 1;
  }
  if (qoff > t.queue_cap) return FP_ENOMEM;  // nothing launched; the caller fails t.tiles
  // from here on the tiles belong to this tick: a failure below still
  // completes through t.done, so no request memory is released while
  // kernels that were launched may use it
  for (const Tile& tl : t.tiles) {
    Request& q = *s->reqs[tl.id];
    q.next += tl.len;
    ++q.inflight;
  }
  t.busy = true;
  t.fail_rc = FP_OK;
  t.started = Clock::now();
  s->stats.ticks++;
  const int rc = enqueue_tick(s, t, launches, ni, na, atotal);
  if (rc != FP_OK) t.fail_rc = rc;
  if (cudaEventRecord(t.done, t.st) != cudaSuccess && t.fail_rc == FP_OK) t.fail_rc = FP_ELAUNCH;
  return rc;
}

int enqueue_tick(fp_server_s* s, TickSlot& t, const std::vector<TickLaunch>& launches, int ni, int na,
                 int64_t atotal) {
  FP_CUDA_TRY(cudaMemcpyAsync(t.items_d, t.items_h, sizeof(BatchItem) * ni, cudaMemcpyHostToDevice, t.st));
  if (na) FP_CUDA_TRY(cudaMemcpyAsync(t.adv_d, t.adv_h, sizeof(AdvItem) * na, cudaMemcpyHostToDevice, t.st));
  FP_CUDA_TRY(cudaEventRecord(t.fork_ev, t.st));
  int rc = FP_OK;
  bool used[kTickForks] = {};
  int64_t ooff = 0;  // next free int of the cell-order scratch
  for (size_t li = 0; li < launches.size() && rc == FP_OK; ++li) {
    const TickLaunch& L = launches[li];
    const int first = std::get<0>(L), cnt = std::get<1>(L);
    const int64_t total = std::get<2>(L), off = std::get<3>(L);
    const int N = std::get<0>(std::get<4>(L)), d = std::get<1>(std::get<4>(L)), dr = std::get<2>(std::get<4>(L));
    const fp_mesh_s* m0 = std::get<5>(L);
    const int64_t buckets = std::get<6>(L);
    const int f = (int)(li % kTickForks);
    cudaStream_t fs = t.fork[f];
    if (!used[f]) {
      if (cudaStreamWaitEvent(fs, t.fork_ev, 0) != cudaSuccess) {
        rc = FP_ELAUNCH;
        break;
      }
      used[f] = true;
    }
    rc = [&]() -> int {
      int* qq = t.queue + off;
      if (s->opts.precision == FP_MIXED) FP_CUDA_TRY(cudaMemsetAsync(qq + total, 0, sizeof(int), fs));
      // each shape has its own range of the order scratch (ranges 64-int aligned)
      int* order = nullptr;
      const int64_t need = (batch_cell_order_ints(total, buckets) + 63) / 64 * 64;
      if (total >= (1 << 14) && ooff + need <= t.order_cap) {
        FP_TRY(batch_cell_order(t.items_d + first, cnt, total, d, buckets, t.order + ooff, &order, fs));
        ooff += need;
      }
      FP_TRY(launch_batch_class(t.items_d + first, cnt, total, N, d, dr, m0->basis, s->opts.precision, 0, 5,
                                order, qq, qq + total, nullptr, fs));
      // FP_MIXED, quads, hexes and surfaces (fields split at creation): the
      // double-float contraction, in the find's point order where the tick
      // has one (the order changes no value: a request's result stays the
      // same alone and in any mix); else the FP64 one
      const bool df = s->opts.precision == FP_MIXED && dr >= 2;
      return dispatch_shape(N, d, dr, [&](auto Nc, auto Dc, auto DRc) -> int {
        constexpr int NN = decltype(Nc)::value, DR = decltype(DRc)::value;
        (void)Dc;
        if (df)
          k_eval_items_df<NN, DR><<<grid_for(total, 128, sm_count() * 16), 128, 0, fs>>>(t.items_d + first, cnt,
                                                                                       total, order, m0->basis);
        else
          k_serve_eval<NN, DR><<<grid_for(total, 128, sm_count() * 16), 128, 0, fs>>>(t.items_d + first, cnt, total,
                                                                                    m0->basis);
        return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ELAUNCH;
      });
    }();
  }
  // join every fork that took work, whatever happened, so the tick's event
  // (recorded on st by the caller) covers all of its kernels
  for (int f = 0; f < kTickForks; ++f) {
    if (!used[f]) continue;
    if (cudaEventRecord(t.join_ev[f], t.fork[f]) != cudaSuccess ||
        cudaStreamWaitEvent(t.st, t.join_ev[f], 0) != cudaSuccess) {
      // the join failed: wait for the fork on the host so that no kernel
      // outlives the tick
      cudaStreamSynchronize(t.fork[f]);
      if (rc == FP_OK) rc = FP_ELAUNCH;
    }
  }
  if (rc != FP_OK) return rc;
  if (na) {
    k_advance<<<grid_for(atotal, 256, sm_count() * 8), 256, 0, t.st>>>(t.adv_d, na, atotal);
    FP_CUDA_TRY(cudaGetLastError());
  }
  return FP_OK;
}

// Tick t finished (lock held): count its tiles; a request whose current
// stage is complete moves to the next stage or to its download.
void complete_tick(fp_server_s* s, TickSlot& t, int status) {
  for (const Tile& tl : t.tiles) {
    auto f = s->reqs.find(tl.id);
    if (f == s->reqs.end()) continue;
    Request& q = *f->second;
    --q.inflight;
    q.done += tl.len;
    s->served += tl.len;
    if (status != FP_OK && q.status == FP_OK) q.status = status;
    if (q.inflight > 0) continue;  // memory in use by the other tick
    if (q.status != FP_OK) {
      finish(s, q, q.status);
      continue;
    }
    if (q.done < q.n) continue;
    ++q.stage;
    q.next = q.done = 0;
    if (q.stage >= q.nstages) start_download(s, q);
  }
  t.tiles.clear();
  t.busy = false;
  t.timed_out = false;
}

void worker_loop(fp_server_s* s) {
  cudaSetDevice(s->device);
  const auto tick_limit = std::chrono::duration<double>(s->opts.tick_timeout_s > 0 ? s->opts.tick_timeout_s : 30.0);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    admit(s);
    bool progressed = false;
    // uploads and downloads that finished
    for (auto& kv : s->reqs) {
      Request& q = *kv.second;
      if (q.state == R_UPLOADING || q.state == R_DOWNLOADING) {
        const cudaError_t e = cudaEventQuery(q.ev);
        if (e == cudaErrorNotReady) continue;
        progressed = true;
        if (e != cudaSuccess) q.status = FP_ELAUNCH;
        if (q.state == R_UPLOADING && q.status == FP_OK) q.state = R_READY;
        else finish(s, q, FP_OK);
      }
    }
    // ticks that finished (bounded: a tick past the limit fails its requests)
    for (auto& t : s->slot) {
      if (!t.busy) continue;
      const cudaError_t e = cudaEventQuery(t.done);
      if (e == cudaErrorNotReady) {
        // past the limit: the requests fail, but their memory stays reserved
        // until the tick's kernels have finished with it
        if (!t.timed_out && Clock::now() - t.started > tick_limit) {
          t.timed_out = true;
          s->stats.timeouts++;
          for (const Tile& tl : t.tiles) s->reqs[tl.id]->status = FP_ETIMEDOUT;
        }
        continue;
      }
      complete_tick(s, t, e != cudaSuccess ? FP_ELAUNCH : t.fail_rc);
      progressed = true;
    }
    // launch new ticks on free slots
    for (auto& t : s->slot) {
      if (t.busy) continue;
      const int rc = launch_tick(s, t);
      if (rc < 0 && !t.busy) {
        // nothing was launched (no queue room): fail the requests it picked
        for (const Tile& tl : t.tiles) {
          Request& q = *s->reqs[tl.id];
          if (q.status == FP_OK) q.status = rc;
          if (q.inflight == 0 && q.state != R_DONE) finish(s, q, rc);
        }
        t.tiles.clear();
      } else if (t.busy) {
        progressed = true;
      }
    }
    // drop finished requests' bookkeeping once collected (kept for queries)
    if (!progressed) {
      bool busy = s->slot[0].busy || s->slot[1].busy || s->active > 0;
      if (busy) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(50));
        lk.lock();
      } else {
        s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
      }
    }
  }
}

// Waits, with the tick deadline, for the work the server queued on its own
// streams (not for anything else on the device): an event recorded on each
// stream, polled with a sleep.  Returns false if the deadline passed.
bool drain_server_streams(fp_server_s* s) {
  std::vector<cudaStream_t> streams;
  for (auto& t : s->slot) {
    if (t.st) streams.push_back(t.st);
    for (int f = 0; f < kTickForks; ++f)
      if (t.fork[f]) streams.push_back(t.fork[f]);
  }
  if (s->up) streams.push_back(s->up);
  if (s->down) streams.push_back(s->down);
  std::vector<cudaEvent_t> evs;
  for (cudaStream_t st : streams) {
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) continue;
    if (cudaEventRecord(ev, st) != cudaSuccess) {
      cudaEventDestroy(ev);
      continue;
    }
    evs.push_back(ev);
  }
  const double limit = s->opts.tick_timeout_s > 0 ? s->opts.tick_timeout_s : 30.0;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(limit));
  bool done = false;
  while (true) {
    done = true;
    for (cudaEvent_t ev : evs) done &= cudaEventQuery(ev) != cudaErrorNotReady;
    if (done || Clock::now() > deadline) break;
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
  for (cudaEvent_t ev : evs) cudaEventDestroy(ev);  // released once complete
  return done;
}

// Stops the scheduler, waits (bounded) for the server's streams and frees
// its resources.  If the wait runs out, the device and pinned buffers the
// kernels may still use are left allocated (leaked) and FP_ETIMEDOUT is
// returned, rather than blocking or freeing memory under a running kernel.
int destroy_server(fp_server_s* s) {
  if (s->worker.joinable()) {
    s->stop = true;
    s->cv_work.notify_all();
    s->worker.join();
  }
  if (!drain_server_streams(s)) {
    s->stats.timeouts++;
    return FP_ETIMEDOUT;
  }
  for (auto& t : s->slot) {
    if (t.st) cudaStreamDestroy(t.st);
    if (t.done) cudaEventDestroy(t.done);
    for (int f = 0; f < kTickForks; ++f) {
      if (t.fork[f]) cudaStreamDestroy(t.fork[f]);
      if (t.join_ev[f]) cudaEventDestroy(t.join_ev[f]);
    }
    if (t.fork_ev) cudaEventDestroy(t.fork_ev);
    cudaFreeHost(t.items_h);
    cudaFreeHost(t.adv_h);
    cudaFree(t.items_d);
    cudaFree(t.adv_d);
    cudaFree(t.queue);
    cudaFree(t.order);
  }
  for (auto& kv : s->reqs)
    if (kv.second->ev) cudaEventDestroy(kv.second->ev);
  if (s->up) cudaStreamDestroy(s->up);
  if (s->down) cudaStreamDestroy(s->down);
  cudaFree(s->arena.base);
  for (auto& me : s->meshes) {
    cudaFree(me.remap_fs);
    cudaFree(me.remap_fexp);
    cudaFree(me.vel_fs);
    cudaFree(me.vel_fexp);
  }
  return FP_OK;
}

}  // namespace
}  // namespace fp

extern "C" void fp_server_opts_default(fp_server_opts* o) {
  if (!o) return;
  o->mem_budget = (size_t)1 << 30;
  o->max_active = 64;
  o->precision = FP_MIXED;
  o->tick_timeout_s = 30.0;
  o->tick_points = (int64_t)1 << 19;
  o->policy = FP_SCHED_SLACK;
  o->slack_base = (double)((int64_t)1 << 20);
  o->slack_factor = 4.0;
}

extern "C" int fp_server_create(const fp_mesh* meshes, int nm, const double* const* remap_fields,
                                const int* nc_remap, const double* const* velocity,
                                const fp_server_opts* opts, fp_server* out) {
  using namespace fp;
  if (!out) return FP_EINVAL;
  *out = nullptr;
  if (!meshes || nm <= 0) return FP_EINVAL;
  fp_server_opts o;
  fp_server_opts_default(&o);
  if (opts) o = *opts;
  if (o.mem_budget < ((size_t)1 << 20) || o.max_active < 1 || (o.precision != FP_F64 && o.precision != FP_MIXED) ||
      o.tick_points < 1 || (o.policy != FP_SCHED_SRPT && o.policy != FP_SCHED_SLACK) ||
      !(o.slack_factor >= 0.0) || !(o.slack_base == o.slack_base))
    return FP_EINVAL;
  for (int i = 0; i < nm; ++i) {
    if (!meshes[i]) return FP_EINVAL;
    if (remap_fields && remap_fields[i] && (!nc_remap || nc_remap[i] < 1)) return FP_EINVAL;
  }
  auto* s = new fp_server_s();
  s->opts = o;
  memset(&s->stats, 0, sizeof(s->stats));
  cudaGetDevice(&s->device);
  for (int i = 0; i < nm; ++i)
    s->meshes.push_back({meshes[i], remap_fields ? remap_fields[i] : nullptr,
                         (remap_fields && remap_fields[i]) ? nc_remap[i] : 0, velocity ? velocity[i] : nullptr});
  s->max_items = o.max_active;
  s->tick_points = o.tick_points;
  // bytes per point >= 72, so the budget bounds the points in flight
  const int64_t qcap = (int64_t)(o.mem_budget / 72) + 2 * 64 + 16;
  int64_t all_buckets = 0;
  for (auto& me : s->meshes) all_buckets += order_keys(me.m);
  // one order range per shape: the single-range size plus, per shape, its
  // own scan's constant part and the 64-int alignment
  const int64_t ocap = batch_cell_order_ints(std::min(qcap, o.tick_points), all_buckets) +
                       (int64_t)(s->meshes.size() + 1) * 256;
  int rc = FP_OK;
  if (!s->arena.init(o.mem_budget)) rc = FP_ENOMEM;
  if (rc == FP_OK && o.precision == FP_MIXED) {
    // the double-float copies of the resident fields (quads, hexes, surfaces)
    for (auto& me : s->meshes) {
      if (rc != FP_OK || me.m->dr < 2) continue;
      const int64_t per = me.m->NE * (int64_t)me.m->ne;
      if (me.remap_field) rc = split_resident(me.remap_field, me.nc_remap, per, &me.remap_fs, &me.remap_fexp, 0);
      if (rc == FP_OK && me.vel) rc = split_resident(me.vel, me.m->d, per, &me.vel_fs, &me.vel_fexp, 0);
    }
    if (rc == FP_OK && cudaStreamSynchronize(0) != cudaSuccess) rc = FP_ELAUNCH;
  }
  if (rc == FP_OK && (cudaStreamCreateWithFlags(&s->up, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaStreamCreateWithFlags(&s->down, cudaStreamNonBlocking) != cudaSuccess))
    rc = FP_ELAUNCH;
  for (auto& t : s->slot) {
    if (rc != FP_OK) break;
    t.queue_cap = qcap;
    t.order_cap = ocap;
    bool forks_ok = cudaEventCreateWithFlags(&t.fork_ev, cudaEventDisableTiming) == cudaSuccess;
    for (int f = 0; f < kTickForks && forks_ok; ++f)
      forks_ok = cudaStreamCreateWithFlags(&t.fork[f], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&t.join_ev[f], cudaEventDisableTiming) == cudaSuccess;
    if (!forks_ok || cudaStreamCreateWithFlags(&t.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&t.items_h, sizeof(BatchItem) * s->max_items) != cudaSuccess ||
        cudaMallocHost(&t.adv_h, sizeof(AdvItem) * s->max_items) != cudaSuccess)
      rc = FP_ELAUNCH;
    else if (cudaMalloc(&t.items_d, sizeof(BatchItem) * s->max_items) != cudaSuccess ||
             cudaMalloc(&t.adv_d, sizeof(AdvItem) * s->max_items) != cudaSuccess ||
             cudaMalloc(&t.queue, sizeof(int) * qcap) != cudaSuccess ||
             cudaMalloc(&t.order, sizeof(int) * ocap) != cudaSuccess)
      rc = FP_ENOMEM;
  }
  if (rc != FP_OK) {
    destroy_server(s);
    delete s;
    return rc;
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return FP_OK;
}

extern "C" int fp_server_submit(fp_server s, int mesh, int kind, const double* pts_host, int64_t n,
                                int rk_steps, double dt, int32_t* code_host, int32_t* elem_host,
                                double* r_host, double* dist2_host, double* out_host, int64_t* req_id) {
  using namespace fp;
  if (!s || !req_id || mesh < 0 || mesh >= (int)s->meshes.size() || n <= 0 || n > INT32_MAX || !pts_host)
    return FP_EINVAL;
  if (kind != FP_REQ_REMAP && kind != FP_REQ_PARTICLE) return FP_EINVAL;
  const MeshEntry& me = s->meshes[mesh];
  if (kind == FP_REQ_PARTICLE && (!me.vel || rk_steps < 1 || !(dt == dt))) return FP_EINVAL;
  const size_t bytes = request_bytes(s, mesh, kind, n);
  if (bytes > s->arena.size) return FP_ENOMEM;  // can never be admitted
  auto q = std::make_unique<Request>();
  q->mesh = mesh;
  q->kind = kind;
  q->n = n;
  q->rk_steps = rk_steps;
  q->dt = dt;
  q->pts_h = pts_host;
  q->code_h = code_host;
  q->elem_h = elem_host;
  q->r_h = r_host;
  q->dist2_h = dist2_host;
  q->out_h = out_host;
  q->bytes = bytes;
  q->nstages = kind == FP_REQ_REMAP ? 1 : 2 * rk_steps + 1;
  q->t_submit = Clock::now();
  if (cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming) != cudaSuccess) return FP_ELAUNCH;
  std::lock_guard<std::mutex> lk(s->mu);
  q->id = s->next_id++;
  q->born = s->served;
  *req_id = q->id;
  s->queued.push_back(q->id);
  s->reqs[q->id] = std::move(q);
  s->stats.submitted++;
  s->cv_work.notify_all();
  return FP_OK;
}

extern "C" int fp_server_poll(fp_server s, int64_t id, int* done, int* status) {
  if (!s || !done) return FP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto f = s->reqs.find(id);
  if (f == s->reqs.end()) return FP_EINVAL;
  *done = f->second->state == fp::R_DONE;
  if (status) *status = *done ? f->second->status : FP_OK;
  return FP_OK;
}

extern "C" int fp_server_wait(fp_server s, int64_t id, double timeout_s) {
  if (!s) return FP_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto f = s->reqs.find(id);
  if (f == s->reqs.end()) return FP_EINVAL;
  fp::Request* q = f->second.get();
  // clamp so that the deadline arithmetic cannot overflow (about 115 days)
  const double t = timeout_s > 1e7 ? 1e7 : (timeout_s > 0.0 ? timeout_s : 0.0);
  const auto deadline = fp::Clock::now() + std::chrono::duration_cast<fp::Clock::duration>(
                                                 std::chrono::duration<double>(t));
  while (q->state != fp::R_DONE) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && q->state != fp::R_DONE)
      return FP_ETIMEDOUT;
  }
  return q->status;
}

extern "C" int fp_server_cancel(fp_server s, int64_t id) {
  if (!s) return FP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto f = s->reqs.find(id);
  if (f == s->reqs.end()) return FP_EINVAL;
  fp::Request& q = *f->second;
  if (q.state != fp::R_QUEUED) return FP_EBUSY;
  s->queued.erase(std::find(s->queued.begin(), s->queued.end(), id));
  q.state = fp::R_DONE;
  q.status = FP_ECANCELED;
  q.t_done = fp::Clock::now();
  s->stats.cancelled++;
  s->cv_done.notify_all();
  return FP_OK;
}

extern "C" int fp_server_timing(fp_server s, int64_t id, double* queued_s, double* total_s) {
  if (!s) return FP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto f = s->reqs.find(id);
  if (f == s->reqs.end() || f->second->state != fp::R_DONE) return FP_EINVAL;
  const fp::Request& q = *f->second;
  using sec = std::chrono::duration<double>;
  if (queued_s) *queued_s = (q.t_admit.time_since_epoch().count() ? sec(q.t_admit - q.t_submit).count() : 0.0);
  if (total_s) *total_s = sec(q.t_done - q.t_submit).count();
  return FP_OK;
}

extern "C" int fp_server_release(fp_server s, int64_t id) {
  if (!s) return FP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto f = s->reqs.find(id);
  if (f == s->reqs.end()) return FP_EINVAL;
  if (f->second->state != fp::R_DONE) return FP_EBUSY;
  if (f->second->ev) cudaEventDestroy(f->second->ev);
  s->reqs.erase(f);
  return FP_OK;
}

extern "C" int fp_server_get_stats(fp_server s, fp_server_stats* out) {
  if (!s || !out) return FP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->active = s->active;
  out->queued = (int64_t)s->queued.size();
  return FP_OK;
}

extern "C" int fp_server_destroy(fp_server s) {
  if (!s) return FP_EINVAL;
  const int rc = fp::destroy_server(s);
  delete s;
  return rc;
}
