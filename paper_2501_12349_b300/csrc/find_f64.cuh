// The FP64 find kernel (Sec. 3.2), shared by the FP64 path and by the mixed
// path, which runs it on the points its FP32 phase could not settle.
//
// On this GPU the FP64 FMA pipe (about 1.2 TFLOP/s, 1/62 of FP32) bounds the
// kernel, and a warp instruction costs the same FP64 issue time whether 1 or
// 32 lanes are active.  So:
//  * lanes refill themselves: each lane walks its own sequence of
//    (point, candidate, Newton iteration) states and pulls the next point
//    from a per-CTA counter, so no lane idles while its warp has work;
//  * each round of the loop has one warp-uniform site where every busy lane
//    evaluates x(r) and G(r) of its current element at a trial point (the
//    sum-factorised contraction that is most of the FP64 work), inlined once;
//  * a candidate starts at its closest GLL node, where x is the node itself
//    and G takes N terms per direction: the lanes that start one do it right
//    after the warp's node search (the warp sharing the N-term sums of all
//    of them) and take their first Newton step in a second bookkeeping
//    pass, so their first full evaluation is already a trial step;
//  * the box tests and the closest-node search, done by whichever lanes
//    start a candidate, run in FP32 with rigorous rounding margins and fall
//    back to FP64 only inside the margin, so every decision equals the FP64
//    one while the divergent part costs almost no FP64 issue slots.
#pragma once
#include "beta_warp.cuh"
#include "coop_eval.cuh"
#include "find_common.cuh"

namespace fp {

enum : int { M_IDLE = 0, M_SCAN = 1, M_START = 2, M_NEWTON = 3, M_RESTORE = 4, M_DONE = 5 };
enum : int { E_TRIAL = 1, E_RESTORE = 2 };

// Group mode (kGroup): for launches whose time is the dependency chain of
// their slowest points rather than their total work (the few points a mixed
// launch hands over), a warp takes 8 points at a time and gives each 4
// lanes: slot k = 0, 1, 2 searches the point's k-th candidate element
// alone, slot 3 the 4th and any later ones in order, so a point's
// candidates run side by side instead of one after another.  When the whole
// warp is done the slots merge under the selection rule of Sec. 3.2 (the
// first INTERIOR in candidate order, else the smallest distance, ties to
// the earlier candidate), which gives the one-lane result exactly.
constexpr int kGroupPoints = 8;

// Group mode: the 4 slots of each point merge into its first lane, which
// writes the point's result.
template <int DR, class Work>
__device__ __forceinline__ void group_merge(const Work& w, bool valid, int slot, int item, int64_t pi, int bcode,
                                            int be, const double (&br)[DR], double bd) {
  constexpr unsigned kAll = 0xffffffffu;
  const int lead = (threadIdx.x & 31) & ~3;
  int sc = bcode, se = be;
  double sd = bd, sr[DR];
#pragma unroll
  for (int j = 0; j < DR; ++j) sr[j] = br[j];
  bool fin = sc == FP_INTERIOR;
#pragma unroll
  for (int k = 1; k < 4; ++k) {
    const int oc = __shfl_sync(kAll, bcode, lead + k);
    const int oe = __shfl_sync(kAll, be, lead + k);
    const double od = __shfl_sync(kAll, bd, lead + k);
    double orr[DR];
#pragma unroll
    for (int j = 0; j < DR; ++j) orr[j] = __shfl_sync(kAll, br[j], lead + k);
    const bool take = !fin && (oc == FP_INTERIOR || od < sd);
    fin |= take && oc == FP_INTERIOR;
    if (take) {
      sc = oc;
      se = oe;
      sd = od;
#pragma unroll
      for (int j = 0; j < DR; ++j) sr[j] = orr[j];
    }
  }
  if (valid && slot == 0) w.write(item, pi, sc, se, sr, sd);
}

// Group mode: the warp takes the next kGroupPoints points of its CTA's
// chunks (lane l gets point l / 4, slot l % 4) and sets up their cells; a
// lane without a point waits (M_IDLE), and every lane stops (M_DONE) once
// the chunks are used up.
template <int D, int DR, class Work>
__device__ __forceinline__ void group_fetch(const Work& w, unsigned long long& s_next, int clog2, int64_t nchunks,
                                            int64_t n, const DevMesh*& mp, int& item, int64_t& pi, double (&xs)[D],
                                            float (&x32)[D], int& q, int& qend, int& mode, bool& valid) {
  const int lane = threadIdx.x & 31;
  unsigned long long s0 = 0;
  if (lane == 0) s0 = atomicAdd(&s_next, (unsigned long long)kGroupPoints);
  s0 = __shfl_sync(0xffffffffu, s0, 0);
  const unsigned long long s = s0 + (unsigned long long)(lane >> 2);
  const int64_t chunk = (int64_t)(s0 >> clog2) * w.ctas() + w.cta();
  valid = false;
  if (chunk >= nchunks) {
    mode = M_DONE;
    return;
  }
  const int64_t g = (chunk << clog2) + (int64_t)(s & ((1u << clog2) - 1));
  mode = M_IDLE;
  if (g >= n) return;
  valid = true;
  w.locate(g, mp, item, pi);
  w.load(item, pi, xs);
#pragma unroll
  for (int c = 0; c < D; ++c) x32[c] = (float)xs[c];
  const int64_t cell = point_cell<D>(*mp, xs);
  if (cell < 0) return;
  q = __ldg(mp->cell_start + cell);
  qend = __ldg(mp->cell_start + cell + 1);
  mode = M_SCAN;
}

// Shared memory of one CTA of the FP64 lane loop: the t-basis slabs, the
// beta term's per-thread entries and per-warp scratch, the node start's
// entries of G and table of starting lanes, the GLL differentiation matrix
// and the CTA's point counter.
template <int N, int D, int DR>
struct F64Shared {
  double slab[DR == 3 ? 2 * N * kFindThreads : 1];
  double hs[beta_entries<DR>() * kFindThreads];
  double bscr[(kFindThreads / 32) * kBetaScratch];
  double sg[D * DR * kFindThreads];  // node start: G of the starting lanes
  double dn[N * N];
  int sl[kFindThreads];              // node start: starting lanes by rank
  unsigned long long next;
};

// The FP64 lane loop over a source of work (SingleWork, BatchWork or a tile
// of one); all meshes of one call share N, D, DR and so the basis table B.
template <int N, int D, int DR, class Work, bool kGroup = false>
__device__ __forceinline__ void find_f64_loop(const Work& w, const BasisTab& B, unsigned long long* stats,
                                              F64Shared<N, D, DR>& sh) {
  constexpr int NN = ipow(N, DR);
  double* const s_hs = sh.hs;
  double* const s_dn = sh.dn;
  unsigned long long& s_next = sh.next;
  const TSlots<N, double> ts{sh.slab};
  double* const wscr = sh.bscr + (threadIdx.x >> 5) * kBetaScratch;
  if (threadIdx.x == 0) {
    s_next = 0;
#pragma unroll
    for (int i = 0; i < N * N; ++i) s_dn[i] = B.dn[i];
  }
  __syncthreads();
  Counters cnt;
  const int64_t n = w.n;
  const int clog2 = w.clog2;
  const int64_t nchunks = (n + (1 << clog2) - 1) >> clog2;
  const DevMesh* mp = w.first();
  int item = 0;
  int mode = M_IDLE, etype = E_TRIAL;
  int64_t pi = 0;
  double xs[D];
  float x32[D];
  int q = 0, qend = 0, e = -1, l = 0;
  int bcode = FP_NOT_FOUND, be = -1;
  double br[DR], bd = INFINITY;
  double r[DR], rn[DR], dx[D], G[D * DR];
  double alpha = 1.0, F = 0.0, pred = 0.0, xscale = 1.0;
  bool clipped = false;
  unsigned guard = 0;
  [[maybe_unused]] const int slot = threadIdx.x & 3;  // group mode: the lane's candidate slot
  [[maybe_unused]] int skip = 0;                      // group mode: candidates still to pass over
  [[maybe_unused]] bool valid = false;                // group mode: the lane holds a point
#pragma unroll
  for (int j = 0; j < DR; ++j) br[j] = r[j] = rn[j] = 0.0;

  while (true) {
    if constexpr (kGroup) {
      // the group is done when every lane waits (M_IDLE) or has run out
      if (__all_sync(0xffffffffu, mode == M_IDLE || mode == M_DONE)) {
        group_merge<DR>(w, valid, slot, item, pi, bcode, be, br, bd);
        group_fetch<D, DR>(w, s_next, clog2, nchunks, n, mp, item, pi, xs, x32, q, qend, mode, valid);
        skip = slot;
        bcode = FP_NOT_FOUND;
        be = -1;
        bd = INFINITY;
#pragma unroll
        for (int j = 0; j < DR; ++j) br[j] = 0.0;
      }
    }
    bool need = false, finished = false;
    for (int pass = 0;; ++pass) {
      // ---- per-lane bookkeeping until this lane needs an evaluation or a start
      while (mode != M_DONE && mode != M_START && !need && !(kGroup && mode == M_IDLE)) {
        if (++guard > (1u << 26)) {
          record_status(mp->status, FP_DEV_SPIN_CAP);
          mode = M_DONE;
          break;
        }
        if (mode == M_IDLE) {
          const unsigned long long s = atomicAdd(&s_next, 1ull);
          const int64_t chunk = (int64_t)(s >> clog2) * w.ctas() + w.cta();
          if (chunk >= nchunks) {
            mode = M_DONE;
            break;
          }
          const int64_t g = (chunk << clog2) + (int64_t)(s & ((1u << clog2) - 1));
          if (g >= n) continue;
          w.locate(g, mp, item, pi);
          w.load(item, pi, xs);
#pragma unroll
          for (int c = 0; c < D; ++c) x32[c] = (float)xs[c];
          bcode = FP_NOT_FOUND;
          be = -1;
          bd = INFINITY;
#pragma unroll
          for (int j = 0; j < DR; ++j) br[j] = 0.0;
          const int64_t cell = point_cell<D>(*mp, xs);
          if (cell < 0) {
            w.write(item, pi, bcode, be, br, bd);
            continue;
          }
          q = __ldg(mp->cell_start + cell);
          qend = __ldg(mp->cell_start + cell + 1);
          mode = M_SCAN;
        }
        if (mode == M_SCAN) {
          e = next_candidate<D>(*mp, xs, x32, q, qend, cnt);
          if (e < 0) {
            if constexpr (!kGroup) w.write(item, pi, bcode, be, br, bd);
            mode = M_IDLE;
            continue;
          }
          if constexpr (kGroup) {
            if (skip > 0) {  // an earlier slot's candidate
              --skip;
              continue;
            }
          }
          ++cnt.v[0];
          xscale = aabb_scale<D>(*mp, e);
          mode = M_START;  // the start r0, the closest node, is found by the warp below
          break;
        }
        if (mode == M_RESTORE) {
          etype = E_RESTORE;
          need = true;
          break;
        }
        // mode == M_NEWTON: one step of Sec. 3.2.1 from (r, dx, G, F, alpha)
        bool done = false;
        if (l >= mp->max_iter) {
          done = true;
        } else {
          const bool beta = (l > 0) && at_bound<DR>(r);
          double HS[DR][DR] = {};
          if (beta) {
            beta_load<DR, double>(s_hs, HS);  // computed by the warp after the last evaluation
            ++cnt.v[3];
          }
          double ds[DR];
          bool used_beta;
          const double mx = newton_step<D, DR>(G, dx, r, alpha, beta, HS, rn, ds, clipped, used_beta);
          bool stop = below_nonneg(mx, mp->newton_tol);
          if (stop) F = model_dist2<D, DR>(G, dx, ds);  // dist2 from the linear model at r
          if constexpr (DR == D) {
            // volumes: the step before the last one can be certified
            if (!stop && !beta && !clipped && below_nonneg(mx, kCertMaxStep)) {
              stop = certified_stop<D>(G, dx, ds, rn, mx, __ldg(mp->curv + e), xscale, F);
              if (stop) ++cnt.v[4];
            }
          }
          if (stop) {  // the step is taken
#pragma unroll
            for (int j = 0; j < DR; ++j) r[j] = rn[j];
            ++cnt.v[1];
            done = true;
          } else {
            pred = predicted_decrease<D, DR>(G, dx, ds, used_beta, HS);
            if (!is_pos(pred)) {
              done = true;
            } else {
              ++cnt.v[1];
              etype = E_TRIAL;
              need = true;
            }
          }
        }
        if (done) {
          bool inside = true;
#pragma unroll
          for (int j = 0; j < DR; ++j) inside &= below_unit(r[j]);
          if (DR < D) inside &= below_nonneg(F, mp->dist_tol);
          if (inside || below_nonneg(F, bd)) {
            bcode = inside ? FP_INTERIOR : FP_BORDER;
            be = e;
            bd = F;
#pragma unroll
            for (int j = 0; j < DR; ++j) br[j] = r[j];
          }
          if constexpr (kGroup) {
            mode = (inside || slot < 3) ? M_IDLE : M_SCAN;
          } else if (inside) {
            w.write(item, pi, bcode, be, br, bd);
            mode = M_IDLE;
          } else {
            mode = M_SCAN;
          }
        }
      }
      // a lane that starts another candidate in the second pass waits for
      // the next round's node search
      if (pass == 1) break;
      if (__all_sync(0xffffffffu, mode == M_DONE)) {
        finished = true;
        break;
      }
      // ---- warp-uniform closest-node search, then the start at that node
      const bool start = mode == M_START;
      if (!__any_sync(0xffffffffu, start)) break;
      float xr[D];
      if (start) rel_point<D>(*mp, e, xs, xr);
      int nb = 0;
      closest_node_warp<N, D, DR>(start, *mp, e, xs, xr, nb);
      double xv[D];
      node_start_warp<N, D, DR>(start, *mp, e, nb, s_dn, sh.sg, sh.sl, xv, G);
      if (start) {
        node_coords<N, DR>(B, nb, r);
        F = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          dx[c] = xs[c] - xv[c];
          F += dx[c] * dx[c];
        }
        alpha = 1.0;
        l = 0;
        mode = M_NEWTON;
      }
    }
    if (finished) break;
    // ---- warp-uniform evaluation of x(r) and G(r) -------------------------
    // (hexes: with at most kCoopLanes lanes needing it, the whole warp
    // evaluates for each of them in turn, bit-identically; see coop_eval.cuh)
    bool coop = false;
    if constexpr (DR == 3) coop = __popc(__ballot_sync(0xffffffffu, need)) <= kCoopLanes;
    double xv[D];
    if (coop) {
      if constexpr (DR == 3) {
        double re[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) re[j] = (etype == E_TRIAL) ? rn[j] : r[j];
        coop_eval_hex<N, D>(need, mp->coords + (int64_t)e * NN, mp->cstride, B, re, xv, G);
      }
    }
    if (need) {
      double re[DR];
#pragma unroll
      for (int j = 0; j < DR; ++j) re[j] = (etype == E_TRIAL) ? rn[j] : r[j];
      if (etype == E_TRIAL) ++cnt.v[7];
      if (!coop) eval_xG<N, D, DR, true, double>(mp->coords + (int64_t)e * NN, mp->cstride, B, re, ts, xv, G);
      double Fn = 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        dx[c] = xs[c] - xv[c];
        Fn += dx[c] * dx[c];
      }
      if (etype == E_TRIAL) {
        ++l;
        if (trial_accepts(F, Fn, pred, clipped, xscale, alpha)) {
#pragma unroll
          for (int j = 0; j < DR; ++j) r[j] = rn[j];
          F = Fn;
          mode = M_NEWTON;
        } else {
          ++cnt.v[2];
          mode = M_RESTORE;  // dx and G now belong to rn: re-evaluate at r
        }
      } else {
        F = Fn;
        mode = M_NEWTON;
      }
    }
    // ---- warp-uniform beta term for the next Newton step -----------------
    {
      const bool want = need && mode == M_NEWTON && l > 0 && at_bound<DR>(r);
      const BetaReq bq = beta_request<N, D, DR, double>(want, r, dx, G);
      if (__any_sync(0xffffffffu, bq.kind != BETA_NONE))
        beta_warp<N, D, DR, double>(bq, mp->coords + (int64_t)e * NN, mp->cstride, r, dx, B, wscr, s_hs);
    }
  }
  cnt.flush(stats);
}

template <int N, int D, int DR>
__global__ void __launch_bounds__(kFindThreads, f64_ctas(N))
    k_find_f64(const __grid_constant__ DevMesh m, const BasisTab B, const double* __restrict__ pts,
               const int* __restrict__ pidx, int64_t n, const int* __restrict__ n_dev,
               int* __restrict__ code, int* __restrict__ elem, double* __restrict__ rout,
               double* __restrict__ dist2, int clog2, unsigned long long* stats) {
  const SingleWork<D, DR> w{&m, pts, pidx, n_dev ? (int64_t)*n_dev : n, code, elem, rout, dist2, clog2};
  __shared__ F64Shared<N, D, DR> sh;
  find_f64_loop<N, D, DR>(w, B, stats, sh);
}

// Every item of a batch (one element shape) in one persistent launch; gidx /
// n_dev optionally restrict it to a device-produced list of global indices.
template <int N, int D, int DR>
__global__ void __launch_bounds__(kFindThreads, f64_ctas(N))
    k_find_f64_batch(const BatchItem* __restrict__ items, int nitems, int64_t total,
                     const int* __restrict__ gidx, const int* __restrict__ n_dev, const BasisTab B,
                     int clog2, unsigned long long* stats) {
  const BatchWork<D, DR> w{items, nitems, gidx, n_dev ? (int64_t)*n_dev : total, clog2};
  __shared__ F64Shared<N, D, DR> sh;
  find_f64_loop<N, D, DR>(w, B, stats, sh);
}

// Group mode (see find_f64_loop) over one mesh's points or a batch's, for
// the points a mixed launch hands over.
template <int N, int D, int DR>
__global__ void __launch_bounds__(kFindThreads, f64_ctas(N))
    k_find_f64_group(const __grid_constant__ DevMesh m, const BasisTab B, const double* __restrict__ pts,
                     const int* __restrict__ pidx, int64_t n, const int* __restrict__ n_dev,
                     int* __restrict__ code, int* __restrict__ elem, double* __restrict__ rout,
                     double* __restrict__ dist2, unsigned long long* stats) {
  const SingleWork<D, DR> w{&m, pts, pidx, n_dev ? (int64_t)*n_dev : n, code, elem, rout, dist2, 5};
  __shared__ F64Shared<N, D, DR> sh;
  find_f64_loop<N, D, DR, SingleWork<D, DR>, true>(w, B, stats, sh);
}

template <int N, int D, int DR>
__global__ void __launch_bounds__(kFindThreads, f64_ctas(N))
    k_find_f64_group_batch(const BatchItem* __restrict__ items, int nitems, int64_t total,
                           const int* __restrict__ gidx, const int* __restrict__ n_dev, const BasisTab B,
                           unsigned long long* stats) {
  const BatchWork<D, DR> w{items, nitems, gidx, n_dev ? (int64_t)*n_dev : total, 5};
  __shared__ F64Shared<N, D, DR> sh;
  find_f64_loop<N, D, DR, BatchWork<D, DR>, true>(w, B, stats, sh);
}

}  // namespace fp
