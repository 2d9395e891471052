// The FP64 find kernel (Sec. 3.2), shared by the FP64 path and by the mixed
// path, which runs it on the points its FP32 phase could not settle.
//
// On this GPU the FP64 FMA pipe (about 1.1 TFLOP/s, 1/62 of FP32) bounds the
// kernel, and a warp instruction costs the same FP64 issue time whether 1 or
// 32 lanes are active.  So:
//  * lanes refill themselves: each lane walks its own sequence of
//    (point, candidate, Newton iteration) states and pulls the next point
//    from a per-CTA counter, so no lane idles while its warp has work;
//  * each round of the loop has one warp-uniform site where every busy lane
//    evaluates x(r) and G(r) of its current element (the sum-factorised
//    contraction that is most of the FP64 work), inlined once;
//  * the box tests and the closest-node search, done by whichever lanes
//    start a candidate, run in FP32 with rigorous rounding margins and fall
//    back to FP64 only inside the margin, so every decision equals the FP64
//    one while the divergent part costs almost no FP64 issue slots.
#pragma once
#include "find_common.cuh"

namespace fp {

enum : int { M_IDLE = 0, M_SCAN = 1, M_NEWTON = 2, M_RESTORE = 3, M_DONE = 4 };
enum : int { E_INIT = 1, E_TRIAL = 2, E_RESTORE = 3 };

template <int N, int D, int DR>
__global__ void __launch_bounds__(kFindThreads, 2)
    k_find_f64(const DevMesh m, const BasisTab B, const double* __restrict__ pts,
               const int* __restrict__ pidx, int64_t n, const int* __restrict__ n_dev,
               int* __restrict__ code,
               int* __restrict__ elem, double* __restrict__ rout, double* __restrict__ dist2,
               unsigned long long* stats) {
  constexpr int NN = (DR == 3) ? N * N * N : N * N;
  __shared__ double s_slab[DR == 3 ? 3 * N * kFindThreads : 1];
  const TSlots<N, double> ts{s_slab};
  __shared__ unsigned long long s_next;
  if (threadIdx.x == 0) s_next = 0;
  __syncthreads();
  Counters cnt;
  if (n_dev) n = *n_dev;  // a queue length produced on the device
  const int64_t nchunks = (n + 31) / 32;
  int mode = M_IDLE, etype = E_INIT;
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
#pragma unroll
  for (int j = 0; j < DR; ++j) br[j] = r[j] = rn[j] = 0.0;

  while (true) {
    bool need = false;
    // ---- per-lane bookkeeping until this lane needs one evaluation --------
    while (mode != M_DONE && !need) {
      if (++guard > (1u << 26)) {
        record_status(m.status, FP_DEV_SPIN_CAP);
        mode = M_DONE;
        break;
      }
      if (mode == M_IDLE) {
        const unsigned long long s = atomicAdd(&s_next, 1ull);
        const int64_t chunk = (int64_t)(s >> 5) * gridDim.x + blockIdx.x;
        if (chunk >= nchunks) {
          mode = M_DONE;
          break;
        }
        const int64_t p = chunk * 32 + (int64_t)(s & 31);
        if (p >= n) continue;
        pi = pidx ? (int64_t)__ldg(pidx + p) : p;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          xs[c] = __ldg(pts + pi * D + c);
          x32[c] = (float)xs[c];
        }
        bcode = FP_NOT_FOUND;
        be = -1;
        bd = INFINITY;
#pragma unroll
        for (int j = 0; j < DR; ++j) br[j] = 0.0;
        const int64_t cell = point_cell<D>(m, xs);
        if (cell < 0) {
          write_result<DR>(pi, bcode, be, br, bd, code, elem, rout, dist2);
          continue;
        }
        q = __ldg(m.cell_start + cell);
        qend = __ldg(m.cell_start + cell + 1);
        mode = M_SCAN;
      }
      if (mode == M_SCAN) {
        e = next_candidate<D>(m, xs, x32, q, qend, cnt);
        if (e < 0) {
          write_result<DR>(pi, bcode, be, br, bd, code, elem, rout, dist2);
          mode = M_IDLE;
          continue;
        }
        ++cnt.v[0];
        xscale = aabb_scale<D>(m, e);
        float xr[D];
        rel_point<D>(m, e, xs, xr);
        const int nb = closest_node<N, D, DR>(m, e, xs, xr);
        node_coords<N, DR>(B, nb, r);
        etype = E_INIT;
        need = true;
        break;
      }
      if (mode == M_RESTORE) {
        etype = E_RESTORE;
        need = true;
        break;
      }
      // mode == M_NEWTON: one step of Sec. 3.2.1 from (r, dx, G, F, alpha)
      bool done = false;
      if (l >= m.max_iter) {
        done = true;
      } else {
        const bool beta = (l > 0) && at_bound<DR>(r);
        double HS[DR][DR];
        if (beta) {
          hess_term<N, D, DR, double>(m.coords + (int64_t)e * NN, m.cstride, B, r, dx, ts, HS);
        }
        double ds[DR];
        bool used_beta;
        const double mx = newton_step<D, DR>(G, dx, r, alpha, beta, HS, rn, ds, clipped, used_beta);
        if (mx < m.newton_tol) {
          // the last step is taken; dist2 from the linear model at r
          F = model_dist2<D, DR>(G, dx, ds);
#pragma unroll
          for (int j = 0; j < DR; ++j) r[j] = rn[j];
          ++cnt.v[1];
          done = true;
        } else {
          pred = predicted_decrease<D, DR>(G, dx, ds, used_beta, HS);
          if (!(pred > 0.0)) {
            done = true;
          } else {
            ++cnt.v[1];
            if (beta) ++cnt.v[3];
            etype = E_TRIAL;
            need = true;
          }
        }
      }
      if (done) {
        bool inside = true;
#pragma unroll
        for (int j = 0; j < DR; ++j) inside &= fabs(r[j]) < 1.0;
        if (DR < D) inside &= F < m.dist_tol;
        if (inside || F < bd) {
          bcode = inside ? FP_INTERIOR : FP_BORDER;
          be = e;
          bd = F;
#pragma unroll
          for (int j = 0; j < DR; ++j) br[j] = r[j];
        }
        if (inside) {
          write_result<DR>(pi, bcode, be, br, bd, code, elem, rout, dist2);
          mode = M_IDLE;
        } else {
          mode = M_SCAN;
        }
      }
    }
    if (__all_sync(0xffffffffu, mode == M_DONE)) break;
    // ---- warp-uniform evaluation of x(r) and G(r) -------------------------
    if (need) {
      double re[DR];
#pragma unroll
      for (int j = 0; j < DR; ++j) re[j] = (etype == E_TRIAL) ? rn[j] : r[j];
      double xv[D];
      eval_xG<N, D, DR, true, double>(m.coords + (int64_t)e * NN, m.cstride, B, re, ts, xv, G);
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
        if (etype == E_INIT) {
          alpha = 1.0;
          l = 0;
        }
        F = Fn;
        mode = M_NEWTON;
      }
    }
  }
  cnt.flush(stats);
}

}  // namespace fp
