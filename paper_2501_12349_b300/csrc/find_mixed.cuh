// Mixed-precision find (FP_MIXED): FP32 box filter and early Newton
// steps, FP64 final steps, residual check and ill-conditioned solves.
//
// Kernel k_find_mixed, per point (lanes refill as in the FP64 kernel):
//  1. Psi_L cell in FP64; candidates from the certified FP32 box tests
//     (decisions equal the FP64 ones; inside the margin the FP64 test runs).
//  2. Per candidate, trust-region Newton of Sec. 3.2.1 in FP32 on the
//     element's FP32 coordinates taken relative to its reference point
//     (values O(h), so the FP32 Jacobian keeps ~1e-7 relative accuracy).
//  3. A candidate whose FP32 iteration converged strictly inside the element
//     is parked for FP64 refinement: x(r) in FP64, the Gauss-Newton step
//     solved with the FP32 Jacobian at the converged iterate (volumes) or
//     the FP64 one (surfaces and lines, whose converged residual is not
//     zero), repeated until the step is below the Newton tolerance.  For
//     volumes the first correction stands when the step after it is
//     estimated far below that tolerance (certified), so most points take
//     one FP64 evaluation.  Parked lanes wait until most of their warp is
//     parked, so the FP64 work runs with nearly full warps.
//  4. A candidate the FP32 iteration leaves clearly outside (on the boundary
//     with a distance far above FP32 rounding) is BORDER, as FP64 would find;
//     the search continues with the next candidate.
//  5. Anything else — a point with only BORDER candidates (its answer is the
//     closest BORDER candidate, needing FP64 distances), a refinement that
//     leaves the element, an ill-conditioned Jacobian, an FP32 iteration at
//     its rounding floor near a face — goes to a queue in scratch memory, and
//     the FP64 kernel then runs the full FP64 path on the queued points (in
//     group mode up to kGroupMaxPoints points per launch, see find_f64.cuh).
// Points with no candidate are NOT_FOUND straight away.
#pragma once
#include "find_f64.cuh"

namespace fp {
namespace {

enum : int { X_IDLE = 0, X_SCAN = 1, X_NEWTON = 2, X_RESTORE = 3, X_PARK = 4, X_DONE = 5, X_CONV = 6 };
enum : int { X_INIT = 1, X_TRIAL = 2, X_REST = 3, X_FINAL = 4 };

constexpr float kTol32 = 1e-4f;    // FP32 phase: stop when |dr|_inf < kTol32 (the step taken
                                   // then leaves an error near the FP32 floor)
constexpr float kTau32 = 1e-5f;    // FP32 rounding-level acceptance factor
constexpr float kBorder32 = 1e-4f; // "clearly outside": distance > kBorder32 * Xrel
constexpr int kPark = 31;          // run the FP64 refinement with >= kPark lanes parked
constexpr int kMaxRefine = 4;
constexpr double kCertStep = 2e-11;  // volumes: accept the first FP64 correction when the
                                     // next step is estimated below this (see certified)
                                     // and the result is kCertEdge (find_common.cuh)
                                     // inside the element

// The FP64 kernel that finishes the queued points counts into the second
// half of the statistics array, so the two precisions' work stays separate.
inline unsigned long long* fallback_stats(unsigned long long* stats) { return stats ? stats + 8 : nullptr; }

// Gauss-Newton correction s from (G^T G) s = G^T dx, in the precision T of
// its arguments; false where G^T G is not positive definite or det(G^T G) is
// below rel_det times the product of its diagonal (ill-conditioned for T).
template <int D, int DR, typename T>
__device__ __forceinline__ bool gauss_newton_step(const T* G, const T (&dx)[D], T rel_det, T (&s)[DR]) {
  T H[DR][DR], b[DR];
#pragma unroll
  for (int j = 0; j < DR; ++j) {
    T t = T(0);
#pragma unroll
    for (int c = 0; c < D; ++c) t += G[c * DR + j] * dx[c];
    b[j] = t;
#pragma unroll
    for (int k = 0; k < DR; ++k) {
      T u = T(0);
#pragma unroll
      for (int c = 0; c < D; ++c) u += G[c * DR + j] * G[c * DR + k];
      H[j][k] = u;
    }
  }
  T dprod = T(1);
#pragma unroll
  for (int j = 0; j < DR; ++j) dprod *= H[j][j];
  T det;
  if constexpr (DR == 1) {
    det = H[0][0];
  } else if constexpr (DR == 2) {
    det = H[0][0] * H[1][1] - H[0][1] * H[1][0];
  } else {
    det = H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) - H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +
          H[0][2] * (H[1][0] * H[2][1] - H[1][1] * H[2][0]);
  }
  return spd_solve<DR, T>(H, b, s) && det > rel_det * dprod;
}

// Volumes: may the first FP64 correction s1 (step size mx) from the
// converged FP32 iterate r0 stand as the result?  The FP64 iteration of
// Sec. 3.2.1 stops once its proposed step is below the Newton tolerance;
// with the residual at r0 taken in FP64 and the correction solved with the
// FP32 Jacobian J~ evaluated at r0, the error after the correction is
// e1 <= q / (1 - q) |s1| (inf-norms), q = |J~^-1| (|J~ - G(r0)| + L |e0| / 2),
// and the next step would be about e1.  Two parts of q:
//  * the curvature term |J~^-1| L |s1|, L the element's bound on the second
//    derivatives of the map (setup: the nodes' distance from the map's
//    tangent at r = 0 times the sums of |phi''|, |phi'| |phi'| of the basis;
//    box32 slot 19), with |e0| <= 2 |s1| while q <= 1/2;
//  * the relative error of the FP32 Jacobian and of the FP32 solve,
//    estimated as 64 u cond(J~) with u = 2^-24 (an estimate, not a bound:
//    the Jacobian's error measured on the deformed 32^3 mesh is a few
//    u cond(J~)); the FP64 residual's rounding moves r by |J~^-1| times a
//    few ulp of the coordinates, far below kCertStep.
// Certified when that estimate of e1 is below kCertStep and every |r_j| is
// below 1 - kCertEdge, so the code INTERIOR is the FP64 iteration's too.
template <int D>
__device__ __forceinline__ bool certified(const float* G, float curv, double mx, const double* rn) {
  static_assert(D == 2 || D == 3, "volumes only");
  float inv[D * D], det;
  if constexpr (D == 2) {
    det = G[0] * G[3] - G[1] * G[2];
    inv[0] = G[3];
    inv[1] = -G[1];
    inv[2] = -G[2];
    inv[3] = G[0];
  } else {
    inv[0] = G[4] * G[8] - G[5] * G[7];
    inv[1] = G[2] * G[7] - G[1] * G[8];
    inv[2] = G[1] * G[5] - G[2] * G[4];
    inv[3] = G[5] * G[6] - G[3] * G[8];
    inv[4] = G[0] * G[8] - G[2] * G[6];
    inv[5] = G[2] * G[3] - G[0] * G[5];
    inv[6] = G[3] * G[7] - G[4] * G[6];
    inv[7] = G[1] * G[6] - G[0] * G[7];
    inv[8] = G[0] * G[4] - G[1] * G[3];
    det = G[0] * inv[0] + G[1] * inv[3] + G[2] * inv[6];
  }
  float nG = 0.f, nI = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      a += fabsf(G[i * D + j]);
      b += fabsf(inv[i * D + j]);
    }
    nG = fmaxf(nG, a);
    nI = fmaxf(nI, b);
  }
  nI = nI / fabsf(det) * 1.001f;  // covers the FP32 rounding of the adjugate
  const float m = (float)mx;
  const float q = 64.f * 5.9604645e-08f * nG * nI + nI * curv * m;
  if (!(q < 0.5f) || !(q / (1.f - q) * m <= (float)kCertStep)) return false;
  bool in = true;
#pragma unroll
  for (int j = 0; j < D; ++j) in &= fabs(rn[j]) < 1.0 - kCertEdge;
  return in;
}

// Shared memory of one CTA of the mixed-precision lane loop.
template <int N, int D, int DR>
struct MixedShared {
  double slab64[DR == 3 ? 2 * N * kFindThreads : 1];
  float slab32[DR == 3 ? 2 * N * kFindThreads : 1];
  float hs[beta_entries<DR>() * kFindThreads];
  float bscr[(kFindThreads / 32) * kBetaScratch];
  unsigned long long next;
};

// The mixed-precision lane loop over a source of work (see find_f64.cuh).
template <int N, int D, int DR, class Work>
__device__ __forceinline__ void find_mixed_loop(const Work& w, const BasisTab& B, int* __restrict__ queue,
                                                int* __restrict__ qcount, unsigned long long* stats,
                                                MixedShared<N, D, DR>& sh) {
  constexpr int NN = ipow(N, DR);
  constexpr int P32 = pitch32(N), NE32 = NN / N * P32;  // the padded FP32 copy
  float* const s_hs = sh.hs;
  float* const wscr = sh.bscr + (threadIdx.x >> 5) * kBetaScratch;
  const TSlots<N, double> ts64{sh.slab64};
  const TSlots<N, float> ts32{sh.slab32};
  unsigned long long& s_next = sh.next;
  if (threadIdx.x == 0) s_next = 0;
  __syncthreads();
  Counters cnt;
  const int64_t n = w.n;
  const int clog2 = w.clog2;
  const int64_t nchunks = (n + (1 << clog2) - 1) >> clog2;
  const DevMesh* mp = w.first();
  int item = 0;
  int mode = X_IDLE, etype = X_INIT;
  int64_t pi = 0;
  double xs[D];
  float x32[D], xr[D];
  int q = 0, qend = 0, e = -1, l = 0, nref = 0;
  bool has_border = false, clipped = false;
  float r[DR], rn[DR], dx[D], G[D * DR];
  float alpha = 1.f, F = 0.f, pred = 0.f, xrel = 1.f;
  double r64[DR];
  unsigned guard = 0;
#pragma unroll
  for (int j = 0; j < DR; ++j) r[j] = rn[j] = 0.f, r64[j] = 0.0;

  while (true) {
    bool need = false;
    while (mode != X_DONE && mode != X_PARK && !need) {
      if (++guard > (1u << 26)) {
        record_status(mp->status, FP_DEV_SPIN_CAP);
        mode = X_DONE;
        break;
      }
      if (mode == X_IDLE) {
        const unsigned long long s = atomicAdd(&s_next, 1ull);
        const int64_t chunk = (int64_t)(s >> clog2) * w.ctas() + w.cta();
        if (chunk >= nchunks) {
          mode = X_DONE;
          break;
        }
        const int64_t g = (chunk << clog2) + (int64_t)(s & ((1u << clog2) - 1));
        if (g >= n) continue;
        w.locate(g, mp, item, pi);
        w.load(item, pi, xs);
#pragma unroll
        for (int c = 0; c < D; ++c) x32[c] = (float)xs[c];
        has_border = false;
        const int64_t cell = point_cell<D>(*mp, xs);
        if (cell < 0) {
          const double z0[DR] = {};
          w.write(item, pi, FP_NOT_FOUND, -1, z0, INFINITY);
          continue;
        }
        q = __ldg(mp->cell_start + cell);
        qend = __ldg(mp->cell_start + cell + 1);
        mode = X_SCAN;
      }
      if (mode == X_SCAN) {
        e = next_candidate<D>(*mp, xs, x32, q, qend, cnt);
        if (e < 0) {
          if (has_border) {
            queue[atomicAdd(qcount, 1)] = (int)w.global(item, pi);
            ++cnt.v[6];
          } else {
            const double z0[DR] = {};
            w.write(item, pi, FP_NOT_FOUND, -1, z0, INFINITY);
          }
          mode = X_IDLE;
          continue;
        }
        ++cnt.v[0];
        rel_point<D>(*mp, e, xs, xr);
        xrel = __ldg(mp->box32 + (int64_t)e * BOX32 + 18);
        // start from the linearised map, r0 = clamp(T (x* - x(0))): the FP32
        // phase promises the converged result, not the FP64 path's iterates
        {
          // slots 20..31 of the record, xc[3] T[9], as three 16-byte vectors
          const float4* r4 = reinterpret_cast<const float4*>(mp->box32 + (int64_t)e * BOX32 + 20);
          const float4 a = __ldg(r4), b = __ldg(r4 + 1), c4 = __ldg(r4 + 2);
          const float lin[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c4.x, c4.y, c4.z, c4.w};
#pragma unroll
          for (int j = 0; j < DR; ++j) {
            float v = 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) v = fmaf(lin[3 + j * 3 + c], xr[c] - lin[c], v);
            r[j] = fminf(1.f, fmaxf(-1.f, v));
          }
        }
        etype = X_INIT;
        need = true;
        break;
      }
      if (mode == X_RESTORE) {
        etype = X_REST;
        need = true;
        break;
      }
      // X_NEWTON: one FP32 step (X_CONV: the converged iterate, evaluated)
      bool done = false, converged = false;
      if (mode == X_CONV) {
        done = converged = true;
      } else if (l >= mp->max_iter) {
        done = true;
      } else {
        const bool beta = (l > 0) && at_bound<DR>(r);
        float HS[DR][DR] = {};
        if (beta) {
          beta_load<DR, float>(s_hs, HS);  // computed by the warp after the last evaluation
          ++cnt.v[3];
        }
        float ds[DR];
        bool used_beta;
        const float mx = newton_step<D, DR, float>(G, dx, r, alpha, beta, HS, rn, ds, clipped, used_beta);
        if (mx < kTol32) {
          F = model_dist2<D, DR, float>(G, dx, ds);
#pragma unroll
          for (int j = 0; j < DR; ++j) r[j] = rn[j];
          ++cnt.v[1];
          if constexpr (DR == D) {
            // volumes: evaluate at the converged iterate, so that the FP64
            // correction uses the FP32 Jacobian at that point (certified)
            etype = X_FINAL;
            need = true;
          } else {
            done = converged = true;
          }
        } else {
          pred = predicted_decrease<D, DR, float>(G, dx, ds, used_beta, HS);
          if (!(pred > 0.f)) {
            done = true;
          } else {
            ++cnt.v[1];
            etype = X_TRIAL;
            need = true;
          }
        }
      }
      if (done) {
        bool inside = true;
#pragma unroll
        for (int j = 0; j < DR; ++j) inside &= below_unit(r[j]);
        const float far2 = (kBorder32 * xrel) * (kBorder32 * xrel);
        const float dtol = (float)mp->dist_tol;
        if (converged && inside && (DR == D || F < 0.5f * dtol)) {
#pragma unroll
          for (int j = 0; j < DR; ++j) r64[j] = (double)r[j];
          nref = 0;
          mode = X_PARK;
        } else if (F > far2 && (!inside || (DR < D && converged && F > 2.f * dtol))) {
          has_border = true;
          mode = X_SCAN;
        } else {
          queue[atomicAdd(qcount, 1)] = (int)w.global(item, pi);
          ++cnt.v[6];
          mode = X_IDLE;
        }
      }
    }
    const unsigned parked = __ballot_sync(0xffffffffu, mode == X_PARK);
    const unsigned busy = __ballot_sync(0xffffffffu, need);
    if (parked == 0 && busy == 0) {
      if (__all_sync(0xffffffffu, mode == X_DONE)) break;
      continue;
    }
    // ---- FP64 refinement, warp-batched --------------------------------------
    if ((__popc(parked) >= kPark || busy == 0) && mode == X_PARK) {
      ++cnt.v[4];
      // Volumes converge to dx = 0, where the FP32 Jacobian only sets the
      // rate.  On a surface or line the converged residual is normal to the
      // manifold and not zero, and the stationary point G^T dx = 0 moves by
      // |dx| times the Jacobian's error, so there G is evaluated in FP64.
      constexpr bool kG64 = DR < D;
      double xv[D], dxd[D], Gd[kG64 ? D * DR : 1];
      eval_xG<N, D, DR, kG64, double>(mp->coords + (int64_t)e * NN, mp->cstride, B, r64, ts64, xv,
                                      kG64 ? Gd : nullptr);
#pragma unroll
      for (int c = 0; c < D; ++c) dxd[c] = xs[c] - xv[c];
      double s[DR];
      bool ok;
      if constexpr (kG64) {
        ok = gauss_newton_step<D, DR, double>(Gd, dxd, 1e-8, s);
      } else {
        // Iterative refinement: the residual in FP64, the correction from
        // the FP32 Jacobian solved in FP32.  The correction's relative error
        // (about cond(G) times the FP32 rounding) only slows the FP64
        // iteration from quadratic to linear convergence at that rate, so
        // the FP32 solve is used where G^T G is well enough conditioned
        // for a rate far below 1 and the FP64 solve otherwise.
        float d32[D], s32[DR];
#pragma unroll
        for (int c = 0; c < D; ++c) d32[c] = (float)dxd[c];
        ok = gauss_newton_step<D, DR, float>(G, d32, 1e-3f, s32);
#pragma unroll
        for (int j = 0; j < DR; ++j) s[j] = (double)s32[j];
        if (!ok) {
          double G64[D * DR];
#pragma unroll
          for (int q2 = 0; q2 < D * DR; ++q2) G64[q2] = (double)G[q2];
          ok = gauss_newton_step<D, DR, double>(G64, dxd, 1e-8, s);
        }
      }
      bool inside = ok;
      double mx = 0.0, rnn[DR];
#pragma unroll
      for (int j = 0; j < DR; ++j) {
        rnn[j] = r64[j] + s[j];
        inside &= below_unit(rnn[j]);
        mx = fmax(mx, fabs(s[j]));
      }
      bool cert = false;
      if constexpr (DR == D) {
        if (inside && nref == 0 && !(mx < mp->newton_tol))
          cert = certified<D>(G, __ldg(mp->box32 + (int64_t)e * BOX32 + 19), mx, rnn);
      }
      if (!inside) {
        queue[atomicAdd(qcount, 1)] = (int)w.global(item, pi);
        ++cnt.v[6];
        mode = X_IDLE;
      } else if (mx < mp->newton_tol || cert) {
        double f = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          double t = dxd[c];
          if constexpr (kG64) {
#pragma unroll
            for (int j = 0; j < DR; ++j) t -= Gd[c * DR + j] * s[j];
          } else {
            // G s is below the Newton tolerance times |G|: FP32 keeps it to
            // 1e-7 relative, far below the FP64 rounding of dx
            float gs = 0.f;
#pragma unroll
            for (int j = 0; j < DR; ++j) gs = fmaf(G[c * DR + j], (float)s[j], gs);
            t -= (double)gs;
          }
          f += t * t;
        }
        if (DR < D && !(f < mp->dist_tol)) {
          queue[atomicAdd(qcount, 1)] = (int)w.global(item, pi);
          ++cnt.v[6];
        } else {
          w.write(item, pi, FP_INTERIOR, e, rnn, f);
        }
        mode = X_IDLE;
      } else if (++nref >= kMaxRefine) {
        queue[atomicAdd(qcount, 1)] = (int)w.global(item, pi);
        ++cnt.v[6];
        mode = X_IDLE;
      } else {
#pragma unroll
        for (int j = 0; j < DR; ++j) r64[j] = rnn[j];
      }
    }
    // ---- FP32 evaluation -----------------------------------------------------
    if (need) {
      float re[DR];
#pragma unroll
      for (int j = 0; j < DR; ++j) re[j] = (etype == X_TRIAL) ? rn[j] : r[j];
      float xv[D];
      if (etype != X_REST) ++cnt.v[7];
      eval_xG<N, D, DR, true, float, P32>(mp->coords32p + (int64_t)e * NE32, mp->cstride32p, B, re, ts32, xv,
                                          G);
      float Fn = 0.f;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        dx[c] = xr[c] - xv[c];
        Fn = fmaf(dx[c], dx[c], Fn);
      }
      if (etype == X_TRIAL) {
        ++l;
        if (trial_accepts<float>(F, Fn, pred, clipped, xrel, alpha, kTau32)) {
#pragma unroll
          for (int j = 0; j < DR; ++j) r[j] = rn[j];
          F = Fn;
          mode = X_NEWTON;
        } else {
          ++cnt.v[2];
          mode = X_RESTORE;
        }
      } else if (etype == X_FINAL) {
        F = Fn;
        mode = X_CONV;
      } else {
        if (etype == X_INIT) {
          alpha = 1.f;
          l = 0;
        }
        F = Fn;
        mode = X_NEWTON;
      }
    }
    // ---- warp-uniform beta term for the next FP32 Newton step ------------
    {
      const bool want = need && mode == X_NEWTON && l > 0 && at_bound<DR>(r);
      const BetaReq bq = beta_request<N, D, DR, float, P32>(want, r, dx, G);
      if (__any_sync(0xffffffffu, bq.kind != BETA_NONE))
        beta_warp<N, D, DR, float, P32>(bq, mp->coords32p + (int64_t)e * NE32, mp->cstride32p, r, dx, B, wscr,
                                        s_hs);
    }
  }
  cnt.flush(stats);
}

}  // namespace
}  // namespace fp
