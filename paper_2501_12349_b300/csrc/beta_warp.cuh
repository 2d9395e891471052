// The beta term of Eq. newton_hessian, HS_jk = sum_c dx_c d2x_c/dr_j dr_k,
// computed by the whole warp for the lanes that need it.
//
// Only iterates on the element boundary need the term, about one Newton
// step in ten, so a per-lane contraction runs with a few of the warp's lanes
// active while the FP64 pipe charges every warp instruction in full.  Here
// the term is computed at the warp-uniform site right after the evaluation
// that made r current, with all 32 lanes sharing the work of each request:
//  * the components are first folded into one scalar field,
//    W = sum_c dx_c x_c, so the second derivatives are those of one
//    polynomial;
//  * a face or edge request (every on-boundary coordinate held: the
//    held coordinates sit on a GLL end node, where the basis is a unit
//    vector, so only the face or edge slice of the element data enters)
//    takes a group of 8 lanes, four requests per pass: lane q evaluates the
//    q-th basis function and two derivatives, then contracts row q of the
//    face (or node q of the edge);
//  * a full-element request (a coordinate on the boundary is free, hexes
//    only) takes the whole warp: lanes 8d+q evaluate basis function q along
//    direction d, each lane contracts one (or two) of the N^2 rows, and a
//    warp reduction sums the six entries.
// The owner lane finds its entries (upper triangle) in shared memory when it
// takes its next Newton step.
#pragma once
#include "find_common.cuh"

namespace fp {

enum : int { BETA_NONE = 0, BETA_ZERO = 1, BETA_SLICE = 2, BETA_FULL = 3 };

// What one lane's beta term needs.
struct BetaReq {
  int kind;  // BETA_*
  int nf;    // free directions of a slice: 1 or 2
  int a, b;  // the free directions, a < b (b unused when nf == 1)
  int base;  // node offset of the slice (the held coordinates' end nodes)
};

// Number of stored entries (upper triangle of HS) and their index.
template <int DR>
constexpr int beta_entries() { return DR * (DR + 1) / 2; }
template <int DR>
__device__ __forceinline__ int beta_index(int j, int k) { return j * DR - j * (j - 1) / 2 + (k - j); }

// Per warp: the basis values of four slice requests (one direction, 3 x 8)
// or of one full request (three directions, 3 x 3 x 8).
constexpr int kBetaScratch = 96;

// The held set as newton_step defines it (g = -G^T dx; a coordinate on a
// bound is held when the gradient points out of the box).
template <int N, int D, int DR, typename T, int P = N>
__device__ __forceinline__ BetaReq beta_request(bool want, const T (&r)[DR], const T (&dx)[D],
                                                const T (&G)[D * DR]) {
  BetaReq q{BETA_NONE, 0, 0, 0, 0};
  if (!want) return q;
  const int stride[3] = {1, P, P * N};
  int fr[DR];
  int nf = 0, base = 0;
  bool full = false;
#pragma unroll
  for (int j = 0; j < DR; ++j) {
    T g = T(0);
#pragma unroll
    for (int c = 0; c < D; ++c) g -= G[c * DR + j] * dx[c];
    const bool onb = is_unit(r[j]);
    const bool held = held_at_bound(r[j], g);
    full |= onb && !held;
    if (held) base += (sign_bit(r[j]) ? 0 : N - 1) * stride[j];
    else fr[nf++] = j;
  }
  if (full) {
    // quads and surface quads: the whole element is the 2D slice (0, 1)
    q.kind = (DR == 3) ? BETA_FULL : BETA_SLICE;
    q.nf = DR;
    q.a = 0;
    q.b = 1;
    q.base = 0;
    return q;
  }
  if (nf == 0) {
    q.kind = BETA_ZERO;
    return q;
  }
  q.kind = BETA_SLICE;
  q.nf = nf;
  q.a = fr[0];
  q.b = nf > 1 ? fr[1] : 0;
  q.base = base;
  return q;
}

// phi_q(x), phi_q'(x), phi_q''(x) of the single basis function q (product
// form w_q prod_{m != q} (x - z_m), derivatives by the product rule), the
// N - 1 factors taken in ascending node order with node q skipped by
// selection (no work for it).  The second derivative is carried halved,
// h = p''/2 (h <- h t + p'), and scaled by the table's 2 w_q at the end, so
// the recurrence needs no doubling: at N = 5, 15 FP64 operations.  q >= N
// gives zeros.
template <int N, typename T>
__device__ __forceinline__ void basis_one(const T* z, const T* w, const T* w2, int q, T x, T& v0, T& v1,
                                          T& v2) {
  T wq = T(0), w2q = T(0);
#pragma unroll
  for (int m = 0; m < N; ++m) {
    wq = (m == q) ? w[m] : wq;
    w2q = (m == q) ? w2[m] : w2q;
  }
  T p0 = T(1), p1 = T(0), h = T(0);
#pragma unroll
  for (int m = 0; m < N - 1; ++m) {
    const T t = x - ((m >= q) ? z[m + 1] : z[m]);
    if (m == 0) {
      p0 = t;
      p1 = T(1);
    } else if (m == 1) {
      h = T(1);
      p1 = p1 * t + p0;  // t + p0: the product is exact
      p0 = p0 * t;
    } else {
      h = fma(h, t, p1);
      p1 = fma(p1, t, p0);
      p0 = p0 * t;
    }
  }
  v0 = wq * p0;
  v1 = wq * p1;
  v2 = w2q * h;
}

template <int DR, typename T>
__device__ __forceinline__ T pick(const T (&v)[DR], int j) {
  T s = v[0];
#pragma unroll
  for (int i = 1; i < DR; ++i)
    if (i == j) s = v[i];
  return s;
}

template <typename T>
__device__ __forceinline__ const T* shfl_ptr(const T* p, int src) {
  return reinterpret_cast<const T*>(
      __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(p), src));
}

// Called by all 32 lanes of a converged warp.  X, cs: this lane's element
// data (component c at X + c*cs, rows of N r-nodes at pitch P, as
// beta_request's base assumes); scr: the warp's kBetaScratch values;
// hs: [beta_entries][kFindThreads] values of the CTA.
template <int N, int D, int DR, typename T, int P = N>
__device__ void beta_warp(const BetaReq& q, const T* X, int64_t cs, const T (&r)[DR], const T (&dx)[D],
                          const BasisTab& B, T* scr, T* hs) {
  constexpr unsigned kAll = 0xffffffffu;
  constexpr int NH = beta_entries<DR>();
  const int lane = threadIdx.x & 31;
  const int wbase = threadIdx.x & ~31;
  const T* z = TabOf<T>::z(B);
  const T* w = TabOf<T>::w(B);
  const T* w2 = TabOf<T>::w2(B);
  const int stride[3] = {1, P, P * N};

  if (q.kind == BETA_ZERO) {
#pragma unroll
    for (int v = 0; v < NH; ++v) hs[v * kFindThreads + threadIdx.x] = T(0);
  }

  // ---- face / edge slices: groups of 8 lanes, four requests per pass ----
  unsigned ms = __ballot_sync(kAll, q.kind == BETA_SLICE);
  const int grp = lane >> 3, gq = lane & 7;
  while (ms) {
    unsigned m = ms;
    for (int k = 0; k < grp && m; ++k) m &= m - 1;
    const int src = m ? __ffs(m) - 1 : -1;
    for (int k = 0; k < 4 && ms; ++k) ms &= ms - 1;
    const int s = src < 0 ? lane : src;
    const int nf = __shfl_sync(kAll, q.nf, s);
    const int a = __shfl_sync(kAll, q.a, s);
    const int b = __shfl_sync(kAll, q.b, s);
    const int base = __shfl_sync(kAll, q.base, s);
    const T ra = __shfl_sync(kAll, pick<DR, T>(r, q.a), s);
    const T rb = __shfl_sync(kAll, pick<DR, T>(r, q.b), s);
    T dxs[D];
#pragma unroll
    for (int c = 0; c < D; ++c) dxs[c] = __shfl_sync(kAll, dx[c], s);
    const T* Xs = shfl_ptr(X, s);
    const int64_t css = __shfl_sync(kAll, (long long)cs, s);
    T a0, a1, a2, b0, b1, b2;
    basis_one<N, T>(z, w, w2, gq, ra, a0, a1, a2);
    basis_one<N, T>(z, w, w2, gq, rb, b0, b1, b2);
    T* sc = scr + grp * 24;
    sc[gq] = a0;
    sc[8 + gq] = a1;
    sc[16 + gq] = a2;
    __syncwarp();
    int sa = 1, sb = 1;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (j == a) sa = stride[j];
      if (j == b) sb = stride[j];
    }
    T h0 = T(0), h1 = T(0), h2 = T(0);
    if (src >= 0 && gq < N) {
      if (nf == 2) {
        // row b = gq of the face: contract W along a
        const T* row = Xs + base + gq * sb;
        T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          T W = T(0);
#pragma unroll
          for (int c = 0; c < D; ++c) W = fma(dxs[c], ldg(row + c * css + i * sa), W);
          s0 = fma(W, sc[i], s0);
          s1 = fma(W, sc[8 + i], s1);
          s2 = fma(W, sc[16 + i], s2);
        }
        h0 = s2 * b0;  // d2/da2
        h1 = s1 * b1;  // d2/da db
        h2 = s0 * b2;  // d2/db2
      } else {
        // node gq of the edge
        T W = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) W = fma(dxs[c], ldg(Xs + base + c * css + gq * sa), W);
        h0 = W * a2;
      }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      h0 += __shfl_xor_sync(kAll, h0, o);
      h1 += __shfl_xor_sync(kAll, h1, o);
      h2 += __shfl_xor_sync(kAll, h2, o);
    }
    if (src >= 0 && gq == 0) {
      T* o = hs + wbase + src;
#pragma unroll
      for (int v = 0; v < NH; ++v) o[v * kFindThreads] = T(0);
      o[beta_index<DR>(a, a) * kFindThreads] = h0;
      if (nf == 2) {
        o[beta_index<DR>(a, b) * kFindThreads] = h1;
        o[beta_index<DR>(b, b) * kFindThreads] = h2;
      }
    }
    __syncwarp();
  }

  // ---- full element (hexes): the whole warp on one request per pass ----
  if constexpr (DR == 3) {
    unsigned mf = __ballot_sync(kAll, q.kind == BETA_FULL);
    while (mf) {
      const int src = __ffs(mf) - 1;
      mf &= mf - 1;
      T rs[3], dxs[D];
#pragma unroll
      for (int j = 0; j < 3; ++j) rs[j] = __shfl_sync(kAll, r[j], src);
#pragma unroll
      for (int c = 0; c < D; ++c) dxs[c] = __shfl_sync(kAll, dx[c], src);
      const T* Xs = shfl_ptr(X, src);
      const int64_t css = __shfl_sync(kAll, (long long)cs, src);
      const int dd = lane >> 3;
      T v0, v1, v2;
      basis_one<N, T>(z, w, w2, gq, dd == 0 ? rs[0] : (dd == 1 ? rs[1] : rs[2]), v0, v1, v2);
      if (dd < 3) {
        scr[dd * 24 + gq] = v0;
        scr[dd * 24 + 8 + gq] = v1;
        scr[dd * 24 + 16 + gq] = v2;
      }
      __syncwarp();
      T h[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
      for (int row = lane; row < N * N; row += 32) {
        const int j = row % N, k = row / N;
        const T* xr = Xs + P * j + P * N * k;
        T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          T W = T(0);
#pragma unroll
          for (int c = 0; c < D; ++c) W = fma(dxs[c], ldg(xr + c * css + i), W);
          s0 = fma(W, scr[i], s0);
          s1 = fma(W, scr[8 + i], s1);
          s2 = fma(W, scr[16 + i], s2);
        }
        const T p1 = scr[24 + j], dp1 = scr[32 + j], d2p1 = scr[40 + j];
        const T p2 = scr[48 + k], dp2 = scr[56 + k], d2p2 = scr[64 + k];
        h[0] = fma(s2 * p1, p2, h[0]);
        h[1] = fma(s1 * dp1, p2, h[1]);
        h[2] = fma(s1 * p1, dp2, h[2]);
        h[3] = fma(s0 * d2p1, p2, h[3]);
        h[4] = fma(s0 * dp1, dp2, h[4]);
        h[5] = fma(s0 * p1, d2p2, h[5]);
      }
#pragma unroll
      for (int o = 1; o < 32; o <<= 1)
#pragma unroll
        for (int v = 0; v < 6; ++v) h[v] += __shfl_xor_sync(kAll, h[v], o);
      if (lane == 0) {
#pragma unroll
        for (int v = 0; v < 6; ++v) hs[v * kFindThreads + wbase + src] = h[v];
      }
      __syncwarp();
    }
  }
}

// The owner's entries back as a full DR x DR matrix.
template <int DR, typename T>
__device__ __forceinline__ void beta_load(const T* hs, T (&HS)[DR][DR]) {
#pragma unroll
  for (int j = 0; j < DR; ++j)
#pragma unroll
    for (int k = j; k < DR; ++k) {
      const T v = hs[beta_index<DR>(j, k) * kFindThreads + threadIdx.x];
      HS[j][k] = v;
      HS[k][j] = v;
    }
}

}  // namespace fp
