// Pieces of the find kernels (Sec. 3.2) shared by the FP64 and mixed paths:
// certified FP32 prefilters with exact FP64 fallbacks, the trust-region
// Newton step of Sec. 3.2.1 split into its parts, result writes, counters.
#pragma once
#include <math.h>

#include "fp_basis.cuh"
#include "fp_common.cuh"

namespace fp {

constexpr int kFindThreads = 128;

// Per-thread counters: [0] candidates, [1] Newton iterations, [2] rejected
// steps, [3] beta = 1 iterations, [4] FP64 refinement evaluations (mixed),
// [5] box tests decided in FP64, [6] points handed to the FP64 kernel (mixed).
struct Counters {
  unsigned v[8];
  __device__ Counters() {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = 0;
  }
  __device__ void flush(unsigned long long* stats) {
    if (!stats) return;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      unsigned x = v[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) == 0 && x) atomicAdd(stats + i, (unsigned long long)x);
    }
  }
};

// CTAs of kFindThreads per SM that the FP64 find kernel is compiled for:
// its registers fit three per SM up to N = 6 and two above.
__host__ __device__ constexpr int f64_ctas(int N) { return N <= 6 ? 3 : 2; }
// The same for the mixed-precision kernel: four per SM where its registers
// fit 128 without spilling, three elsewhere (surface quads of N >= 5, whose
// FP64 refinement also evaluates G, and hexes of N >= 7), two for surface
// quads of N = 8.
__host__ __device__ constexpr int mixed_ctas(int N, int D, int DR) {
  return (DR == 3 && N <= 6) || (DR == 2 && (D == 2 || N <= 4)) || DR == 1 ? 4
         : (D == 3 && DR == 2 && N >= 8)                                ? 2
                                                                         : 3;
}

inline int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 148;
  }
  return n;
}

// Persistent grid: per_sm CTAs per SM, fewer when n is small.
// The FP64 kernel over the points a mixed launch hands over (about 1% of
// them) takes as long as its slowest points, each a chain of full-warp FP64
// instructions.  Up to kGroupMaxPoints points per launch (a queue of tens
// of thousands) it runs in group mode, which searches a point's candidate
// elements side by side; above, the queue is long enough for its total work
// to count, and the one-lane-per-point loop runs as one-warp CTAs with
// chunks of 4 points (in 128-thread CTAs the first warp to ask takes the
// CTA's whole chunk, so the few busy warps can share one sub-partition's
// FP64 unit).
constexpr int64_t kGroupMaxPoints = (int64_t)1 << 22;
constexpr int kFollowThreads = 32;
constexpr int kFollowClog2 = 2;
inline int follow_blocks() { return sm_count() * 8; }

inline int persistent_blocks(int64_t n, int per_sm) {
  const int64_t want = (n + kFindThreads - 1) / kFindThreads;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

// ---- exact FP64 tests ---------------------------------------------------------

// Eq. AABB_test (as lo <= x <= hi) and Eq. OBB_test on the expanded boxes,
// with the same rounded operations as the FP64 definition.
template <int D>
__device__ __forceinline__ bool in_boxes_f64(const DevMesh& m, int64_t e, const double (&xs)[D]) {
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const double lo = __ldg(m.aabb + e * 2 * D + c), hi = __ldg(m.aabb + e * 2 * D + D + c);
    if (!(xs[c] >= lo && xs[c] <= hi)) return false;
  }
#pragma unroll
  for (int c = 0; c < D; ++c) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < D; ++q)
      s = __dadd_rn(s, __dmul_rn(__ldg(m.obb_A + (e * D + c) * D + q),
                                 __dsub_rn(xs[q], __ldg(m.obb_c + e * D + q))));
    if (!(fabs(s) <= 1.0)) return false;
  }
  return true;
}

// ---- certified FP32 tests -----------------------------------------------------

// The box test of element rec in FP32: 0 = outside, 1 = inside, 2 = too
// close to a face to decide in FP32.  The margins bound the rounding of the
// FP32 inputs and operations (u = 2^-24): an AABB difference is off by at
// most 2u(|x| + |b|) + u|x - b| < 4u(|x| + |b|); an OBB coordinate
// sum_k A_jk (x_k - c_k) by at most 6u sum_k |A_jk| (|x_k| + |c_k|); the FP64
// computation of the same quantities is off by ~1e-16 of them.  Margins of
// 4u and 16u are used, so a decision taken here equals the FP64 one.
// The record (128-byte aligned) is read as 16-byte vectors: a scalar load
// per value costs an L1 access per lane, and with the lanes of a warp on
// different elements the L1 is the bound of the box loops; the AABB test
// needs the first two vectors, the OBB test three more.
template <int D>
__device__ __forceinline__ int boxes_f32(const float* __restrict__ rec, const float (&x)[D]) {
  const float4* r4 = reinterpret_cast<const float4*>(rec);
  const float4 v0 = __ldg(r4), v1 = __ldg(r4 + 1);
  float b[18];  // lo[3] hi[3] c[3] A[9]
  b[0] = v0.x, b[1] = v0.y, b[2] = v0.z, b[3] = v0.w, b[4] = v1.x, b[5] = v1.y, b[6] = v1.z, b[7] = v1.w;
  int res = 1;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const float lo = b[c], hi = b[3 + c];
    const float dl = x[c] - lo, dh = hi - x[c];
    const float ml = 2.3841858e-07f * (fabsf(x[c]) + fabsf(lo));  // 4u
    const float mh = 2.3841858e-07f * (fabsf(x[c]) + fabsf(hi));
    if (dl < -ml || dh < -mh) return 0;
    if (!(dl > ml && dh > mh)) res = 2;
  }
  const float4 v2 = __ldg(r4 + 2), v3 = __ldg(r4 + 3), v4 = __ldg(r4 + 4);
  b[8] = v2.x, b[9] = v2.y, b[10] = v2.z, b[11] = v2.w, b[12] = v3.x, b[13] = v3.y, b[14] = v3.z;
  b[15] = v3.w, b[16] = v4.x, b[17] = v4.y;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    float v = 0.f, eb = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float a = b[9 + j * 3 + k], cc = b[6 + k];
      v = fmaf(a, x[k] - cc, v);
      eb = fmaf(fabsf(a), fabsf(x[k]) + fabsf(cc), eb);
    }
    eb *= 9.5367432e-07f;  // 16u
    const float av = fabsf(v);
    if (av > 1.f + eb) return 0;
    if (!(av < 1.f - eb)) res = 2;
  }
  return res;
}

// Next element of the cell list [q, qend) that passes the box filter, or -1.
template <int D>
__device__ __forceinline__ int next_candidate(const DevMesh& m, const double (&xs)[D],
                                              const float (&x32)[D], int& q, int qend,
                                              Counters& cnt) {
  while (q < qend) {
    const int c = __ldg(m.cell_elems + q);
    ++q;
    if (c < 0 || c >= m.NE) {
      record_status(m.status, FP_DEV_BAD_ELEM);
      continue;
    }
    int t = boxes_f32<D>(m.box32 + (int64_t)c * BOX32, x32);
    if (t == 2) {
      ++cnt.v[5];
      t = in_boxes_f64<D>(m, c, xs) ? 1 : 0;
    }
    if (t == 1) return c;
  }
  return -1;
}

// x* relative to the element reference point, in FP64 and rounded to FP32.
template <int D>
__device__ __forceinline__ void rel_point(const DevMesh& m, int64_t e, const double (&xs)[D],
                                          float (&xr)[D]) {
#pragma unroll
  for (int c = 0; c < D; ++c) xr[c] = (float)(xs[c] - elem_ref(m.aabb, D, e, c));
}

// Closest GLL node of element e to xs (Sec. 3.2.1, initial guess), ties to
// the lowest node index, as the FP64 definition computes it: squared
// distances sum_c (x_c - X_c)^2 in non-contracted FP64.  The FP32 scan over
// the relative coordinates (xr = fl(x* - x_ref), X32 = fl(X - x_ref)) is
// certified when its best distance beats the second best by more than both
// rounding bounds; otherwise the FP64 scan decides.  Bound, with
// E = 4u (|xr|_inf + Xrel) per component (u = 2^-24, Xrel >= |X - x_ref|):
// |d32 - d| <= 2 sqrt(D d) E + D E^2 + 8u d.
template <int N, int D, int DR>
__device__ int closest_node(const DevMesh& m, int e, const double (&xs)[D], const float (&xr)[D]) {
  constexpr int NN = ipow(N, DR);
  const float* X32 = m.coords32 + (int64_t)e * NN;
  float b1 = INFINITY, b2 = INFINITY;
  int nb = 0;
#pragma unroll 4
  for (int n = 0; n < NN; ++n) {
    float d = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const float t = xr[c] - __ldg(X32 + c * m.cstride + n);
      d = fmaf(t, t, d);
    }
    if (d < b1) {
      b2 = b1;
      b1 = d;
      nb = n;
    } else if (d < b2) {
      b2 = d;
    }
  }
  float xm = 0.f;
#pragma unroll
  for (int c = 0; c < D; ++c) xm = fmaxf(xm, fabsf(xr[c]));
  const float E = 2.3841858e-07f * (xm + __ldg(m.box32 + (int64_t)e * BOX32 + 18));
  const float B1 = 2.f * sqrtf(D * b1) * E + D * E * E + 4.7683716e-07f * b1;
  const float B2 = 2.f * sqrtf(D * b2) * E + D * E * E + 4.7683716e-07f * b2;
  if (b2 - B2 > b1 + B1) return nb;
  const double* X = m.coords + (int64_t)e * NN;
  double best = INFINITY;
  nb = 0;
  for (int n = 0; n < NN; ++n) {
    double dd = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const double t = __dsub_rn(xs[c], __ldg(X + c * m.cstride + n));
      dd = __dadd_rn(dd, __dmul_rn(t, t));
    }
    if (dd < best) {
      best = dd;
      nb = n;
    }
  }
  return nb;
}

// closest_node for every lane of a converged warp that wants it, the whole
// warp on one request at a time: lane l scans nodes l, l + 32, ... (loads
// coalesced across the warp), and a butterfly merges the lanes' best two
// (distance, node) pairs, ties to the lowest node index; the certification
// and the FP64 fallback are those of closest_node, the fallback scan shared
// the same way.  Returns the owner's node in nb.
template <int N, int D, int DR>
__device__ void closest_node_warp(bool want, const DevMesh& m, int e, const double (&xs)[D], const float (&xr)[D],
                                  int& nb) {
  constexpr int NN = ipow(N, DR);
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  unsigned mask = __ballot_sync(kAll, want);
  // this lane's request data, broadcast below
  const float* X32m = m.coords32 + (int64_t)e * NN;
  const double* X64m = m.coords + (int64_t)e * NN;
  float xm = 0.f;
#pragma unroll
  for (int c = 0; c < D; ++c) xm = fmaxf(xm, fabsf(xr[c]));
  const float Em = want ? 2.3841858e-07f * (xm + __ldg(m.box32 + (int64_t)e * BOX32 + 18)) : 0.f;
  while (mask) {
    const int src = __ffs(mask) - 1;
    mask &= mask - 1;
    const float* X32 = reinterpret_cast<const float*>(
        __shfl_sync(kAll, reinterpret_cast<unsigned long long>(X32m), src));
    const int64_t cs = __shfl_sync(kAll, (long long)m.cstride, src);
    float r32[D];
#pragma unroll
    for (int c = 0; c < D; ++c) r32[c] = __shfl_sync(kAll, xr[c], src);
    float b1 = INFINITY, b2 = INFINITY;
    int i1 = NN;
    for (int n = lane; n < NN; n += 32) {
      float d = 0.f;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const float t = r32[c] - __ldg(X32 + c * cs + n);
        d = fmaf(t, t, d);
      }
      if (d < b1) {  // nodes ascend per lane: ties keep the lower index
        b2 = b1;
        b1 = d;
        i1 = n;
      } else if (d < b2) {
        b2 = d;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob1 = __shfl_xor_sync(kAll, b1, o), ob2 = __shfl_xor_sync(kAll, b2, o);
      const int oi1 = __shfl_xor_sync(kAll, i1, o);
      const bool other = ob1 < b1 || (ob1 == b1 && oi1 < i1);
      const float lo = other ? ob1 : b1, hi = other ? b1 : ob1;
      b2 = fminf(hi, fminf(b2, ob2));
      b1 = lo;
      i1 = other ? oi1 : i1;
    }
    const float E = __shfl_sync(kAll, Em, src);
    const float B1 = 2.f * sqrtf(D * b1) * E + D * E * E + 4.7683716e-07f * b1;
    const float B2 = 2.f * sqrtf(D * b2) * E + D * E * E + 4.7683716e-07f * b2;
    int best_n = i1;
    if (!(b2 - B2 > b1 + B1)) {  // uncertified: the FP64 scan decides
      const double* X = reinterpret_cast<const double*>(
          __shfl_sync(kAll, reinterpret_cast<unsigned long long>(X64m), src));
      double x64[D];
#pragma unroll
      for (int c = 0; c < D; ++c) x64[c] = __shfl_sync(kAll, xs[c], src);
      double best = INFINITY;
      int bi = NN;
      for (int n = lane; n < NN; n += 32) {
        double dd = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const double t = __dsub_rn(x64[c], __ldg(X + c * cs + n));
          dd = __dadd_rn(dd, __dmul_rn(t, t));
        }
        if (dd < best) {
          best = dd;
          bi = n;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(kAll, best, o);
        const int oi = __shfl_xor_sync(kAll, bi, o);
        if (ob < best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      best_n = bi;
    }
    if (lane == src) nb = best_n;
  }
}

template <int N, int DR, typename T>
__device__ __forceinline__ void node_coords(const BasisTab& B, int n, T (&r)[DR]) {
  const int idx[3] = {n % N, (n / N) % N, n / (N * N)};
#pragma unroll
  for (int j = 0; j < DR; ++j) {
    T v = T(0);
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i == idx[j]) v = TabOf<T>::z(B)[i];
    r[j] = v;
  }
}

// x and G at the GLL node nb of element e, the start r0 of Newton, for
// every lane of a converged warp that wants it: the Lagrange basis is a unit
// vector at a node, so x is the node's coordinates, and column j of G is the
// derivative along the node's grid line in direction j, an N-term sum with
// the differentiation matrix dn (row dn + i*N, i the node's index in
// direction j).  The warp shares the work: the D * DR entries of G of all
// starting lanes are tasks spread over the 32 lanes (one N-term FMA chain
// each, in the order of the nodes along the line), written to the owner's
// column of sg ([D * DR][kFindThreads]) and read back by it; sl
// ([kFindThreads]) holds the warp's starting lanes by rank.  A lane that
// formed its own entries would charge the FP64 pipe all D * DR * N FMAs of
// its start as full-warp instructions.
template <int N, int D, int DR>
__device__ __forceinline__ void node_start_warp(bool want, const DevMesh& m, int e, int nb,
                                                const double* __restrict__ dn, double* sg, int* sl,
                                                double (&x)[D], double (&G)[D * DR]) {
  constexpr unsigned kAll = 0xffffffffu;
  constexpr int NN = ipow(N, DR);
  constexpr int NT = D * DR;  // tasks per starting lane
  const int lane = threadIdx.x & 31;
  const int wbase = threadIdx.x & ~31;
  const unsigned sm = __ballot_sync(kAll, want);
  if (want) sl[wbase + __popc(sm & ((1u << lane) - 1u))] = lane;
  __syncwarp();
  const double* X = want ? m.coords + (int64_t)e * NN : m.coords;
  const int64_t cs = m.cstride;
  const int total = __popc(sm) * NT;
  for (int t0 = 0; t0 < total; t0 += 32) {  // warp-uniform trip count
    const int t = t0 + lane;
    const bool act = t < total;
    const int si = act ? t / NT : 0;
    const int src = act ? sl[wbase + si] : lane;
    const double* Xs = reinterpret_cast<const double*>(
        __shfl_sync(kAll, reinterpret_cast<unsigned long long>(X), src));
    const int64_t css = __shfl_sync(kAll, (long long)cs, src);
    const int nbs = __shfl_sync(kAll, nb, src);
    if (act) {
      const int ent = t - si * NT;  // = c * DR + j, the entry of G
      const int c = ent / DR, j = ent - c * DR;
      const int idx = j == 0 ? nbs % N : (j == 1 ? (nbs / N) % N : nbs / (N * N));
      const int st = j == 0 ? 1 : (j == 1 ? N : N * N);
      const double* line = Xs + c * css + (nbs - idx * st);
      const double* row = dn + idx * N;
      double g = 0.0;
#pragma unroll
      for (int k = 0; k < N; ++k) g = fma(__ldg(line + k * st), row[k], g);
      sg[ent * kFindThreads + wbase + src] = g;
    }
  }
  __syncwarp();
  if (want) {
#pragma unroll
    for (int c = 0; c < D; ++c) x[c] = __ldg(X + c * cs + nb);
#pragma unroll
    for (int q = 0; q < NT; ++q) G[q] = sg[q * kFindThreads + threadIdx.x];
  }
}

template <int D>
__device__ __forceinline__ double aabb_scale(const DevMesh& m, int64_t e) {
  double X = 0.0;
#pragma unroll
  for (int c = 0; c < 2 * D; ++c) X = fmax(X, fabs(__ldg(m.aabb + e * 2 * D + c)));
  return X;
}

// Psi_L cell of x, or -1 when x lies outside the grid (then outside every
// AABB) or has a non-finite coordinate.
template <int D>
__device__ __forceinline__ int64_t point_cell(const DevMesh& m, const double (&xs)[D]) {
  int64_t cell = 0, mul = 1;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    if (!(xs[c] >= m.lo[c] && xs[c] <= m.hi[c])) return -1;
    cell += mul * cell_coord(xs[c], m.lo[c], m.scale[c], m.NL);
    mul *= m.NL;
  }
  return cell;
}

template <int DR>
__device__ __forceinline__ void write_result(int64_t p, int code_, int e, const double (&r)[DR],
                                             double d2, int* __restrict__ code, int* __restrict__ elem,
                                             double* __restrict__ rout, double* __restrict__ dist2) {
  code[p] = code_;
  elem[p] = e;
#pragma unroll
  for (int j = 0; j < DR; ++j) rout[p * DR + j] = r[j];
  dist2[p] = d2;
}

// ---- the trust-region step of Sec. 3.2.1 ------------------------------------

// |v| == 1, |v| < 1 and the sign of v from the bit pattern, on the integer
// pipe (the FP64 one is the kernels' bound): exact for every value, NaN
// included (neither test holds for it), -0 included (|-0| < 1).
__device__ __forceinline__ bool is_unit(double v) {
  return (__double_as_longlong(v) & 0x7fffffffffffffffLL) == 0x3ff0000000000000LL;
}
__device__ __forceinline__ bool is_unit(float v) { return (__float_as_int(v) & 0x7fffffff) == 0x3f800000; }
__device__ __forceinline__ bool below_unit(double v) {
  return (__double_as_longlong(v) & 0x7fffffffffffffffLL) < 0x3ff0000000000000LL;
}
__device__ __forceinline__ bool below_unit(float v) { return (__float_as_int(v) & 0x7fffffff) < 0x3f800000; }
__device__ __forceinline__ bool sign_bit(double v) { return __double_as_longlong(v) < 0; }
__device__ __forceinline__ bool sign_bit(float v) { return __float_as_int(v) < 0; }

// r_j = -1 with the gradient pointing out (g > 0), or r_j = +1 with g < 0.
template <typename T>
__device__ __forceinline__ bool held_at_bound(T r, T g) {
  return is_unit(r) && (sign_bit(r) ? is_pos(g) : is_neg(g));
}

template <int DR, typename T>
__device__ __forceinline__ bool at_bound(const T (&r)[DR]) {
  bool b = false;
#pragma unroll
  for (int j = 0; j < DR; ++j) b |= is_unit(r[j]);
  return b;
}

// Solves H_FF s_F = -g_F on the free coordinates (held ones get s = 0): the
// held rows and columns are replaced by the identity, which leaves the free
// block's leading minors unchanged.
template <int DR, typename T>
__device__ __forceinline__ bool masked_solve(const T (&H)[DR][DR], const bool (&held)[DR],
                                             const T (&g)[DR], T (&s)[DR]) {
  T A[DR][DR], b[DR];
#pragma unroll
  for (int j = 0; j < DR; ++j) {
#pragma unroll
    for (int k = 0; k < DR; ++k)
      A[j][k] = (held[j] || held[k]) ? (j == k ? T(1) : T(0)) : H[j][k];
    b[j] = held[j] ? T(0) : -g[j];
  }
  if (!spd_solve<DR, T>(A, b, s)) return false;
#pragma unroll
  for (int j = 0; j < DR; ++j)
    if (held[j]) s[j] = T(0);
  return true;
}

// Shared-memory slabs for the t-direction basis values of every thread of
// the CTA (hexes only): 3N slots of kFindThreads values.
template <int N, typename T>
struct TSlots {
  T* base;
  __device__ __forceinline__ Slots<T> slot(int which) const { return Slots<T>{base + which * N * kFindThreads, kFindThreads}; }
};

// x(re) and, if WANT_G, G(re) of element data X (rows at pitch P): the
// uniform evaluation site.
template <int N, int D, int DR, bool WANT_G, typename T, int P = N>
__device__ __forceinline__ void eval_xG(const T* __restrict__ X, int64_t cs, const BasisTab& B,
                                        const T (&re)[DR], const TSlots<N, T>& ts, T* x, T* G) {
  T ph[3][N], dph[3][N];
#pragma unroll
  for (int j = 0; j < DR; ++j) {
    if constexpr (WANT_G) {
      lagrange_sym<N, T>(B, re[j], ph[j], dph[j]);
    } else {
      lagrange_sym_values<N, T>(B, re[j], ph[j]);
#pragma unroll
      for (int i = 0; i < N; ++i) dph[j][i] = T(0);
    }
  }
  if constexpr (DR == 3) {
    const Slots<T> pt = ts.slot(0), dpt = ts.slot(1);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      pt(k) = ph[2][k];
      dpt(k) = dph[2][k];
    }
    map_eval_rolled<N, D, WANT_G, T, P>(X, cs, ph, dph, pt, dpt, x, G);
  } else {
    T ph2[DR][N], dph2[DR][N];
#pragma unroll
    for (int j = 0; j < DR; ++j)
#pragma unroll
      for (int i = 0; i < N; ++i) {
        ph2[j][i] = ph[j][i];
        dph2[j][i] = dph[j][i];
      }
    map_eval<N, DR, D, WANT_G, T, P>(X, cs, ph2, dph2, x, G);
  }
}

// Gradient g = -G^T dx, held set, Hessian G^T G - beta HS, masked solve with
// the fallbacks (beta = 0 block, then no step), clip to [-alpha, alpha] and
// projection on [-1,1].  Returns |dr|_inf of the projected step.
template <int D, int DR, typename T>
__device__ __forceinline__ T newton_step(const T (&G)[D * DR], const T (&dx)[D], const T (&r)[DR],
                                         T alpha, bool beta, const T (&HS)[DR][DR], T (&rn)[DR],
                                         T (&ds)[DR], bool& clipped, bool& used_beta) {
  T g[DR], HGN[DR][DR], H[DR][DR], step[DR];
  bool held[DR];
#pragma unroll
  for (int j = 0; j < DR; ++j) {
    T s = T(0);
#pragma unroll
    for (int c = 0; c < D; ++c) s -= G[c * DR + j] * dx[c];
    g[j] = s;
    held[j] = held_at_bound(r[j], s);
  }
#pragma unroll
  for (int j = 0; j < DR; ++j)
#pragma unroll
    for (int k = j; k < DR; ++k) {  // G^T G is symmetric: the upper triangle, mirrored
      T s = T(0);
#pragma unroll
      for (int c = 0; c < D; ++c) s += G[c * DR + j] * G[c * DR + k];
      HGN[j][k] = HGN[k][j] = H[j][k] = H[k][j] = s;
    }
  if (beta) {  // a branch of its own: skipped by warps where no lane holds beta
#pragma unroll
    for (int j = 0; j < DR; ++j)
#pragma unroll
      for (int k = j; k < DR; ++k) H[j][k] = H[k][j] = HGN[j][k] - HS[j][k];
  }
  used_beta = beta;
  bool ok = masked_solve<DR, T>(H, held, g, step);
  if (!ok && beta) {
    used_beta = false;
    ok = masked_solve<DR, T>(HGN, held, g, step);
  }
  if (!ok) {
    used_beta = false;
#pragma unroll
    for (int j = 0; j < DR; ++j) step[j] = T(0);
  }
  // clip and projection with the bit-pattern tests (alpha > 0), and for
  // double |dr|_inf as the largest magnitude's bit pattern (a NaN ignored,
  // as fmax ignores it)
  using FB = FBits<T>;
  typename FB::I mx = 0;
  T mxf = T(0);
  clipped = false;
#pragma unroll
  for (int j = 0; j < DR; ++j) {
    T s = step[j];
    if (above_nonneg(s, alpha)) {
      s = alpha;
      clipped = true;
    }
    if (above_nonneg(-s, alpha)) {
      s = -alpha;
      clipped = true;
    }
    T v = r[j] + s;
    if (above_nonneg(v, T(1))) v = T(1);
    if (above_nonneg(-v, T(1))) v = T(-1);
    rn[j] = v;
    ds[j] = v - r[j];
    if constexpr (std::is_same_v<T, float>) {
      mxf = fmaxf(mxf, fabsf(ds[j]));
    } else {
      const auto a = FB::of(ds[j]) & FB::kAbs;
      if (a <= FB::kInf && a > mx) mx = a;
    }
  }
  if constexpr (std::is_same_v<T, float>) return mxf;
  return FB::from(mx);
}

// -2 g.dr - dr^T H dr with H = G^T G (beta = 0: the same value as
// |dx|^2 - |dx - G dr|^2) or G^T G - HS (beta = 1).
template <int D, int DR, typename T>
__device__ __forceinline__ T predicted_decrease(const T (&G)[D * DR], const T (&dx)[D], const T (&ds)[DR],
                                                bool used_beta, const T (&HS)[DR][DR]) {
  T lin = T(0), quad = T(0);
#pragma unroll
  for (int c = 0; c < D; ++c) {
    T gd = T(0);
#pragma unroll
    for (int j = 0; j < DR; ++j) gd += G[c * DR + j] * ds[j];
    lin -= gd * dx[c];  // g.ds with g = -G^T dx
    quad += gd * gd;
  }
  if (used_beta) {
#pragma unroll
    for (int j = 0; j < DR; ++j)
#pragma unroll
      for (int k = 0; k < DR; ++k) quad -= ds[j] * HS[j][k] * ds[k];
  }
  return T(-2) * lin - quad;
}

// |dx - G dr|^2: the distance after the last (sub-tolerance) step.
template <int D, int DR, typename T>
__device__ __forceinline__ T model_dist2(const T (&G)[D * DR], const T (&dx)[D], const T (&ds)[DR]) {
  T f = T(0);
#pragma unroll
  for (int c = 0; c < D; ++c) {
    T t = dx[c];
#pragma unroll
    for (int j = 0; j < DR; ++j) t -= G[c * DR + j] * ds[j];
    f += t * t;
  }
  return f;
}

// Certified stop of the FP64 iteration (volumes, D == DR).  The iteration
// of Sec. 3.2.1 stops once its proposed step is below the Newton tolerance;
// the full evaluation of x and G after the step before it serves only to
// compute that last, sub-tolerance step.  Here the next step is bounded
// instead, from quantities at hand, and the iteration stops at r' = r + s
// when the bound leaves nothing the last step would still correct:
//   * the exact residual at r' is e' = (dx - G s) - R, |R|_inf <= L |s|^2 / 2
//     with L the element's bound on sum_jk |d2 x_c / dr_j dr_k| (setup:
//     DevMesh::curv); dx - G s is the linear model's residual t, computed
//     here with rounding <= 4u (|dx| + |G| |s|), and dx itself carries the
//     evaluation's rounding, covered by 1e-14 X (X the element's coordinate
//     scale);
//   * |G(r')^-1|_inf <= g / (1 - g L |s|), g = |G^-1|_inf (adjugate / det,
//     widened by 1e-6 for its own rounding), by the Banach lemma, since
//     |G(r') - G(r)|_inf <= L |s|;
//   * so with q = g L |s| < 1 the next step, and the distance from r' to the
//     root the iteration converges to (the later steps shrink
//     quadratically), are at most g (|t| + slack + L |s|^2 / 2) / (1 - q)
//     (1 + q'), q' tiny (covered by the widening of g).
// Certified when (a) that bound without the evaluation's rounding is at
// most kF64CertModel: the stop then moves r by no more than the rounding
// noise the full iteration's last step carries as well, so r, dist2 and the
// interpolated values agree with the full iteration's to its own accuracy;
// (b) the whole bound is at most kF64CertStep (half the tolerance); and
// (c) every |r'_j| < 1 - kCertEdge, so the code (INTERIOR) is the full
// iteration's.  Both tests are done without a division, as
// g_num (num + k L |s|) <= k |det|.  On success the step is taken and dist2
// is the model value |t|^2, as for a sub-tolerance step.  The caller passes
// only unclipped, beta-free steps of an iterate off the element boundary.
constexpr double kF64CertModel = 2e-15;
constexpr double kF64CertStep = 5e-11;
constexpr double kCertEdge = 1e-10;
constexpr double kCertMaxStep = 1e-4;  // larger steps are not tried (g L |s|^2 >> kF64CertModel on curved elements)

template <int D>
__device__ __forceinline__ bool certified_stop(const double (&G)[D * D], const double (&dx)[D], const double (&ds)[D],
                                               const double (&rn)[D], double mx, float curv, double xscale,
                                               double& F) {
  using FB = FBits<double>;
  // |r'_j| < 1 - kCertEdge, on the bit patterns
  constexpr long long kEdge = 0x3feffffffff24190LL;  // the bits of 1 - kCertEdge (0.9999999999)
  bool in = true;
#pragma unroll
  for (int j = 0; j < D; ++j) in &= (FB::of(rn[j]) & FB::kAbs) < kEdge;
  if (!in) return false;
  // adjugate of G (row-major, G[c * D + j]), det, row sums of |adj| and |G|
  double adj[D * D], det;
  if constexpr (D == 2) {
    adj[0] = G[3];
    adj[1] = -G[1];
    adj[2] = -G[2];
    adj[3] = G[0];
    det = G[0] * G[3] - G[1] * G[2];
  } else {
    adj[0] = G[4] * G[8] - G[5] * G[7];
    adj[1] = G[2] * G[7] - G[1] * G[8];
    adj[2] = G[1] * G[5] - G[2] * G[4];
    adj[3] = G[5] * G[6] - G[3] * G[8];
    adj[4] = G[0] * G[8] - G[2] * G[6];
    adj[5] = G[2] * G[3] - G[0] * G[5];
    adj[6] = G[3] * G[7] - G[4] * G[6];
    adj[7] = G[1] * G[6] - G[0] * G[7];
    adj[8] = G[0] * G[4] - G[1] * G[3];
    det = G[0] * adj[0] + G[1] * adj[3] + G[2] * adj[6];
  }
  long long arow = 0, grow = 0, tmax = 0, dmax = 0;
  double t[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double a = 0.0, b = 0.0, ti = dx[i];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      a += fabs(adj[i * D + j]);
      b += fabs(G[i * D + j]);
      ti = fma(-G[i * D + j], ds[j], ti);
    }
    t[i] = ti;
    arow = max(arow, FB::of(a));
    grow = max(grow, FB::of(b));
    tmax = max(tmax, FB::of(ti) & FB::kAbs);
    dmax = max(dmax, FB::of(dx[i]) & FB::kAbs);
  }
  const double adet = fabs(det);
  const double an = FB::from(arow) * (1.0 + 1e-6);  // g = an / adet
  const double L = (double)curv;
  const double Ls = L * mx;
  constexpr double u4 = 4.0 * 1.1102230246251565e-16;
  const double num = FB::from(tmax) + fma(u4, fma(FB::from(grow), mx, FB::from(dmax)), 0.5 * Ls * mx);
  // g num / (1 - q) <= k with g = an / |det|, q = g L |s| (which the
  // inequalities also hold below 1)
  if (!(an * fma(kF64CertModel, Ls, num) <= kF64CertModel * adet)) return false;
  if (!(an * fma(kF64CertStep, Ls, fma(1e-14, xscale, num)) <= kF64CertStep * adet)) return false;
  double f = 0.0;
#pragma unroll
  for (int c = 0; c < D; ++c) f = fma(t[c], t[c], f);
  F = f;
  return true;
}

// Ratio test of Sec. 3.2.1 with the rounding-level acceptance; updates alpha.
template <typename T>
__device__ __forceinline__ bool trial_accepts(T F, T Fn, T pred, bool clipped, T xscale, T& alpha,
                                              T tau_factor = T(1e-12)) {
  const T decr = F - Fn;
  const T tau = tau_factor * xscale * sqrt(F);
  if (!clipped && pred < tau) return true;
  if (decr >= T(0.9) * pred) {
    alpha *= T(2);
    return true;
  }
  if (decr >= T(0.01) * pred) return true;
  alpha *= T(0.25);
  return false;
}

// ---- sources of work: one mesh, or a batch of (mesh, points) items ---------

// One mesh; the point sequence is pts[0..n) or pts[pidx[0..n)].  The
// "global" index of a point (what the mixed path queues) is its index.
template <int D, int DR>
struct SingleWork {
  const DevMesh* mesh;
  const double* pts;
  const int* pidx;
  int64_t n;
  int* code;
  int* elem;
  double* r;
  double* dist2;
  int clog2;  // a CTA takes 2^clog2 consecutive points per chunk
  __device__ __forceinline__ const DevMesh* first() const { return mesh; }
  __device__ __forceinline__ void locate(int64_t g, const DevMesh*& m, int& item, int64_t& p) const {
    m = mesh;
    item = 0;
    p = pidx ? (int64_t)__ldg(pidx + g) : g;
  }
  __device__ __forceinline__ void load(int, int64_t p, double (&xs)[D]) const {
#pragma unroll
    for (int c = 0; c < D; ++c) xs[c] = __ldg(pts + p * D + c);
  }
  __device__ __forceinline__ void write(int, int64_t p, int c, int e, const double (&rr)[DR], double d2) const {
    write_result<DR>(p, c, e, rr, d2, code, elem, r, dist2);
  }
  __device__ __forceinline__ int64_t global(int, int64_t p) const { return p; }
  // the CTAs that share the point sequence in chunks, and this CTA's index
  __device__ __forceinline__ int64_t ctas() const { return gridDim.x; }
  __device__ __forceinline__ int64_t cta() const { return blockIdx.x; }
};

// One (mesh, points, outputs) item of a batch; `start` is the index of its
// first point in the batch's global point sequence (items in order).
struct BatchItem {
  DevMesh m;
  const double* pts;
  int64_t n;
  int64_t start;
  int* code;
  int* elem;
  double* r;
  double* dist2;
  const double* field;
  int nc;
  double* out;        // [nc] components, component c at out + c * ld
  int64_t ld;
  int64_t key_base;   // first of this item's order keys (order_keys of its mesh) in the batch's order
  const float2* fs;   // FP_MIXED double-float interpolation: the field as (hi, lo) pairs, or NULL
  const int* fexp;    // ... and its components' scaling exponents
};

// A batch of items of one element shape; the point sequence is the items'
// points in order, or the global indices gidx[0..n).
template <int D, int DR>
struct BatchWork {
  const BatchItem* items;
  int nitems;
  const int* gidx;
  int64_t n;
  int clog2;
  __device__ __forceinline__ const DevMesh* first() const { return &items[0].m; }
  __device__ __forceinline__ void locate(int64_t g, const DevMesh*& m, int& item, int64_t& p) const {
    const int64_t gg = gidx ? (int64_t)__ldg(gidx + g) : g;
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {  // last item with start <= gg
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].start <= gg) lo = mid;
      else hi = mid - 1;
    }
    item = lo;
    m = &items[lo].m;
    p = gg - items[lo].start;
  }
  __device__ __forceinline__ void load(int item, int64_t p, double (&xs)[D]) const {
    const double* pts = items[item].pts;
#pragma unroll
    for (int c = 0; c < D; ++c) xs[c] = __ldg(pts + p * D + c);
  }
  __device__ __forceinline__ void write(int item, int64_t p, int c, int e, const double (&rr)[DR], double d2) const {
    const BatchItem& it = items[item];
    write_result<DR>(p, c, e, rr, d2, it.code, it.elem, it.r, it.dist2);
  }
  __device__ __forceinline__ int64_t global(int item, int64_t p) const { return items[item].start + p; }
  __device__ __forceinline__ int64_t ctas() const { return gridDim.x; }
  __device__ __forceinline__ int64_t cta() const { return blockIdx.x; }
};

// A tile of a batch class: points base .. base + n - 1 of the class's point
// sequence, searched by one CTA alone (the fused launch, batch_fused.cu).
template <int D, int DR>
struct TileWork : BatchWork<D, DR> {
  int64_t base;
  __device__ __forceinline__ void locate(int64_t g, const DevMesh*& m, int& item, int64_t& p) const {
    BatchWork<D, DR>::locate(base + g, m, item, p);
  }
  __device__ __forceinline__ int64_t ctas() const { return 1; }
  __device__ __forceinline__ int64_t cta() const { return 0; }
};

// A class (element shape) of a batch as the fused launch sees it
// (batch_fused.cu), and a tile of one class's point sequence.
struct FusedClass {
  const BatchItem* items;
  int nitems;
  int shape;          // shape_of(N, d, dr)
  const int* order;   // the class's point order (global indices), or null
  int* queue;         // FP_MIXED: the class's hand-over queue and its counter
  int* qcount;
  BasisTab B;
};
struct FusedTile {
  int cls;
  int n;
  int64_t base;
};
// CTAs per SM of the fused launch: its register budget is that of the
// costliest shape (hexes of order 6 and 7 need more than a third of the
// register file per CTA of 128 threads).
constexpr int kFusedCtas = 2;
int shape_of(int N, int d, int dr);
// One persistent launch over all tiles (counter zeroed by the caller).
int launch_fused(const FusedClass* classes, const FusedTile* tiles, int ntiles, int* counter, int precision,
                 int* status, cudaStream_t st);
// FP_MIXED, one element shape of a batch: the FP64 kernel over the queued
// global indices only (the launch_batch_class follow-up).
int launch_batch_follow(const BatchItem* items, int nitems, int64_t total, int N, int d, int dr,
                        const BasisTab& B, int* queue, int* qcount, cudaStream_t st);

int find_f64(const fp_mesh_s* m, const double* pts, const int* pidx, int64_t n, int* code,
             int* elem, double* r, double* dist2, unsigned long long* stats, cudaStream_t st);
// The two launches of the mixed path; with mid given and the mesh's timer
// on, *mid is a timing event recorded between them.
int launch_mixed_with_queue(const fp_mesh_s* m, const double* pts, const int* pidx, int64_t n, int* code,
                            int* elem, double* r, double* dist2, int* queue, int* qcount,
                            unsigned long long* stats, cudaStream_t st, cudaEvent_t* mid = nullptr);
// One element shape of a batch (find_mixed.cu): the find kernel(s) over
// all items; order (may be NULL) is the batch cell order of the points.
int launch_batch_class(const BatchItem* items, int nitems, int64_t total, int N, int d, int dr,
                       const BasisTab& B, int precision, int ctas_per_sm, int clog2, const int* order,
                       int* queue, int* qcount, unsigned long long* stats, cudaStream_t st);
// Cell-grouped point order (order.cu): scratch of cell_order_ints ints;
// *perm points into it.  order_keys: the keys a mesh takes per cost class.
int64_t order_keys(const fp_mesh_s* m);
int64_t cell_order_ints(const fp_mesh_s* m, int64_t n);
int cell_order(const fp_mesh_s* m, const double* pts, int64_t n, int* scratch, int** perm, cudaStream_t st);
// The same for one element shape of a batch: the points of all items grouped
// by cost class, then (item, first candidate element); buckets = sum over
// items of order_keys, with each item's key_base set; scratch of
// batch_cell_order_ints(total, buckets) ints.
int64_t batch_cell_order_ints(int64_t total, int64_t buckets);
int batch_cell_order(const BatchItem* items, int nitems, int64_t total, int d, int64_t buckets, int* scratch,
                     int** perm, cudaStream_t st);

}  // namespace fp
