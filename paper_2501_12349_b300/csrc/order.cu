// Element-grouped traversal of the query points.
//
// The paper notes (Sec. 3.2, on the CPU implementation) that handling the
// points of one element together improves memory locality.  On this GPU the
// find kernels read each candidate element's coordinates (125 nodes x 3
// components at p = 4) once per Newton evaluation; with points in random
// order the lanes of a warp touch 32 different elements and the L1 serves
// one access per lane.  Grouping the points by the first candidate element
// that the find kernels will search (found through the point's Psi_L cell
// and the FP32 box test) makes the lanes of a warp share that element, so
// its reads become broadcasts.  The result of each point does not depend on
// the order, so the outputs are bit-identical to those of the unordered
// traversal.
//
// The order is a counting sort by key (cost class, element): one pass
// computes each point's key (points outside the grid, or with non-finite
// coordinates, take the last key) and counts the keys, a scan gives the
// bucket starts, and a second pass scatters the point indices.  The order
// within a bucket is whatever the atomics give; it affects only which lane
// handles a point, as do the keys themselves, which are computed in FP32 (a
// point on a box face may land in a neighbouring bucket).
#include "find_common.cuh"

namespace fp {

namespace {

constexpr int kCostClasses = 4;  // candidates 3+, 2, 1, 0

// The order only decides which lane handles a point, so its buckets may be
// computed approximately: in FP32, from each coordinate truncated to FP32
// on the integer pipe (conversions from FP64 run at the FP64 pipe's rate
// on this GPU, a small fraction of FP32's).  Non-finite values become NaN,
// magnitudes beyond FP32 infinity, tiny ones zero.
__device__ __forceinline__ float trunc_to_float(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  if (e == 0x7ff) return __int_as_float(0x7fc00000);
  const int fe = e - 1023 + 127;
  if (fe >= 255) return __int_as_float((int)(sign | 0x7f800000u));
  if (fe <= 0) return __int_as_float((int)sign);
  return __int_as_float((int)(sign | ((unsigned)fe << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29)));
}

// Psi_L cell of x (x32 its FP32 copy) in FP32 arithmetic, or -1 outside
// the grid (or not finite): close to point_cell, which decides candidates.
template <int D>
struct CellF32 {
  float lo[D], hi[D], scale[D];
  int NL;
  __device__ __forceinline__ explicit CellF32(const DevMesh& m) : NL(m.NL) {
#pragma unroll
    for (int c = 0; c < D; ++c) {
      lo[c] = (float)m.lo[c];
      hi[c] = (float)m.hi[c];
      scale[c] = (float)m.scale[c];
    }
  }
  __device__ __forceinline__ int64_t operator()(const float (&x)[D]) const {
    int64_t cell = 0, mul = 1;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      if (!(x[c] >= lo[c] && x[c] <= hi[c])) return -1;
      const int k = (int)floorf((x[c] - lo[c]) * scale[c]);
      cell += mul * (k < 0 ? 0 : (k >= NL ? NL - 1 : k));
      mul *= NL;
    }
    return cell;
  }
};

// Bucket of a point: its cost class, then its first candidate element.
// The class counts the candidate elements whose boxes may hold the point
// (the FP32 box test, undecided cases counted), 3 or more first: every
// candidate but the last costs a Newton run, so points with many candidates
// are the slow ones, and taking them first leaves cheap points for the end
// of the launch, where lanes that run out of points wait for the slowest of
// their warp.  Within a class the points are grouped by the first candidate
// (the element the find kernels search first, in Psi_L's ascending order),
// so the lanes of a warp mostly evaluate the same element and its
// coordinates are read once for all of them.  Key = class * (NE + 1) +
// element (NE: no candidate); points outside the grid take the last key.
template <int D>
__device__ __forceinline__ int order_key(const DevMesh& m, const float (&x32)[D], int64_t nkeys) {
  const int64_t cell = CellF32<D>(m)(x32);
  if (cell < 0) return (int)(kCostClasses * nkeys - 1);
  int cand = 0, first = (int)(nkeys - 1);
  const int q0 = __ldg(m.cell_start + cell), q1 = __ldg(m.cell_start + cell + 1);
  for (int q = q0; q < q1 && cand < kCostClasses - 1; ++q) {
    const int el = __ldg(m.cell_elems + q);
    if (boxes_f32<D>(m.box32 + (int64_t)el * BOX32, x32) != 0) {
      if (cand == 0) first = el;
      ++cand;
    }
  }
  return (int)((kCostClasses - 1 - cand) * nkeys + first);
}

template <int D>
__global__ void __launch_bounds__(256)
    k_point_cells(const __grid_constant__ DevMesh m, int64_t nkeys, const double* __restrict__ pts, int64_t n,
                  int* __restrict__ cellof, int* __restrict__ counts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float x32[D];
#pragma unroll
    for (int c = 0; c < D; ++c) x32[c] = trunc_to_float(__ldg(pts + i * D + c));
    const int k = order_key<D>(m, x32, nkeys);
    cellof[i] = k;
    atomicAdd(counts + k, 1);
  }
}

__global__ void __launch_bounds__(256)
    k_point_scatter(const int* __restrict__ cellof, int64_t n, const int* __restrict__ start,
                    int* __restrict__ cursor, int* __restrict__ perm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int k = cellof[i];
    perm[start[k] + atomicAdd(cursor + k, 1)] = (int)i;
  }
}

template <int D>
__global__ void __launch_bounds__(256)
    k_batch_point_cells(const BatchItem* __restrict__ items, int nitems, int64_t total, int64_t buckets,
                        int* __restrict__ key, int* __restrict__ counts) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {  // last item with start <= g
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].start <= g) lo = mid;
      else hi = mid - 1;
    }
    const BatchItem& it = items[lo];
    const int64_t p = g - it.start;
    float x32[D];
#pragma unroll
    for (int c = 0; c < D; ++c) x32[c] = trunc_to_float(__ldg(it.pts + p * D + c));
    // the item's key in [0, kCostClasses * (NE + 1)), as in k_point_cells,
    // spread over the batch: class * buckets + the item's base + element
    const int64_t nk = it.m.NE + 1;
    const int k1 = order_key<D>(it.m, x32, nk);
    const int64_t cls = k1 / nk, el = k1 - cls * nk;
    const int k = (int)(cls * buckets + it.key_base + el);
    key[g] = k;
    atomicAdd(counts + k, 1);
  }
}

// Exclusive scan of counts[0, n) into start[0, n], start[n] = total, over
// tiles of kScanTile elements: each CTA scans its tile and writes the tile's
// total; one CTA scans the tile totals; a last pass adds each tile's offset.
constexpr int kScanThreads = 512, kScanItems = 8, kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads)
    k_scan_tiles(const int* __restrict__ counts, int64_t n, int* __restrict__ start, int* __restrict__ tile_sum) {
  __shared__ int s[kScanThreads];
  const int t = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)t * kScanItems;
  int v[kScanItems], sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? counts[base + k] : 0;
    sum += v[k];
  }
  s[t] = sum;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {
    const int add = t >= o ? s[t - o] : 0;
    __syncthreads();
    s[t] += add;
    __syncthreads();
  }
  int run = s[t] - sum;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) start[base + k] = run;
    run += v[k];
  }
  if (t == kScanThreads - 1) tile_sum[blockIdx.x] = s[t];
}

__global__ void __launch_bounds__(kScanThreads)
    k_scan_add(int* __restrict__ start, int64_t n, const int* __restrict__ tile_pre, int64_t ntiles) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  const int off = tile_pre[blockIdx.x];
  for (int k = threadIdx.x; k < kScanTile; k += kScanThreads)
    if (base + k < n) start[base + k] += off;
  if (blockIdx.x == 0 && threadIdx.x == 0) start[n] = tile_pre[ntiles];
}

int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

// scratch: 2 scan_tiles(n) + 1 ints
int exclusive_scan(const int* counts, int64_t n, int* start, int* scratch, cudaStream_t st) {
  const int64_t nt = scan_tiles(n);
  int* tsum = scratch;
  int* tpre = scratch + nt;
  k_scan_tiles<<<(unsigned)nt, kScanThreads, 0, st>>>(counts, n, start, tsum);
  k_scan<<<1, 1024, 0, st>>>(tsum, nt, tpre);
  k_scan_add<<<(unsigned)nt, kScanThreads, 0, st>>>(start, n, tpre, nt);
  FP_CUDA_TRY(cudaGetLastError());
  return FP_OK;
}

}  // namespace

int64_t batch_cell_order_ints(int64_t total, int64_t buckets) {
  const int64_t nb = kCostClasses * buckets;
  return 2 * total + 2 * nb + 1 + 2 * scan_tiles(nb) + 1;
}

int batch_cell_order(const BatchItem* items, int nitems, int64_t total, int d, int64_t buckets, int* scratch,
                     int** perm, cudaStream_t st) {
  const int64_t nb = kCostClasses * buckets;  // cost class x (items' keys)
  int* p = scratch;          // [total]
  int* key = p + total;      // [total]
  int* counts = key + total; // [nb]
  int* start = counts + nb;  // [nb + 1]
  int* sc = start + nb + 1;  // scan scratch
  FP_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)nb, st));
  const int blocks = (int)((total + 255) / 256 < 8 * 148 ? (total + 255) / 256 : 8 * 148);
  if (d == 2)
    k_batch_point_cells<2><<<blocks, 256, 0, st>>>(items, nitems, total, buckets, key, counts);
  else
    k_batch_point_cells<3><<<blocks, 256, 0, st>>>(items, nitems, total, buckets, key, counts);
  FP_TRY(exclusive_scan(counts, nb, start, sc, st));
  FP_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)nb, st));
  k_point_scatter<<<blocks, 256, 0, st>>>(key, total, start, counts, p);
  FP_CUDA_TRY(cudaGetLastError());
  *perm = p;
  return FP_OK;
}

int64_t order_keys(const fp_mesh_s* m) { return m->NE + 1; }

int64_t cell_order_ints(const fp_mesh_s* m, int64_t n) {
  const int64_t nb = kCostClasses * order_keys(m);
  return 2 * n + 2 * nb + 1 + 2 * scan_tiles(nb) + 1;
}

int cell_order(const fp_mesh_s* m, const double* pts, int64_t n, int* scratch, int** perm, cudaStream_t st) {
  const int64_t nb = kCostClasses * order_keys(m);  // buckets: cost class x (elements and "none")
  int* p = scratch;                  // [n]
  int* cellof = p + n;               // [n]
  int* counts = cellof + n;          // [nb], reused as the scatter cursors
  int* start = counts + nb;          // [nb + 1]
  int* sc = start + nb + 1;          // scan scratch
  FP_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)nb, st));
  const DevMesh v = m->view();
  const int blocks = (int)((n + 255) / 256 < 8 * 148 ? (n + 255) / 256 : 8 * 148);
  if (m->d == 2)
    k_point_cells<2><<<blocks, 256, 0, st>>>(v, order_keys(m), pts, n, cellof, counts);
  else
    k_point_cells<3><<<blocks, 256, 0, st>>>(v, order_keys(m), pts, n, cellof, counts);
  FP_TRY(exclusive_scan(counts, nb, start, sc, st));
  FP_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)nb, st));
  k_point_scatter<<<blocks, 256, 0, st>>>(cellof, n, start, counts, p);
  FP_CUDA_TRY(cudaGetLastError());
  *perm = p;
  return FP_OK;
}

}  // namespace fp
