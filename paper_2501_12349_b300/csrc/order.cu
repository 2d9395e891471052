// Cell-grouped traversal of the query points.
//
// The paper notes (Sec. 3.2, on the CPU implementation) that handling the
// points of one element together improves memory locality.  On this GPU the
// find kernels read each candidate element's coordinates (125 nodes x 3
// components x 8 B at p = 4) once per Newton evaluation; with points in
// random order the lanes of a warp touch 32 different elements and most of
// those reads miss L1.  Grouping the points by their Psi_L cell makes the
// lanes of a warp share candidate elements, so the reads become broadcasts
// that hit L1.  The result of each point does not depend on the order, so
// the outputs are bit-identical to those of the unordered traversal.
//
// The order is a counting sort by cell: one pass computes each point's cell
// (points outside the grid, or with non-finite coordinates, go to an extra
// last bucket) and counts the cells, a scan gives the bucket starts, and a
// second pass scatters the point indices.  The order within a bucket is
// whatever the atomics give; it affects only which lane handles a point.
#include "find_common.cuh"

namespace fp {

namespace {

template <int D>
__global__ void __launch_bounds__(256)
    k_point_cells(const __grid_constant__ DevMesh m, int64_t ncell, const double* __restrict__ pts, int64_t n,
                  int* __restrict__ cellof, int* __restrict__ counts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double xs[D];
#pragma unroll
    for (int c = 0; c < D; ++c) xs[c] = __ldg(pts + i * D + c);
    const int64_t cell = point_cell<D>(m, xs);
    const int k = cell < 0 ? (int)ncell : (int)cell;
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
    k_batch_point_cells(const BatchItem* __restrict__ items, int nitems, int64_t total, int* __restrict__ key,
                        int* __restrict__ counts) {
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
    double xs[D];
#pragma unroll
    for (int c = 0; c < D; ++c) xs[c] = __ldg(it.pts + p * D + c);
    int64_t ncell = 1;
#pragma unroll
    for (int c = 0; c < D; ++c) ncell *= it.m.NL;
    const int64_t cell = point_cell<D>(it.m, xs);
    const int k = (int)(it.cell_base + (cell < 0 ? ncell : cell));
    key[g] = k;
    atomicAdd(counts + k, 1);
  }
}

}  // namespace

int batch_cell_order(const BatchItem* items, int nitems, int64_t total, int d, int64_t buckets, int* scratch,
                     int** perm, cudaStream_t st) {
  int* p = scratch;               // [total]
  int* key = p + total;           // [total]
  int* counts = key + total;      // [buckets]
  int* start = counts + buckets;  // [buckets + 1]
  FP_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)buckets, st));
  const int blocks = (int)((total + 255) / 256 < 8 * 148 ? (total + 255) / 256 : 8 * 148);
  if (d == 2)
    k_batch_point_cells<2><<<blocks, 256, 0, st>>>(items, nitems, total, key, counts);
  else
    k_batch_point_cells<3><<<blocks, 256, 0, st>>>(items, nitems, total, key, counts);
  k_scan<<<1, 1024, 0, st>>>(counts, buckets, start);
  FP_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)buckets, st));
  k_point_scatter<<<blocks, 256, 0, st>>>(key, total, start, counts, p);
  FP_CUDA_TRY(cudaGetLastError());
  *perm = p;
  return FP_OK;
}

int64_t cell_order_ints(const fp_mesh_s* m, int64_t n) { return 2 * n + 2 * (m->ncell + 1) + 1; }

int cell_order(const fp_mesh_s* m, const double* pts, int64_t n, int* scratch, int** perm, cudaStream_t st) {
  const int64_t nb = m->ncell + 1;  // buckets: the cells and "outside"
  int* p = scratch;                  // [n]
  int* cellof = p + n;               // [n]
  int* counts = cellof + n;          // [nb], reused as the scatter cursors
  int* start = counts + nb;          // [nb + 1]
  FP_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)nb, st));
  const DevMesh v = m->view();
  const int blocks = (int)((n + 255) / 256 < 8 * 148 ? (n + 255) / 256 : 8 * 148);
  if (m->d == 2)
    k_point_cells<2><<<blocks, 256, 0, st>>>(v, m->ncell, pts, n, cellof, counts);
  else
    k_point_cells<3><<<blocks, 256, 0, st>>>(v, m->ncell, pts, n, cellof, counts);
  k_scan<<<1, 1024, 0, st>>>(counts, nb, start);
  FP_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)nb, st));
  k_point_scatter<<<blocks, 256, 0, st>>>(cellof, n, start, counts, p);
  FP_CUDA_TRY(cudaGetLastError());
  *perm = p;
  return FP_OK;
}

}  // namespace fp
