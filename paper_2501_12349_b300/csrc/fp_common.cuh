// Internal definitions of libfindpts shared by its translation units (not
// part of the C ABI): status helpers, the mesh object, the by-value views
// the kernels receive, and the grid-cell map of Psi_L.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "findpts.h"

#define FP_CUDA_TRY(expr)                                                  \
  do {                                                                     \
    cudaError_t _e = (expr);                                               \
    if (_e != cudaSuccess) {                                               \
      return _e == cudaErrorMemoryAllocation ? FP_ENOMEM : FP_ELAUNCH;     \
    }                                                                      \
  } while (0)

#define FP_TRY(expr)            \
  do {                          \
    int _s = (expr);            \
    if (_s != FP_OK) return _s; \
  } while (0)

// Device status word values.  A kernel never traps: it records the first
// error here and skips the offending access.
#define FP_DEV_BAD_ELEM 1  // an element id outside [0, NE) was read from Psi_L
#define FP_DEV_BAD_CELL 2  // a cell index outside the grid was formed
#define FP_DEV_SPIN_CAP 3  // a bounded device wait gave up
#define FP_DEV_BAD_ITEM 4  // a work item outside its table was read
#define FP_DEV_DEGENERATE 5  // an element's Jacobian at its centre is singular

namespace fp {

// Record of one element in DevMesh::box32 (floats): lo[3] hi[3] c[3] A[9]
// Xrel curv xc[3] T[9], where Xrel bounds |x - x_ref| over the element
// (largest AABB half-width), curv (volumes) bounds max_c sum_jk |d^2 x_c /
// dr_j dr_k| over the element, xc = x(0) - x_ref and T is the OBB frame
// (J_c^{-1} for volumes, [t1 t2 n]^{-1} for surfaces), so the first dr rows
// of T (x - x(0)) are the reference coordinates of the linearised map.
constexpr int BOX32 = 32;

// Reference point of element e: the centre of its expanded AABB, computed
// with the same rounded operations at setup and at find.
__device__ __forceinline__ double elem_ref(const double* __restrict__ aabb, int d, int64_t e, int c) {
  return (aabb[e * 2 * d + c] + aabb[e * 2 * d + d + c]) * 0.5;
}

// GLL nodes z_i and barycentric weights w_i = 1 / prod_{m!=i} (z_i - z_m) of
// one order, passed by value so the kernels read them from the constant bank.
// The nodes are exactly symmetric about 0 (z_{N-1-i} = -z_i, the middle one
// 0 for odd N) and so are the weights (w_{N-1-i} = (-1)^(N-1) w_i); z2 and
// w2 hold z_m^2 (m < N/2) and 2 w_i for the symmetric form of the basis.
struct BasisTab {
  double z[FP_MAX_N];
  double w[FP_MAX_N];
  double z2[FP_MAX_N / 2];
  double w2[FP_MAX_N];
  float zf[FP_MAX_N];
  float wf[FP_MAX_N];
  float z2f[FP_MAX_N / 2];
  float w2f[FP_MAX_N];
  // double-float forms (value = hi + lo, hi the FP32 rounding, lo the FP32
  // rounding of the rest) of z, w and z^2 for the double-float interpolation
  float zl[FP_MAX_N];
  float wl[FP_MAX_N];
  float z2h[FP_MAX_N / 2];
  float z2l[FP_MAX_N / 2];
  double dn[FP_MAX_N * FP_MAX_N];  // dn[i * N + m] = phi_m'(z_i), the GLL differentiation matrix
};

// Row pitch of the padded FP32 coordinate copy: a row of N r-nodes padded
// to a multiple of 4 floats, so every row starts on a 16-byte boundary and
// loads as whole float4s (for N = 5..8 one 32-byte sector per row); ne32p =
// pitch32(N) N^(dr-1) floats per element and component.
__host__ __device__ constexpr int pitch32(int N) { return (N + 3) & ~3; }

// Everything a find / eval kernel reads about a mesh (passed by value).
struct DevMesh {
  const double* coords;    // [d][NE][ne]
  const float* coords32;   // FP32 copy relative to the element reference point
                           // (elem_ref): fl(x - x_ref), so values are O(h)
  const float* coords32p;  // [d][NE][ne32p]: coords32 with each row of N r-nodes padded
                           // with zeros to pitch32(N) floats (the FP32 Newton phase)
  const double* aabb;      // [NE][2d], expanded
  const double* obb_c;     // [NE][d]
  const double* obb_A;     // [NE][d][d]
  const float* box32;      // [NE][BOX32]: FP32 copy of aabb, obb_c, obb_A and the
                           // coordinate scale X (max |aabb|), for certified FP32 tests
  const float* curv;       // [NE] volumes: bound of sum_jk |d2 x_c / dr_j dr_k| over the element
                           // (the FP64 kernel's certified stop); 0 for surfaces and lines
  const int* cell_start;   // [ncell + 1]
  const int* cell_elems;   // [nnz]
  int64_t NE;
  int64_t cstride;         // NE * ne: distance between coordinate components
  int64_t cstride32p;      // NE * ne32p: the same in coords32p
  double lo[3], hi[3], scale[3];
  int NL;
  int max_iter;
  double newton_tol;
  double dist_tol;
  int* status;
};

// The Psi_L cell coordinate of x along one axis (Sec. 3.1.3): floor of
// (x - lo) * scale, clamped to [0, NL-1].  The same rounded operations serve
// the element corners at setup and the points at find, so x inside an AABB
// implies x's cell lies in the element's cell range.
__device__ __forceinline__ int cell_coord(double x, double lo, double scale, int NL) {
  double t = __dmul_rn(__dsub_rn(x, lo), scale);
  int c = (t >= (double)NL) ? NL - 1 : (int)floor(t);
  return c < 0 ? 0 : c;
}

__device__ __forceinline__ void record_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// A template so that only the translation units that launch it compile it.
// Exclusive scan of counts[0..n) into start[0..n], start[n] = total, by one
// CTA: each thread scans a contiguous chunk.
template <int kUnused = 0>
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ counts, int64_t n,
                                               int* __restrict__ start) {
  __shared__ long long part[1024];
  const int t = threadIdx.x;
  const int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
  const int64_t b = t * chunk, en = b + chunk < n ? b + chunk : n;
  long long s = 0;
  for (int64_t i = b; i < en; ++i) s += counts[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    long long v = (t >= o) ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  long long run = part[t] - s;
  for (int64_t i = b; i < en; ++i) {
    start[i] = (int)run;
    run += counts[i];
  }
  if (t == (int)blockDim.x - 1) start[n] = (int)part[t];
}

}  // namespace fp

// The library-owned mesh object behind the fp_mesh handle.
namespace fp {
struct KernelTimer;
}

struct fp_mesh_s {
  int d, dr, N, ne, M, NL;
  int64_t NE, ncell, nnz;
  fp::KernelTimer* timer;  // per-kernel CUDA-event timing (fp_set_timing), or null
  double setup_ms[2];      // k_boxes and the Psi_L build, CUDA events at setup
  fp_opts opts;
  int precision;
  double* coords;
  float* coords32;
  float* coords32p;
  double* aabb;
  double* obb_c;
  double* obb_A;
  float* box32;
  float* curv;
  int* cell_start;
  int* cell_elems;
  int* status;
  double lo[3], hi[3], scale[3];
  size_t bytes;
  fp::BasisTab basis;
  fp::DevMesh view() const;
};

namespace fp {
// host helpers shared by the translation units
int host_basis_tab(int N, BasisTab* tab);
int check_mesh(const fp_mesh_s* m);
// Kernel timing (timing.cu): with the mesh's timer on, timer_mark records an
// event on st and returns it (null otherwise); timer_span files the interval
// between two marks under a stage (FP_TIME_*); timer_free releases it all.
cudaEvent_t timer_mark(const fp_mesh_s* m, cudaStream_t st);
void timer_span(const fp_mesh_s* m, int stage, cudaEvent_t a, cudaEvent_t b);
void timer_free(fp_mesh_s* m);
// The FP_MIXED double-float interpolation (eval.cu): whether a call of n
// points takes it, and the field split once (df_field_prepare) for any
// number of point sets (df_field_eval), released with df_field_release; all
// stream-ordered on st.
struct DfField {
  float2* fs = nullptr;
  int* emax = nullptr;
  void* scratch = nullptr;
  int nc = 0, Nf = 0;
};
bool eval_uses_df(const fp_mesh_s* m, int64_t n);
int df_field_prepare(const fp_mesh_s* m, const double* field, int Nf, int nc, DfField* f, cudaStream_t st);
int df_field_eval(const fp_mesh_s* m, const DfField& f, const int32_t* code, const int32_t* elem,
                  const double* r, int64_t n, double* out, cudaStream_t st);
void df_field_release(DfField& f, cudaStream_t st);
}  // namespace fp

#include <type_traits>

namespace fp {

template <int V>
using ic = std::integral_constant<int, V>;

// N^dr: nodes of a line, quad or hex element.
__host__ __device__ constexpr int ipow(int n, int k) { return k == 0 ? 1 : n * ipow(n, k - 1); }

// Calls f(ic<N>, ic<D>, ic<DR>) for the element shapes the library is built
// for: N in 2..FP_MAX_N and (d, dr) in {(2,2), (3,3), (3,2), (2,1), (3,1)}:
// quads, hexes, surface quads and line elements in 2D and 3D.
template <typename F>
int dispatch_shape(int N, int d, int dr, F&& f) {
  auto withN = [&](auto Dc, auto DRc) -> int {
    switch (N) {
      case 2: return f(ic<2>{}, Dc, DRc);
      case 3: return f(ic<3>{}, Dc, DRc);
      case 4: return f(ic<4>{}, Dc, DRc);
      case 5: return f(ic<5>{}, Dc, DRc);
      case 6: return f(ic<6>{}, Dc, DRc);
      case 7: return f(ic<7>{}, Dc, DRc);
      case 8: return f(ic<8>{}, Dc, DRc);
      default: return FP_EUNSUPPORTED;
    }
  };
  if (d == 2 && dr == 2) return withN(ic<2>{}, ic<2>{});
  if (d == 3 && dr == 3) return withN(ic<3>{}, ic<3>{});
  if (d == 3 && dr == 2) return withN(ic<3>{}, ic<2>{});
  if (d == 2 && dr == 1) return withN(ic<2>{}, ic<1>{});
  if (d == 3 && dr == 1) return withN(ic<3>{}, ic<1>{});
  return FP_EINVAL;
}

inline int grid_for(int64_t n, int threads, int max_blocks) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)(b < max_blocks ? b : max_blocks);
}

}  // namespace fp
