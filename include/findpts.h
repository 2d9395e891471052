/*
 * findpts.h — C ABI of libfindpts, a B300 (sm_103a) implementation of local
 * point location and field evaluation in high-order curvilinear meshes
 * (Mittal et al., "General Field Evaluation in High-Order Meshes on GPUs",
 * arXiv 2501.12349).
 *
 * Method, by the paper's sections:
 *   Setup (Sec. 3.1): per element, an axis-aligned bounding box (Sec. 3.1.1,
 *     Eqs. 1D_bases_bounds, 1D_bound_final, 2D_function_bound, AABB_test) and
 *     an oriented bounding box (Sec. 3.1.2, Eqs. OBB_transformation, OBB_test),
 *     then the process-local Cartesian map Psi_L from a grid cell to the
 *     elements whose AABB covers it (Sec. 3.1.3).
 *   Find (Sec. 3.2): cell lookup, box filter, trust-region Newton on
 *     f(r) = 0.5 |x* - x(r)|^2 (Sec. 3.2.1, Eqs. newton, newton_jacobian,
 *     newton_hessian), candidate selection (first INTERIOR, else the BORDER
 *     with the smallest distance).
 *   Interpolate (Sec. 3.3, Eq. u_tensor).
 *   Surface meshes (Sec. 4): quadrilaterals embedded in 3D.
 * The multi-rank stages (global map Psi_G, Sec. 3.1.4, and point routing)
 * have no counterpart: one process drives one GPU.
 *
 * Conventions shared by every call:
 *   d  = physical dimension (2 or 3), dr = reference dimension (dr == d for
 *        quads and hexes, dr = 2, d = 3 for surface quads), N = order + 1
 *        (2 <= N <= FP_MAX_N), ne = N^dr nodes per element.
 *   Node index within an element is lexicographic with r fastest:
 *        n = i + N*j (+ N*N*k), node (i,j,k) sits at GLL reference point
 *        (zeta_i, zeta_j, zeta_k).
 *   Coordinates and fields are structure-of-arrays: coords[c][e][n] at
 *        offset (c*NE + e)*ne + n.  Points are array-of-structures:
 *        pts[p][c] at offset p*d + c.
 *   Array arguments of find / eval are DEVICE memory owned by the caller
 *        unless stated otherwise.
 *   `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *        asynchronous on that stream unless stated otherwise; the caller
 *        keeps every buffer alive until the stream has passed the call.
 *   Return value: FP_OK (0) or a negative FP_E* status; no call throws, and
 *        per-point outcomes are reported in `code`, never as a status.
 */
#ifndef FINDPTS_H
#define FINDPTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FP_OK 0
#define FP_EINVAL (-1)       /* bad argument (NULL pointer, size, dimension) */
#define FP_ENOMEM (-2)       /* device allocation failed or budget exceeded  */
#define FP_ELAUNCH (-3)      /* a kernel launch or CUDA runtime call failed  */
#define FP_EDEVICE (-4)      /* a kernel set its device status word          */
#define FP_ETIMEDOUT (-5)    /* a host-side wait ran out                      */
#define FP_EBUSY (-6)        /* resource in use                               */
#define FP_EUNSUPPORTED (-7) /* element type / order not built               */
#define FP_ECANCELED (-8)    /* a server request was cancelled               */

/* ---- per-point location codes (Sec. 3.2, the enum c*) ------------------- */
#define FP_INTERIOR 0
#define FP_BORDER 1
#define FP_NOT_FOUND 2

/* ---- arithmetic of the find kernels ------------------------------------- */
#define FP_F64 0   /* every step in FP64                                        */
#define FP_MIXED 1 /* FP32 box filter and early Newton steps; FP64 final steps,  */
                   /* residual check and ill-conditioned Jacobian solves         */

#define FP_MAX_N 8 /* orders 1..7 */

/* Traversal order of the query points inside fp_findpts.  FP_ORDER_CELL
 * groups the points by their Psi_L cell before the find kernels run (a
 * counting sort on the device, for calls of at least 16384 points), so the
 * points a warp handles share candidate elements; the paper's remark on the
 * CPU implementation (Sec. 3.2) that processing the points of an element
 * together improves locality.  The cells' points come in four cost classes
 * (3 or more candidate boxes, 2, 1, none), the costly ones first, so the end
 * of a launch, where lanes wait for the slowest point of their warp, runs
 * cheap points.  FP_ORDER_GIVEN takes the points as given.  The outputs are
 * identical either way; only the speed differs.  The cell order needs 8
 * bytes per point plus 32 bytes per cell of scratch, taken from the
 * stream-ordered allocator for the duration of the call. */
#define FP_ORDER_GIVEN 0
#define FP_ORDER_CELL 1

typedef struct fp_mesh_s* fp_mesh; /* opaque; library-owned; device-resident */

/* Options of Setup and Find.  fp_opts_default fills the paper's defaults. */
typedef struct {
  double bbox_tol;   /* box expansion, fraction of the extent (Sec. 3.1.1: 10%)    */
  int M;             /* Chebyshev interval points of the bounds; 0 => 2N (3.1.1)   */
  int n_grid;        /* cells per direction of Psi_L; 0 => smallest n, n^d >= NE   */
  double newton_tol; /* stop when |dr|_inf < newton_tol (Sec. 3.2.1: 1e-10)        */
  int max_iter;      /* Newton iteration cap per candidate (Sec. 3.2.1: 50)        */
  double dist_tol;   /* surfaces: INTERIOR needs dist2 < dist_tol (Sec. 4.4: 1e-10) */
  int precision;     /* FP_F64 or FP_MIXED                                          */
  int point_order;   /* FP_ORDER_CELL (default) or FP_ORDER_GIVEN, see below        */
} fp_opts;

void fp_opts_default(fp_opts* opts);

/* Setup (Sec. 3.1).  Copies coords_dev ([d][NE][N^dr] FP64, device) into
 * library-owned device memory, computes element AABBs and OBBs expanded by
 * bbox_tol and builds Psi_L, all on the GPU.  Besides the FP64 copy the mesh
 * keeps two FP32 copies of the coordinates relative to each element's
 * centre (one with its rows of N nodes padded to 16-byte boundaries, for
 * the mixed path's vector loads) and per-element box and curvature records:
 * per coordinate value 8 + 4 + 4 P/N bytes (P = 4 ceil(N/4), so 18.4 bytes
 * at N = 5), plus about 0.3 KB per element; fp_mesh_info reports the total.
 * Blocks until done (it allocates).  *out receives the handle; fp_free
 * releases it.
 * Errors: FP_EINVAL for a bad dimension pair, order, NE <= 0 or M outside
 * [2, 32]; FP_EUNSUPPORTED for N > FP_MAX_N; FP_ENOMEM; FP_ELAUNCH. */
int fp_setup(const double* coords_dev, int d, int dr, int order, int64_t NE,
             const fp_opts* opts, void* stream, fp_mesh* out);

/* Releases every device allocation of the mesh (synchronises the device). */
int fp_free(fp_mesh m);

/* Selects the arithmetic of later fp_findpts calls on this mesh: FP_F64 or
 * FP_MIXED (both sets of device data are built by fp_setup).  Host call. */
int fp_set_precision(fp_mesh m, int precision);

/* Sets the point traversal order (FP_ORDER_GIVEN / FP_ORDER_CELL) of later
 * fp_findpts calls on m.  Errors: FP_EINVAL. */
int fp_set_point_order(fp_mesh m, int order);

/* Find (Sec. 3.2) for n points pts_dev ([n][d] FP64).  Outputs (device):
 *   code[n]  FP_INTERIOR / FP_BORDER / FP_NOT_FOUND
 *   elem[n]  element id, -1 when NOT_FOUND
 *   r[n][dr] reference coordinates in [-1,1]^dr, 0 when NOT_FOUND
 *   dist2[n] |x* - x(r*)|^2, +inf when NOT_FOUND
 * A point with a non-finite coordinate is NOT_FOUND.  n == 0 is a no-op.
 * Errors: FP_EINVAL (NULL pointer with n > 0, n < 0), FP_ELAUNCH. */
int fp_findpts(fp_mesh m, const double* pts_dev, int64_t n, int32_t* code,
               int32_t* elem, double* r, double* dist2, void* stream);

/* As fp_findpts, and adds this call's counters into stats_dev (device,
 * FP_NSTATS uint64 values, caller-zeroed):
 *   [0] candidates that passed the box filter  [1] Newton iterations
 *   [2] rejected trust-region steps            [3] Newton steps with beta = 1
 *   [4] FP64 refinement evaluations (mixed path's FP32 kernel); in the FP64
 *       kernel, the iterations ended by a certified last step (volumes: the
 *       next step is bounded below the rounding noise, so the sub-tolerance
 *       step that Sec. 3.2.1 would take after one more evaluation is left out)
 *                                              [5] box tests decided in FP64
 *   [6] points the mixed path handed to its FP64 kernel
 *   [7] full evaluations of x(r) and G(r), re-evaluations after a rejected
 *       step not counted: in the FP64 kernel one per trial step (a
 *       candidate starts at its closest GLL node, where x is the node and G
 *       one N-term sum per direction); in the mixed path's FP32 kernel also
 *       one per candidate, at its linearised start
 * With FP_MIXED, [0]-[7] count the FP32 kernel (its iterations are FP32
 * iterations) and [8]-[15] count, in the same layout, the FP64 kernel that
 * finishes the points of [6]; with FP_F64, [8]-[15] stay zero. */
#define FP_NSTATS 16
int fp_findpts_stats(fp_mesh m, const double* pts_dev, int64_t n, int32_t* code,
                     int32_t* elem, double* r, double* dist2, uint64_t* stats_dev,
                     void* stream);

/* Mixed-precision find that allocates no device memory.  The paper has no
 * counterpart: it is the FP_MIXED algorithm of fp_findpts, for callers that
 * cannot let a library call cudaMalloc — solvers that reserve the GPU's
 * memory up front and run under a hard budget, and code that must not see
 * the implicit synchronisation or the possible failure of an allocation in
 * the middle of a time step.  Its scratch (the queue of points passed from
 * the FP32 kernel to the FP64 kernel) is a fixed array inside the library of
 * FP_NOALLOC_MAX_POINTS + 1 ints (4 MiB), held on every GPU that loads the
 * library until the process exits.
 *   Arguments, layouts and outputs as fp_findpts; the mesh's precision
 *   setting is ignored (always FP_MIXED).  n > FP_NOALLOC_MAX_POINTS is
 *   rejected with FP_EINVAL before anything runs; split larger sets.
 *   The first call on a device looks up the array's device address (a
 *   one-time set-up per device, with that device current); make that first
 *   call before any stream capture.  The address is kept for the rest of
 *   the process: after a cudaDeviceReset of that device (by any code in the
 *   process) it is stale, so do not call this entry point on a device that
 *   has been reset.
 *   All calls share the one array: calls that can overlap on the GPU (on
 *   different streams, or from different threads) race and must be
 *   serialised by the caller.  Each call clears the queue's counter. */
#define FP_NOALLOC_MAX_POINTS (1 << 20)
int fp_findpts_mixed_noalloc(fp_mesh m, const double* pts_dev, int64_t n, int32_t* code,
                             int32_t* elem, double* r, double* dist2, void* stream);

/* Interpolate (Sec. 3.3): out[c][p] = u_c(r_p) in element elem_p for the
 * nc components of field_dev ([nc][NE][N^dr] FP64, device, same node layout
 * as the coordinates); 0 where code == FP_NOT_FOUND.  The same find output
 * serves any number of fields.
 * Precision follows the mesh's setting (fp_set_precision): FP_F64 contracts
 * in FP64.  FP_MIXED, for quads, hexes and surfaces with n >= 16384 and
 * n >= 8 NE, contracts in double-float arithmetic on the FP32 pipe (pairs
 * of FP32 values with error-free transformations), within about 1e-13 of
 * the element's nodal scale of the FP64 result, visiting the points in
 * element order; it then takes 8 bytes of device scratch per field value
 * (the field split into those pairs after an exact power-of-two scaling
 * per component) plus 4 (n + 2 NE + nc + 3) bytes, from the stream-ordered
 * allocator for the duration of the call.  Smaller FP_MIXED calls contract
 * in FP64.
 * Errors: FP_EINVAL, FP_ENOMEM (FP_MIXED scratch), FP_ELAUNCH. */
int fp_eval(fp_mesh m, const int32_t* code, const int32_t* elem, const double* r,
            int64_t n, const double* field_dev, int nc, double* out, void* stream);

/* Find, and optionally Interpolate, end to end from host memory.  The paper
 * has no counterpart: it is fp_findpts followed by fp_eval, with the points
 * copied to the device and the results copied back in chunks of `chunk`
 * points (0: automatic, chunks of n/4 points, at least 2^19), each chunk's
 * copies overlapping the search of the others, and consecutive chunks
 * searched on two streams so that one's launch fills the other's tail.
 *   pts_host [n][d]; outputs code_host [n], elem_host [n], r_host [n][dr],
 *   dist2_host [n] as fp_findpts; with field_dev (device, [nc][NE][N^dr])
 *   not NULL, out_host [nc][n] as fp_eval.  All host buffers should be
 *   pinned (page-locked), or the copies do not overlap the kernels.
 * Device scratch: (8 (d + dr + 1 + nc) + 8) bytes per point, plus the cell
 * order's and, with FP_MIXED and a field, fp_eval's, from the stream-ordered
 * allocator for the duration of the call.
 * Synchronous: returns when the results are in host memory.
 * Errors: FP_EINVAL, FP_ENOMEM, FP_ELAUNCH. */
int fp_findpts_host(fp_mesh m, const double* pts_host, int64_t n, int32_t* code_host,
                    int32_t* elem_host, double* r_host, double* dist2_host,
                    const double* field_dev, int nc, double* out_host, int64_t chunk,
                    void* stream);

/* Interpolate a field of another order (Sec. 2, after Eq. u_tensor: the
 * solution's order N~ - 1 often differs from the coordinates' order N - 1).
 * field_dev is [nc][NE][(field_order+1)^dr] FP64 on the GLL nodes of
 * field_order + 1 points per direction, in the node layout of the
 * coordinates; code, elem, r come from fp_findpts on the same mesh and
 * out[c][p] as fp_eval (precision and scratch as there).  field_order ==
 * the mesh's order is fp_eval.
 * Errors: FP_EINVAL; FP_EUNSUPPORTED unless 1 <= field_order <= 7;
 * FP_ELAUNCH. */
int fp_eval_order(fp_mesh m, const int32_t* code, const int32_t* elem, const double* r,
                  int64_t n, const double* field, int field_order, int nc, double* out,
                  void* stream);

/* ---- many meshes in one graph launch ---------------------------------------
 * A batch plan runs find (and optionally eval) for many (mesh, point set)
 * items at once: items are grouped by element shape (N, d, dr); per shape one
 * persistent find launch covers every item's points (FP_F64, or FP_MIXED with
 * its FP64 pass) and one launch interpolates the items that carry a field.
 * The launches of all shapes are captured once into a CUDA graph on forked
 * streams; fp_batch_run replays that graph.  Pointers are captured: the
 * caller may change the point and field values between runs, not the
 * buffers.  With FP_MIXED, a shape of quads, hexes or surfaces with the
 * cell order and at least 8 points per element of its items with a field
 * interpolates in double-float arithmetic (as fp_eval), its fields split
 * on every run into plan-owned buffers (8 bytes per field value). */
typedef struct {
  int mesh;              /* index into the meshes array given to fp_batch_create */
  const double* pts;     /* [n][d] device */
  int64_t n;
  int32_t* code;         /* outputs as fp_findpts, [n] / [n][dr], device */
  int32_t* elem;
  double* r;
  double* dist2;
  const double* field;   /* [nc][NE][N^dr] device, or NULL for no eval */
  int nc;
  double* out;           /* [nc][n] device (when field != NULL) */
} fp_batch_item;

typedef struct fp_batch_s* fp_batch;

/* Builds the plan (item tables on the device, a scratch queue per shape for
 * FP_MIXED) and captures the graph.  A shape with at least 16384 points whose
 * items' meshes all use FP_ORDER_CELL takes its points grouped by (item,
 * Psi_L cell), as fp_findpts does (scratch: 8 bytes per point and per
 * cell); the outputs are the same either way.  Launch shapes come from this process's
 * earlier fp_batch_autotune results for the same shape, precision and point
 * count (power-of-two bucket), else defaults.  Synchronous.
 * Errors: FP_EINVAL (bad index, NULL buffer, n > 2^31-1), FP_ENOMEM,
 * FP_ELAUNCH. */
int fp_batch_create(const fp_mesh* meshes, int nm, const fp_batch_item* items, int nitems,
                    int precision, void* stream, fp_batch* out);

/* Replays the captured graph on `stream` (asynchronous). */
int fp_batch_run(fp_batch b, void* stream);

/* The find of all shapes in ONE persistent launch (on = 1) instead of one
 * persistent launch per shape (on = 0, the default): the shapes' point
 * sequences are cut into tiles of 4096 points, which the CTAs pull from a
 * counter, each tile searched by the lane loop of its shape (device-side
 * dispatch over the compiled shapes); FP_MIXED adds each shape's FP64
 * follow-up over its hand-over queue.  The point order, the evals and the
 * results are the same in both forms.  Re-captures the graph; synchronous.
 * Errors: FP_EINVAL, FP_ELAUNCH. */
int fp_batch_set_fused(fp_batch b, int on);

/* The launch shape autotuner: for every element shape of the plan, times the
 * shape's launches for CTAs per SM (the kernel's register-limited maximum
 * and one fewer: for FP_F64 {2, 3} up to order 5 and {1, 2} above; for
 * FP_MIXED {3, 4} or {2, 3} by element shape) and points per CTA chunk in
 * {32, 128, 512} on the plan's own data (best of two timed runs each), keeps
 * the fastest, records it for later plans and re-captures the graph.
 * Overwrites the plan's outputs.  Synchronous. */
int fp_batch_autotune(fp_batch b, void* stream);

typedef struct {
  int N, d, dr, n_items;
  int64_t n_points;
  int ctas_per_sm, chunk_points;
  float tuned_ms; /* time of the chosen shape in the autotuner, -1 if untuned */
} fp_batch_class_info;

int fp_batch_num_classes(fp_batch b);
int fp_batch_describe(fp_batch b, int i, fp_batch_class_info* info);

/* Releases the plan (synchronises the device). */
int fp_batch_free(fp_batch b);

/* ---- continuous-batching server -------------------------------------------
 * Meshes (and their fields) stay resident; requests are submitted from any
 * host thread and run as soon as a slot and device memory are free:
 *   FP_REQ_REMAP    find the points, interpolate the mesh's remap field
 *                   (Find once + Interpolate, Secs. 3.2-3.3; the remap use of
 *                   Sec. 6.4);
 *   FP_REQ_PARTICLE rk_steps explicit-midpoint steps of size dt through the
 *                   mesh's velocity field (Find / Interpolate / Integrate, the
 *                   particle-tracking loop of Sec. 6.7), then a final find of
 *                   the end positions; a particle that leaves the mesh is
 *                   NOT_FOUND and stops.
 * A scheduler thread packs one stage of every ready request into each tick
 * (batched launches across requests, grouped by element shape; up to two
 * ticks in flight), so requests that arrive while others run are admitted
 * and overlap on the device.  A request's result does not depend on what
 * else is in flight. */
#define FP_REQ_REMAP 0
#define FP_REQ_PARTICLE 1

typedef struct fp_server_s* fp_server;

typedef struct {
  size_t mem_budget;     /* device bytes for request buffers (admission)      */
  int max_active;        /* requests admitted at once (slots)                  */
  int precision;         /* FP_F64 or FP_MIXED                                 */
  double tick_timeout_s; /* host watchdog per tick: its requests fail with     */
                         /* FP_ETIMEDOUT (memory kept until the tick ends)     */
  int64_t tick_points;   /* points per tick (default 2^19): a request's stage  */
                         /* is split into tiles, filled in the order of the    */
                         /* policy below; fewer points per tick lower the      */
                         /* latency of small requests and cost capacity        */
  int policy;            /* FP_SCHED_SLACK (default) or FP_SCHED_SRPT          */
  double slack_base;     /* FP_SCHED_SLACK: a request's target is slack_base + */
  double slack_factor;   /* slack_factor x its size, in stage points (below)   */
} fp_server_opts;

/* Tick policies.  Work is counted in stage points (a point searched and
 * interpolated once; a particle request of n points and k steps is
 * (2k + 1) n of them), and time in the stage points the server has
 * finished since a request was submitted (its age).
 *   FP_SCHED_SRPT: the requests with the least work left in their current
 *     stage first (small requests pass large ones; a large one can wait
 *     long under heavy load).
 *   FP_SCHED_SLACK: least slack first, slack = slack_base + slack_factor x
 *     size - age - work left, so a request's priority grows as it waits,
 *     in proportion to its size: small requests still go first, and a
 *     large one is not held back without bound. */
#define FP_SCHED_SRPT 0
#define FP_SCHED_SLACK 1

typedef struct {
  int64_t submitted, admitted, completed, cancelled, ticks, timeouts;
  int64_t active, queued;
  size_t bytes_in_use;
} fp_server_stats;

/* 1 GiB, 64 slots, FP_MIXED, 30 s, 2^19 points per tick, FP_SCHED_SLACK with
 * slack_base 2^20 and slack_factor 4 */
void fp_server_opts_default(fp_server_opts* opts);

/* remap_fields[i] ([nc_remap[i]][NE][N^dr], device) and velocity[i]
 * ([d][NE][N^dr], device) may be NULL (arrays themselves may be NULL); they
 * must stay valid until fp_server_destroy.  With FP_MIXED the server
 * interpolates on quads, hexes and surfaces in double-float arithmetic (as
 * fp_eval) from copies of those fields split at creation (8 bytes of device
 * memory per value): changes to the fields' contents after creation are not
 * seen.  Starts the scheduler thread. */
int fp_server_create(const fp_mesh* meshes, int nm, const double* const* remap_fields,
                     const int* nc_remap, const double* const* velocity,
                     const fp_server_opts* opts, fp_server* out);

/* Queues a request.  Host buffers (pinned memory recommended) must stay
 * valid until the request is done; outputs:
 *   code_host[n], elem_host[n], r_host[n][dr], dist2_host[n] (any may be
 *   NULL), out_host = remap: interpolated values [nc][n]; particle: final
 *   positions [n][d].
 * Errors: FP_EINVAL; FP_ENOMEM if the request could never fit the budget. */
int fp_server_submit(fp_server s, int mesh, int kind, const double* pts_host, int64_t n,
                     int rk_steps, double dt, int32_t* code_host, int32_t* elem_host,
                     double* r_host, double* dist2_host, double* out_host, int64_t* req_id);

/* Never blocks on the device: *done = 1 when finished (*status its result). */
int fp_server_poll(fp_server s, int64_t req_id, int* done, int* status);

/* Blocks up to timeout_s: the request's status, or FP_ETIMEDOUT. */
int fp_server_wait(fp_server s, int64_t req_id, double timeout_s);

/* Cancels a request not yet admitted (FP_EBUSY otherwise). */
int fp_server_cancel(fp_server s, int64_t req_id);

/* Seconds from submission to admission and to completion (done requests). */
int fp_server_timing(fp_server s, int64_t req_id, double* queued_s, double* total_s);

/* Forgets a finished request (its id becomes invalid). */
int fp_server_release(fp_server s, int64_t req_id);

int fp_server_get_stats(fp_server s, fp_server_stats* stats);

/* Stops the scheduler, waits for the work the server queued on its own
 * streams (with the tick watchdog limit as deadline; other work on the
 * device is not waited for) and frees everything.  If that wait runs out,
 * returns FP_ETIMEDOUT and leaves the server's device and pinned buffers
 * allocated (leaked), since kernels may still use them; the handle is
 * invalid either way. */
int fp_server_destroy(fp_server s);

/* ---- introspection (tests, benchmarks) ----------------------------------- */
typedef struct {
  int d, dr, N, M, n_grid;
  int64_t NE, n_cells, n_cell_entries;
  double grid_lo[3], grid_hi[3];
  size_t device_bytes;
  double setup_boxes_ms; /* k_boxes (Secs. 3.1.1-3.1.2) at setup, CUDA events   */
  double setup_grid_ms;  /* the Psi_L build (Sec. 3.1.3) at setup, CUDA events  */
} fp_mesh_info;

/* Per-kernel timing of find and eval calls (the paper has no counterpart;
 * it serves roofline measurements).  With timing on, every later
 * fp_findpts / fp_findpts_stats / fp_eval / fp_eval_order call on the mesh
 * records CUDA events on its stream between its kernels; fp_kernel_times
 * waits for the recorded events, adds up the intervals per stage since its
 * last call and starts over.  Stages: */
#define FP_TIME_ORDER 0  /* the cell order (fp_set_point_order)               */
#define FP_TIME_FIND 1   /* the find kernel (k_find_f64, or k_find_mixed)     */
#define FP_TIME_FOLLOW 2 /* FP_MIXED: the FP64 kernel on the handed-over points */
#define FP_TIME_EVAL 3   /* the interpolation kernel                           */
#define FP_NTIMES 4
/* on = 0 stops recording (intervals recorded so far stay readable).
 * Errors: FP_EINVAL, FP_ENOMEM. */
int fp_set_timing(fp_mesh m, int on);
/* ms[FP_NTIMES]: summed milliseconds per stage; calls[FP_NTIMES] (may be
 * NULL): intervals per stage.  At most 65536 intervals are kept between two
 * reads; later ones are dropped.  Errors: FP_EINVAL, FP_ELAUNCH. */
int fp_kernel_times(fp_mesh m, double* ms, int64_t* calls);

/* Host call; fills *info. */
int fp_get_info(fp_mesh m, fp_mesh_info* info);

/* Copies the boxes into caller device buffers (any may be NULL):
 * aabb[NE][2d] = (lo_0..lo_{d-1}, hi_0..hi_{d-1}), already expanded;
 * obb_c[NE][d] the OBB centre; obb_A[NE][d][d] (row-major) the map A with
 * |A (x - c)|_inf <= 1 exactly on the expanded OBB.  Synchronous. */
int fp_get_boxes(fp_mesh m, double* aabb, double* obb_c, double* obb_A, void* stream);

/* Copies each element's curvature bound into curv_dev[NE] (device, FP64).
 * The paper has no counterpart: the find kernels use it to certify that a
 * Newton step is the last one needed (the next step, bounded from the
 * linear model's residual and this term, is far below the tolerance).
 * Volumes (d == dr): L_e >= max over element e of sum_jk |d2 x_c / dr_j dr_k|
 * for every component c (the second derivatives' values at the GLL nodes
 * through the Lebesgue constant), as stored for the kernels (FP32, widened
 * by 1e-6); 0 for surfaces and lines.  Synchronous.
 * Errors: FP_EINVAL, FP_ELAUNCH. */
int fp_get_curvature(fp_mesh m, double* curv_dev, void* stream);

/* Copies Psi_L in CSR form into caller device buffers: cell_start[n_cells+1],
 * cell_elems[n_cell_entries], element ids ascending within a cell.  Cell
 * (c_0,c_1,c_2) has index c_0 + n_grid*(c_1 + n_grid*c_2).  Synchronous. */
int fp_get_grid(fp_mesh m, int32_t* cell_start, int32_t* cell_elems, void* stream);

/* Reads and clears the mesh's device status word: 0, or the first error a
 * kernel recorded (an out-of-range element or cell index).  Synchronises
 * the stream. */
int fp_device_status(fp_mesh m, int* status, void* stream);

const char* fp_status_string(int status);

/* Measured FMA-pipe throughput in GFLOP/s (1 FMA = 2 flop): which = 0 FP64,
 * 1 FP32.  The roofline denominator of the find / eval kernels, which are
 * bound by these pipes.  Allocates a small scratch buffer; synchronous. */
int fp_alu_peak(int which, int iters, double* gflops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FINDPTS_H */
