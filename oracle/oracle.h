/*
 * FP64 CPU oracle for local findpts — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, direct restatement of the method of Mittal et al.,
 * "General Field Evaluation in High-Order Meshes on GPUs" (arXiv 2501.12349):
 * GLL nodes and Lagrange bases (Sec. 2), piecewise-linear basis bounds and
 * function bounds (Sec. 3.1.1), AABBs and OBBs (Secs. 3.1.1-3.1.2, 4.1-4.2),
 * trust-region Newton (Sec. 3.2.1), candidate selection (Sec. 3.2) and
 * interpolation (Sec. 3.3).  Candidates come from a brute-force box test over
 * every element (no grid); every basis sum is the direct O(N^dr) sum.
 * Element shapes (d, dr): quads (2,2), hexes (3,3), surface quads (3,2) and
 * line elements (2,1), (3,1) (Sec. 2, Eq. x_tensor_surf; Sec. 4.2).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  It shares no code with the CUDA library.
 *
 * Layouts match the CUDA library's C ABI: coords[c][e][n] with node index
 * n = i + N*j (+ N*N*k); points [p][c]; r [p][dr]; aabb [e][2d];
 * obb_c [e][d]; obb_A [e][d][d] row-major.
 */
#ifndef FINDPTS_ORACLE_H
#define FINDPTS_ORACLE_H
#include <stdint.h>

#define OR_MAXN 32
#define OR_MAXM 64

int or_gll_nodes(int N, double* z);
int or_gauss_legendre(int m, double* x, double* w);
void or_lagrange(int N, const double* z, double r, double* phi, double* dphi, double* d2phi);
void or_chebyshev_points(int M, double* eta);
int or_basis_bounds(int N, int M, int reading, double* vlo, double* vhi);
int or_legendre_coeffs(int N, double* c0, double* c1);
int or_bound_1d(int N, int M, const double* u, double* lo, double* hi);
int or_bound_2d(int N, int M, const double* u, double* lo, double* hi);
int or_element_boxes(const double* coords, int d, int dr, int N, int64_t NE, double tol,
                     int M, double* aabb, double* obb_c, double* obb_A);
int or_newton(const double* coords, int d, int dr, int N, int64_t NE, int64_t e,
              const double* xs, double tol, int max_iter, double* r, double* dist2,
              int64_t* stats);
int or_findpts(const double* coords, int d, int dr, int N, int64_t NE, const double* aabb,
               const double* obb_c, const double* obb_A, const double* pts, int64_t n,
               double tol, int max_iter, double dist_tol, int32_t* code, int32_t* elem,
               double* r, double* dist2, int64_t* stats);
int or_locate_in_element(const double* coords, int d, int dr, int N, int64_t NE, int64_t e,
                         const double* pts, int64_t n, double tol, int max_iter,
                         double dist_tol, int32_t* code, double* r, double* dist2);
int or_box_candidates(int d, int64_t NE, const double* aabb, const double* obb_c,
                      const double* obb_A, const double* pts, int64_t n, int32_t* count,
                      int32_t* first);
int or_eval(const double* field, int nc, int dr, int N, int64_t NE, const int32_t* code,
            const int32_t* elem, const double* r, int64_t n, double* out);
int or_forward_map(const double* coords, int d, int dr, int N, int64_t NE,
                   const int32_t* elem, const double* r, int64_t n, double* x, double* jac);
int or_surface_frame(const double* Jc, double* R1, double* R);
int or_num_threads(void);
void or_set_num_threads(int n);

#endif
