/*
 * femasm.h - C ABI of the GB300 (sm_103a) library for P1 finite-element assembly of the Poisson
 * problem -div(k grad u) = f, following L. Chen, "Programming of Finite Element Methods in MATLAB"
 * (arXiv:1804.05156).
 *
 * Conventions (all entry points):
 *  - Array arguments are DEVICE pointers owned by the caller unless stated otherwise; the library
 *    never frees them. Library-owned objects are opaque handles with an explicit destroy call.
 *  - Indices are 0-based int32 (the paper is 1-based). Element arrays are row-major [NT][d+1]
 *    (Sec. 1.1 `elem`); coordinates are row-major double [N][d] (Sec. 1.1 `node`).
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the legacy default stream)
 *    unless its comment says it synchronises.
 *  - Every call returns FEM_OK (0) or a negative FEM_ERR_* code; fem_last_error_string() gives a
 *    host-side message for the last failure in the calling process. No call aborts the process,
 *    throws, or traps the GPU.
 *  - Errors found by kernels (a degenerate element, an index out of range) are recorded in a
 *    device error word; they surface at the next fem_get_error() call.
 *  - Double arrays must be 8-byte aligned and int32 arrays 4-byte aligned (FEM_ERR_ARG otherwise).
 *  - A pattern owns per-call device scratch (packets, work counters, host-step buffers): calls on
 *    one pattern must be ordered (one host thread, one stream, or streams ordered by events).
 *    Different patterns are independent.
 */
#ifndef FEMASM_H
#define FEMASM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FEM_OK 0
#define FEM_ERR_ARG -1        /* null pointer, d not in {2,3}, negative or oversized count, misaligned pointer */
#define FEM_ERR_INDEX -2      /* an element names a vertex outside [0, N) or the same vertex twice */
#define FEM_ERR_DEGENERATE -3 /* 2-D element of zero area, or 3-D element of non-positive volume */
#define FEM_ERR_CUDA -4       /* a CUDA runtime call failed */
#define FEM_ERR_OOM -5        /* device allocation failed */
#define FEM_ERR_TIMEOUT -6    /* a bounded device-side wait gave up */
#define FEM_ERR_STATE -7      /* handle used in a way its construction does not allow */
#define FEM_ERR_RANGE -8      /* a value outside the range the float-float kernels keep 1e-12 accuracy in:
                                 an input value (coefficient or tensor entry, load value f, loss weight w or
                                 r) nonzero and outside [2^-80, 2^96]; a 2-D element whose result scale
                                 2^(p s) (s the exponent of its largest edge component, p the result's
                                 degree of homogeneity) leaves [2^-100, 2^100]; a tetrahedron with 6|tau|
                                 outside [2^-72, 2^87] (edges of about 2^-24 to 2^29); or an element
                                 contribution whose terms are nonzero but below 2^-84 or above 2^120 in
                                 magnitude (the check is on the terms, not on their sum, which may cancel) */

/* Reduction variants of the value kernels (Sec. 2.2: `sparse` sums duplicate (i, j) entries). */
#define FEM_DETERMINISTIC 0 /* fixed summation order per CSR slot: bitwise reproducible */
#define FEM_ATOMIC 1        /* FP64 atomicAdd into the CSR values: order varies run to run */

/* Right-hand side f (Sec. 3.2). */
#define FEM_F_CONST 0    /* f = f_arg[0] (device), or 1 when f_arg is NULL */
#define FEM_F_SINPROD 1  /* f = prod_m sin(pi x_m) over the d coordinates; f_arg unused */
#define FEM_F_QPVALUES 2 /* f given at the quadrature points: f_arg[t * nq + q] (device, caller's
                            element order; 2-D nq = 3, point q = midpoint of the side opposite
                            vertex q; 3-D nq = 4, point q has barycentric weight a on vertex q) */

typedef struct fem_pattern_s* fem_pattern_t;
typedef struct fem_batch_s* fem_batch_t;
typedef void* fem_stream_t; /* cudaStream_t */

/* ---- pattern (Sec. 2.1-2.2 and the (i, j) index lists of Sec. 3.1.2-3.1.3) --------------------
 * Builds the structural CSR pattern of the P1 stiffness matrix of the mesh `elem` [NT][d+1] over N
 * vertices: the set of pairs (elem[t][i], elem[t][j]), rows ascending, columns ascending within a
 * row, kept even where values later cancel. For the symmetric matrix these arrays equal the CSC
 * arrays MATLAB keeps (Sec. 2.1). Also builds the per-element slot map
 *   slot[(i*(d+1) + j) * NT + t] = CSR position of (elem[t][i], elem[t][j])
 * and the vertex-to-element incidence lists used by the deterministic reduction.
 * `elem` is read during the call only; the pattern keeps its own copy of the topology, so later
 * value calls take no `elem` argument. Synchronises `stream` (twice: after validation, and to size
 * col_idx). Each row is formed by one warp from its K = D (d+1) candidate columns, D the number of
 * elements at the row's vertex: duplicates are found by comparing candidates pairwise (O(K^2) work per
 * row) in a shared-memory stage of 5 K bytes per warp, so a vertex may be in at most 40,960 / (d+1)
 * elements (13,653 in 2-D, 10,240 in 3-D) and very high degrees build slowly.
 * Errors: FEM_ERR_ARG (d, N, NT out of range: N < 2^31, NT*(d+1)^2 < 2^31; a vertex degree beyond the
 * limit above; more than 2^31 - 1 structural entries), FEM_ERR_INDEX (bad vertex id), FEM_ERR_OOM,
 * FEM_ERR_CUDA. NT = 0 gives an empty pattern. */
int fem_mesh_build_pattern(int d, int64_t N, int64_t NT, const int32_t* elem, fem_pattern_t* out,
                           fem_stream_t stream);

/* Locality plans of the deterministic value paths (see FEM_PATH_* below). The pattern build makes
 * them from the vertex numbering: the owner-computes plan cuts the vertices into blocks of
 * consecutive ids, one CTA per block's rows; the tile plan orders the elements by their earliest
 * vertex and cuts them into tiles. This call rebuilds both from a geometric order instead: a Morton
 * code of the coordinates `node` [N][d] (device), grouped first by group [N] (device int32,
 * nullable; for example the mesh id in a batch). It also tunes the launch (see
 * fem_pattern_launch_shape and fem_pattern_value_path). The coordinates only choose the order and
 * the timing workload: any values give the same results, and later calls may pass different
 * coordinates. Synchronises `stream`. Rows of more than 32 entries rule out the owner-computes
 * plan, rows of more than 256 entries the tile plan; a mesh with neither takes the two-pass path. */
int fem_pattern_set_locality(fem_pattern_t p, const double* node, const int32_t* group, fem_stream_t stream);
/* The tuned launch of the deterministic value kernel. fem_pattern_set_locality times every feasible
 * combination of rows per block (128, 256, 512), launch shape (threads per CTA x CTAs per SM) and
 * launch mode (one CTA per block, or a persistent wave drawing blocks from a device counter) on the
 * device, assembling with `node` as the geometry (k = 1; 2-D sine-product load, 3-D constant load),
 * and keeps the fastest. Outputs (host, nullable): rows per block, threads per CTA, CTAs per SM,
 * persistent (0/1), and the tuner's time in ms for the chosen launch (0 when not tuned). All are 0
 * when the mesh uses the two-pass path. */
int fem_pattern_launch_shape(fem_pattern_t p, int* rows_per_block, int* threads, int* ctas_per_sm, int* persistent,
                             float* tuned_ms);
/* Override the launch of the deterministic value kernel (the plan's rows per block are kept).
 * Supported shapes: 2-D 512x2, 256x4, 256x2; 3-D 512x1, 256x2, 256x1 (threads x CTAs per SM);
 * persistent 0/1. Every launch gives the same bits. FEM_ERR_ARG if the shape is not supported or the
 * plan does not fit it; FEM_ERR_STATE if the mesh has no blocked plan. */
int fem_pattern_force_launch(fem_pattern_t p, int threads, int ctas_per_sm, int persistent);

/* ---- deterministic value paths --------------------------------------------------------------------
 * All three give every CSR entry as the sum of its element contributions in ascending element order;
 * they differ in where the sums are formed:
 *   FEM_PATH_TILES    elements computed once per tile of 128 or 256 elements in locality order, each
 *                     row's local entries written as packets to the row's incidence slots, then one
 *                     thread per row sums its packets (two launches; float-float arithmetic);
 *   FEM_PATH_TILES_FUSED  the same two phases in one cooperative launch of resident CTAs, tiles and
 *                     row groups taken from device counters, a grid-wide barrier between the phases;
 *   FEM_PATH_BLOCKED  owner-computes blocks of rows, elements on block boundaries computed by every
 *                     block they touch, sums formed in shared memory (one launch; float-float);
 *   FEM_PATH_TWO_PASS per-element FP64 values to scratch, then a per-slot FP64 reduction.
 * TILES, TILES_FUSED and BLOCKED give identical bits. fem_pattern_set_locality times TILES and
 * TILES_FUSED (both tile sizes) against the best BLOCKED launch and keeps the fastest; without
 * coordinates TILES (256) is used. A batch (fem_batch_*) considers the one-launch forms only. */
#define FEM_PATH_TWO_PASS 0
#define FEM_PATH_BLOCKED 1
#define FEM_PATH_TILES 2
#define FEM_PATH_TILES_FUSED 3
/* The path fem_assemble(FEM_DETERMINISTIC) takes, the tile size (0 unless TILES) and the tuner's time
 * for it in ms (0 when not tuned). Outputs are host pointers, nullable. */
int fem_pattern_value_path(fem_pattern_t p, int* path, int* tile_elems, float* tuned_ms);
/* Select the path: TWO_PASS drops both plans; BLOCKED needs the blocked plan (FEM_ERR_STATE if the
 * mesh has none); TILES and TILES_FUSED build the tile plan for tile_elems (128 or 256) if it is not
 * the current one (synchronises `stream`; FEM_ERR_STATE if a row has more than 256 entries, or for
 * TILES_FUSED if its shared memory does not fit). fem_pattern_force_launch selects BLOCKED. */
int fem_pattern_force_path(fem_pattern_t p, int path, int tile_elems, fem_stream_t stream);

/* Fault injection for tests of the bounded wait in FEM_PATH_TILES_FUSED (no counterpart in the paper).
 * The fused launch orders its two phases with a grid-wide barrier: each CTA counts its arrival and
 * polls the count (with a short sleep per poll) until every CTA of the launch has arrived, at most
 * max_polls times; a CTA that gives up records FEM_ERR_TIMEOUT in the device error word and returns
 * without its second phase (val and b are then incomplete). With extra_arrivals > 0 the barrier waits
 * for that many CTAs more than the launch has, arrivals that never come, so every CTA gives up after
 * max_polls polls: the error path can be exercised without a hang. (0, 0) restores the defaults (no
 * extra arrivals; 2^24 polls). The setting belongs to the pattern and applies to its later fused
 * launches. FEM_ERR_ARG for a null pattern or a negative setting. */
int fem_pattern_barrier_fault(fem_pattern_t p, int extra_arrivals, int max_polls);

/* Sizes and library-owned device arrays of a pattern (valid until fem_pattern_destroy):
 * row_ptr [N+1], col_idx [nnz], slot [(d+1)^2 * NT] (layout above). Any output pointer may be NULL. */
int fem_pattern_info(fem_pattern_t p, int* d, int64_t* N, int64_t* NT, int64_t* nnz, const int32_t** row_ptr,
                     const int32_t** col_idx, const int32_t** slot);

void fem_pattern_destroy(fem_pattern_t p);

/* ---- values (Sec. 3.1.3 eq. (dlambda) and the a_ij formula below it; Sec. 3.2) -----------------
 * One pass over the elements: barycentric gradients from the scaled normals n_i, signed measure,
 *   a_ij^tau = k_t * n_i . n_j / (d!^2 |tau|)   (2-D |tau| = |area| as in the paper; 3-D signed)
 * summed into val [nnz] over the pattern (the `sparse(ii, jj, sA)` summation), and the load vector
 *   2-D: b_i += |tau| (f(m_{i+1}) + f(m_{i+2})) / 6, m_q = midpoint of the side opposite vertex q
 *   3-D: b_i += |tau| / 4 * sum_q f(x_q) lambda_i(x_q), points (a,b,b,b) with a = (5+3 sqrt5)/20,
 *        b = (5-sqrt5)/20 (the paper names a 4-point rule without printing it; this is its reading)
 * summed into b [N] (the `accumarray` of Sec. 3.2).
 * node [N][d]; k [NT] per-element coefficient in the caller's element order (NULL means k = 1);
 * val and/or b may be NULL to skip that output; both are overwritten, not accumulated.
 * variant: FEM_DETERMINISTIC or FEM_ATOMIC. A degenerate element sets FEM_ERR_DEGENERATE in the
 * device error word (see fem_get_error); its contribution is then unspecified. */
int fem_assemble(fem_pattern_t p, const double* node, const double* k, int f_kind, const double* f_arg,
                 double* val, double* b, int variant, fem_stream_t stream);
int fem_assemble_stiffness(fem_pattern_t p, const double* node, const double* k, double* val, int variant,
                           fem_stream_t stream);
int fem_assemble_rhs(fem_pattern_t p, const double* node, int f_kind, const double* f_arg, double* b,
                     int variant, fem_stream_t stream);

/* ---- host-resident inputs and outputs -------------------------------------------------------------
 * `steps` assemblies of one pattern from and to host memory (no counterpart in the paper, whose arrays
 * live in one memory). Step i reads node_h[i] [N][d] and k_h[i] [NT] (k_h or k_h[i] NULL: k = 1) and
 * writes val_h[i] [nnz] and b_h[i] [N] (val_h/b_h or an entry NULL: that output is not formed), all
 * HOST pointers; f_kind and f_arg (a DEVICE pointer, as in fem_assemble) are shared by the steps. Each
 * step copies its inputs to device buffers the pattern owns, runs fem_assemble (FEM_DETERMINISTIC) on
 * `stream` and copies its outputs back: the same bits as fem_assemble on device arrays. The steps are
 * pipelined over `stream` and two streams of the pattern's own, with two sets of device buffers: the
 * inputs of step i+1 and the outputs of step i-1 are copied while step i computes. Page-locked host
 * memory lets the copies overlap (pageable memory gives the same results, with less overlap). The call
 * returns when every output is in host memory; later work on `stream` is ordered after it. The first
 * call allocates 2 (N d + NT + nnz + N) doubles of device memory, kept until fem_pattern_destroy.
 * Errors: FEM_ERR_ARG (null pattern or node_h entry, negative steps, misaligned pointer), FEM_ERR_OOM,
 * those of fem_assemble, FEM_ERR_CUDA. */
int fem_assemble_host(fem_pattern_t p, int steps, const double* const* node_h, const double* const* k_h,
                      int f_kind, const double* f_arg, double* const* val_h, double* const* b_h,
                      fem_stream_t stream);

/* ---- boundary (Sec. 1.2, Sec. 3.3) -------------------------------------------------------------
 * is_bd [N] (uint8, overwritten) = 1 for every vertex of a Dirichlet side. Side i of element t is
 * the side opposite vertex i (2-D: vertices (i+1, i+2) mod 3; 3-D: faces [2 4 3], [1 3 4],
 * [1 4 2], [1 2 3] in the paper's 1-based numbering). With bdflag [NT][d+1] (int8), Dirichlet
 * sides are those with bdflag == 1. With bdflag == NULL every side that belongs to exactly one
 * element is Dirichlet ("whole boundary"); that mask depends on the topology only, so the first such
 * call finds it (one pass over the sides) and keeps it in the pattern (N bytes), and later calls copy
 * it. */
int fem_boundary_nodes(fem_pattern_t p, const int8_t* bdflag, uint8_t* is_bd, fem_stream_t stream);

/* ---- Dirichlet (Sec. 3.3) ------------------------------------------------------------------------
 * With u = gD on boundary vertices (0 when gD is NULL) and 0 elsewhere:
 *   b <- b - A u, each (A u)_r summed over row r in ascending column order, s = s + val*u, no FMA;
 *   then the eliminated square system: boundary rows of val become identity rows, boundary
 *   columns of free rows become 0, and b[bd] = gD[bd] (0 when gD is NULL). The pattern is unchanged.
 * free_node (nullable, int32 [N]) receives the free vertices in ascending order; when n_free (a
 * HOST pointer, nullable) is given the call synchronises and stores their count. */
int fem_apply_dirichlet(fem_pattern_t p, const uint8_t* is_bd, const double* gD, double* val, double* b,
                        int32_t* free_node, int64_t* n_free, fem_stream_t stream);

/* ---- other second-order operators on the same element loop (values only) ------------------------
 * FEM_OP_MASS:  m_ij^tau = c_t |tau| (1 + delta_ij) / ((d+1)(d+2)), the exact integral of c lambda_i
 *               lambda_j; coef = c [NT] (device, nullable: c = 1).
 * FEM_OP_ANISO: a_ij^tau = |tau| grad lambda_i^T K_t grad lambda_j = n_i^T K_t n_j / (d!^2 |tau|) (eq.
 *               (dlambda)), the operator -div(K grad u) with a symmetric tensor per element; coef [NT][m]
 *               (device) holds its upper triangle, 2-D m = 3 (xx, xy, yy), 3-D m = 6 (xx, xy, xz, yy, yz, zz).
 * FEM_OP_STIFFNESS: the stiffness matrix with coefficient coef [NT] (= fem_assemble_stiffness).
 * The same pattern, float-float arithmetic and fixed summation order as fem_assemble; mass and
 * anisotropic operators always take the tile path (its plan is built on the first such call if the
 * pattern has none: synchronises). Same element checks (FEM_ERR_DEGENERATE through the error word). */
#define FEM_OP_STIFFNESS 0
#define FEM_OP_MASS 1
#define FEM_OP_ANISO 2
int fem_assemble_operator(fem_pattern_t p, const double* node, int op, const double* coef, double* val,
                          fem_stream_t stream);

/* ---- matrix-free operator --------------------------------------------------------------------------
 * y = A u for the stiffness matrix with coefficient k [NT] (nullable: 1) without forming A: each element
 * recomputes its local matrix (float-float, as fem_assemble) and adds sum_{j != i} a_ij (u_j - u_i) to
 * row i (a_ii = -sum_{j != i} a_ij), summed per row in ascending element order (deterministic). With
 * is_bd [N] (uint8, nullable) the operator is the Dirichlet-eliminated one of fem_apply_dirichlet:
 * eliminated vertices contribute nothing to the free rows and their own rows give y = u. u, y [N]
 * (device, distinct). Uses the tile plan (built on the first call if the pattern has none: synchronises)
 * and its packet buffer. */
int fem_apply_stiffness(fem_pattern_t p, const double* node, const double* k, const double* u, const uint8_t* is_bd,
                        double* y, fem_stream_t stream);

/* ---- reduced solve by conjugate gradients (Sec. 3.3) ------------------------------------------------
 * The paper ends with u(freeNode) = A(freeNode, freeNode) \ b(freeNode) after the boundary lift
 * b <- b - A u_D. This call solves that system by conjugate gradients with the matrix-free operator
 * (fem_apply_stiffness): A is never formed. With u_D = gD on boundary vertices (is_bd [N] uint8, e.g.
 * from fem_boundary_nodes; gD [N] nullable = 0) and 0 elsewhere, it forms r = b - A u_D on the free rows
 * (b [N]: the load vector of fem_assemble, boundary entries ignored; k [NT] nullable = 1), starts from
 * u = u_D and iterates CG on the eliminated operator until ||r||_2 <= rtol ||r_0||_2 or max_iter
 * iterations. u [N] (device, overwritten; distinct from b and gD) receives gD on boundary vertices and
 * the CG iterate on the free ones. Outputs (HOST, nullable): iters = iterations taken, relres =
 * ||r||_2 / ||r_0||_2 (0 when r_0 = 0). Every dot product is a fixed-shape FP64 reduction whose shape
 * depends on N only, so the iterates are bitwise reproducible. Synchronises `stream` every 8 iterations
 * to test convergence; allocates (stream-ordered) and frees 3 N doubles of workspace per call.
 * Errors: FEM_ERR_ARG (null or misaligned arrays, aliasing, max_iter < 0, rtol < 0), FEM_ERR_STATE
 * (breakdown: p.Ap <= 0, i.e. the operator is not positive definite on the free vertices, as for a
 * mesh piece with no boundary vertex; u holds the last iterate), those of fem_apply_stiffness. Element
 * errors of the operator (FEM_ERR_DEGENERATE) surface at fem_get_error. */
int fem_cg_solve(fem_pattern_t p, const double* node, const double* k, const uint8_t* is_bd, const double* b,
                 const double* gD, double* u, int max_iter, double rtol, int* iters, double* relres,
                 fem_stream_t stream);

/* ---- the same solve with the assembled matrix ---------------------------------------------------------
 * fem_csr_spmv: y = A x with the pattern's CSR structure (row_ptr, col_idx) and the values val [nnz]
 * (device; e.g. from fem_assemble_stiffness or fem_assemble), x, y [N] (device, distinct). With is_bd
 * [N] (uint8, nullable) it is the Dirichlet-eliminated operator of fem_apply_dirichlet: a row of an
 * eliminated vertex gives y_i = x_i, and the columns of eliminated vertices are skipped. Each row is
 * summed by one thread in column order (FP64 multiply-adds), so the result is bitwise reproducible; it
 * agrees with fem_apply_stiffness within rounding. Errors: FEM_ERR_ARG (null or misaligned arrays,
 * x == y).
 * fem_cg_solve_csr: the reduced solve of fem_cg_solve (same arguments, outputs, stopping rule and
 * errors) with the operator fem_csr_spmv of the assembled values val instead of the matrix-free one:
 * the matrix is formed once, and an iteration reads val and col_idx instead of recomputing the elements.
 * The paper's own route: A is assembled (Sec. 3.1), then solved on freeNode (Sec. 3.3). */
int fem_csr_spmv(fem_pattern_t p, const double* val, const double* x, const uint8_t* is_bd, double* y,
                 fem_stream_t stream);
int fem_cg_solve_csr(fem_pattern_t p, const double* val, const uint8_t* is_bd, const double* b, const double* gD,
                     double* u, int max_iter, double rtol, int* iters, double* relres, fem_stream_t stream);

/* ---- load vector with rules of any order ("Numerical Quadrature") ---------------------------------
 * I_n(f) = |tau| sum_q w_q f(p_q) on each simplex, with the conical-product Gauss rule of n points per
 * direction (n^d points, exact for total degree 2n - 1; 1 <= n <= FEM_RULE_MAX_N), built by the library
 * from Gauss-Legendre and Gauss-Jacobi rules under the collapsed map of the unit square / cube.
 * fem_quad_rule (HOST, no GPU needed): barycentric points bary [nq][d+1] and weights w [nq] (sum 1),
 *   nq = n^d; any output may be NULL.
 * fem_rule_points: the physical points of every element, pts [NT][nq][d] (device).
 * fem_assemble_rhs_rule: b [N] (device, overwritten) with b_i = sum over elements of
 *   |tau| sum_q w_q f(p_q) lambda_i(p_q); f_kind FEM_F_CONST (f_arg: 1 value or NULL = 1), FEM_F_SINPROD,
 *   or FEM_F_QPVALUES (f_arg [NT][nq], the values at the points of fem_rule_points). Float-float
 *   arithmetic, per-vertex sums in ascending element order (deterministic). Uses the pattern's scratch. */
#define FEM_RULE_MAX_N 8
int fem_quad_rule(int d, int n, double* bary, double* w, int* nq);
int fem_rule_points(fem_pattern_t p, const double* node, int n, double* pts, fem_stream_t stream);
int fem_assemble_rhs_rule(fem_pattern_t p, const double* node, int n, int f_kind, const double* f_arg, double* b,
                          fem_stream_t stream);

/* ---- Neumann and Robin sides, pure-Neumann fixes ("Boundary conditions", Sec. 3.3) --------------
 * Side j of element t is the side opposite local vertex j; bdflag [NT][d+1] (int8, device) = 2 marks it
 * Neumann, 3 Robin (du/dn + alpha u = g). Its vertices are the element's other d vertices; |s| is the
 * edge length (2-D) or triangle area (3-D). g is the side's value at its quadrature point, the midpoint
 * (2-D, the paper's rule) or centroid (3-D): g_side [NT][d+1] (device, nullable: g_const for every side).
 * Adds to b (nullable) |s| g / d for each vertex of each flagged side, and to val (nullable) for each
 * Robin side alpha |s| (1 + delta_ab) / (d (d+1)) at the CSR entry of every pair (a, b) of its vertices
 * (the side mass matrix). Each row is updated by one thread in ascending element order, then ascending
 * side, with uncontracted FP64 operations: deterministic. Flags 0 and 1 are ignored. */
int fem_boundary_terms(fem_pattern_t p, const double* node, const int8_t* bdflag, const double* g_side, double g_const,
                       double alpha, double* val, double* b, fem_stream_t stream);
/* The quadrature point of every side (the mean of its vertices): pts [NT][d+1][d] (device). */
int fem_side_points(fem_pattern_t p, const double* node, double* pts, fem_stream_t stream);
/* Pure Neumann compatibility: x <- x - mean(x) for a device array of n doubles; the sum is a fixed-shape
 * FP64 reduction (deterministic). Allocates a few KB of stream-ordered scratch. */
int fem_mean_shift(double* x, int64_t n, fem_stream_t stream);
/* Zero average: u <- u - c with c = sum_t mean(u over tau_t) |tau_t| / sum_t |tau_t| (2-D |area|, 3-D
 * signed volume), the constraint that fixes the constant of a pure-Neumann solution; c_out (device,
 * nullable) receives c. Fixed-shape FP64 reduction (deterministic). */
int fem_zero_average(fem_pattern_t p, const double* node, double* u, double* c_out, fem_stream_t stream);

/* ---- backward (gradients of the assembled system) ----------------------------------------------
 * For L = sum_s w[s] val[s] + sum_i r[i] b[i] (w [nnz], r [N]; either may be NULL = 0), writes
 * gnode [N][d] = dL/dnode and gk [NT] = dL/dk (either may be NULL to skip). The basis gradients are
 * recomputed from node, not stored. Derivatives follow from eq. (dlambda): d|tau|/dx_m = |tau| g_m
 * and dg_i/dx_m = -g_m g_i^T with g_i = grad lambda_i. f_kind FEM_F_QPVALUES contributes only
 * through |tau| and the point weights (the values are inputs). Node gradients are summed over the
 * incident elements in ascending element order (deterministic). The gradient of |tau| needs the
 * orientation: a 2-D element must be counter-clockwise and a 3-D element positively oriented, else
 * FEM_ERR_DEGENERATE. Arithmetic is float-float (about 2^-44 relative per operation); each output
 * is rounded to double once. */
int fem_assemble_backward(fem_pattern_t p, const double* node, const double* k, int f_kind, const double* f_arg,
                          const double* w, const double* r, double* gnode, double* gk, fem_stream_t stream);

/* ---- batched assembly of many independent meshes -----------------------------------------------
 * B meshes of dimension d; mesh m has N[m] vertices and NT[m] elements (HOST arrays). elem_cat is
 * the DEVICE concatenation of the meshes' elem arrays with each mesh's own 0-based vertex ids. The
 * plan builds the block-diagonal pattern of all meshes at once (vertex ids offset by the preceding
 * meshes' N) and tunes the launch shape of the batched value kernel on the device (synchronises).
 * Offsets (HOST, int64, B+1 entries each, owned by the plan): node_off, elem_off, nnz_off. */
int fem_batch_plan(int d, int B, const int64_t* N, const int64_t* NT, const int32_t* elem_cat, fem_batch_t* out,
                   fem_stream_t stream);
int fem_batch_info(fem_batch_t bt, int* B, const int64_t** node_off, const int64_t** elem_off,
                   const int64_t** nnz_off, fem_pattern_t* pattern);
/* Locality plan and launch tuning for the batch (fem_pattern_set_locality on the block-diagonal
 * pattern, with the vertices grouped by mesh): node_cat [sum N][d] (device) orders and times the
 * plan. Synchronises. */
int fem_batch_set_locality(fem_batch_t bt, const double* node_cat, fem_stream_t stream);
/* One persistent launch over all meshes' elements (work tiles taken from a device counter), plus
 * the per-slot reduction: node_cat [sum N][d], k_cat [sum NT] (nullable), val_cat [sum nnz],
 * b_cat [sum N] (either output nullable). No allocation and no host synchronisation, so the call
 * can be captured in a CUDA graph. */
int fem_batch_assemble(fem_batch_t bt, const double* node_cat, const double* k_cat, int f_kind, const double* f_arg,
                       double* val_cat, double* b_cat, int variant, fem_stream_t stream);
/* Same work, replayed from a CUDA graph the plan captures on first use for these exact pointers
 * (re-captured when any pointer or argument changes). */
int fem_batch_assemble_graph(fem_batch_t bt, const double* node_cat, const double* k_cat, int f_kind,
                             const double* f_arg, double* val_cat, double* b_cat, int variant, fem_stream_t stream);
void fem_batch_destroy(fem_batch_t bt);

/* ---- allocation-free assembly --------------------------------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that cannot allocate device
 * memory while they assemble. One example is an application that hands all device memory to its own
 * pool at start-up. Another is a loop with a fixed latency budget, where the implicit device
 * synchronisation of an allocation is unacceptable.
 * Arguments as fem_assemble with FEM_DETERMINISTIC. It always runs the FP64 two-pass kernels (per-element
 * FP64 values into the scratch, then per-slot FP64 sums in ascending element order), so its values are
 * bitwise those of fem_assemble on the same pattern after fem_pattern_force_path(FEM_PATH_TWO_PASS),
 * bitwise the same from call to call, and within the parity tolerance (1e-12 of each entry's magnitude)
 * of fem_assemble's default float-float paths, whose bits differ. It calls no cudaMalloc, cudaFree or
 * other allocating routine. Its per-element scratch lives in a fixed device array of
 * FEM_NOALLOC_SCRATCH_DOUBLES doubles (16 MiB), compiled into the library. Every GPU that loads the
 * library holds that array until the process exits.
 *  - Size limit: d = 2 meshes up to FEM_NOALLOC_SCRATCH_DOUBLES / 9 = 233,016 elements, d = 3 up to
 *    FEM_NOALLOC_SCRATCH_DOUBLES / 14 = 149,796 elements. Larger meshes return FEM_ERR_ARG and
 *    launch nothing.
 *  - Set-up, two preconditions: (1) the pattern p was built (fem_mesh_build_pattern) on the current
 *    device, which also makes the device error word this call reports through (FEM_ERR_STATE
 *    otherwise); (2) the first call on a device (with that device current) looks up the array's device
 *    address with cudaGetSymbolAddress and caches it. Build the pattern and make that first call before
 *    any stream capture.
 *  - Sharing: all calls on a device share the one array, which keeps the last call's contents.
 *    Every call overwrites the scratch it reads, and val/b are cleared before they are
 *    accumulated. Calls that overlap on the GPU (for example on two streams at once) race on the
 *    array and produce wrong results: serialise them. */
#define FEM_NOALLOC_SCRATCH_DOUBLES ((int64_t)1 << 21)
int fem_assemble_noalloc(fem_pattern_t p, const double* node, const double* k, int f_kind, const double* f_arg,
                         double* val, double* b, fem_stream_t stream);

/* ---- errors and counters -----------------------------------------------------------------------*/
/* Synchronises `stream`, returns the first error recorded by a kernel since the last call on this
 * device (FEM_OK if none), and clears it. */
int fem_get_error(fem_stream_t stream);
/* Host message for the last failed call in this process (static storage; never NULL). */
const char* fem_last_error_string(void);
/* Number of kernels this library has launched in this process (all devices). */
int64_t fem_launch_count(void);
/* Per-kernel timing, off by default. When on, every kernel launch outside stream capture is
 * bracketed by CUDA events recorded on its own stream. fem_timing_report synchronises those events,
 * writes one line "kernel_name launches total_ms" per kernel into buf (HOST, buflen bytes,
 * NUL-terminated, truncated to fit) and clears the records. */
int fem_timing_enable(int on);
int fem_timing_report(char* buf, int64_t buflen);

#ifdef __cplusplus
}
#endif

#endif /* FEMASM_H */
