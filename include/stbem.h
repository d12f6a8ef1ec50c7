/*
 * stbem.h -- C ABI of the GB300 space-time boundary element library for the
 * 3D heat equation (Zapletal, Watschinger, Of, Merta: "Semi-analytic
 * integration for a parallel space-time boundary element method modeling the
 * heat equation").
 *
 * The library assembles the blocks V^d and K^d of the block lower-triangular
 * Toeplitz Galerkin matrices V_h and K_h (Sec. 3.1, eq. V_mat, eq. V_blocks;
 * Sec. 3.2, eq. K_mat) for piecewise-constant test and trial functions on a
 * tensor-product space-time mesh with uniform steps, applies the
 * block-Toeplitz matrix-vector product, builds the Dirichlet right-hand side
 * (1/2 M_h + K_h) g and solves V_h w = (1/2 M_h + K_h) g (Sec. 3.4) by block
 * forward substitution in time.  Every computation runs in the library's own
 * sm_103a CUDA kernels.
 *
 * Conventions
 *   - Host arrays (nodes, tris, sources given to stb_mesh_create /
 *     stb_project_dirichlet) are read during the call and not retained.
 *   - Device arrays are caller-owned, allocated by the caller (cudaMalloc,
 *     PyTorch, ...) on the current device; the library never frees them.
 *   - Scratch memory is caller-owned too: query its size with the matching
 *     *_workspace_size call and pass a device buffer of at least that many
 *     bytes, 256-byte aligned.
 *   - Calls are asynchronous on the given stream unless stated otherwise;
 *     argument and mesh errors are returned immediately.  Device-side errors
 *     (a non-positive pivot, an exhausted bounded wait) are written to a status
 *     word in the workspace and returned by the calls that synchronise
 *     (stb_dirichlet_solve) or by stb_workspace_status.
 *   - No C++ exception crosses this interface.  Functions are thread-safe
 *     except that calls sharing one workspace must not overlap on the GPU.
 *   - Mesh: nodes [n_nodes][3] (double), tris [E][3] (int32), vertex order
 *     counter-clockwise seen from outside (outward normals).  The surface must
 *     be a closed, conforming, consistently oriented 2-manifold of
 *     non-degenerate flat triangles.
 *   - Time grid t_i = i h, h = T / n_steps.  Block d = 0..n_steps-1 of a
 *     Toeplitz matrix is the E x E row-major array A[d][l][j] (row l = test
 *     triangle, column j = trial triangle); a whole matrix is
 *     A[n_steps][E][E], contiguous.
 *   - Space-time vectors are laid out [nrhs][n_steps][E] (time step k holds
 *     the coefficients of interval (t_k, t_{k+1})).
 */
#ifndef STBEM_H
#define STBEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *stb_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef int32_t stb_status;
#define STB_OK 0
#define STB_ERR_INVALID_ARG (-1)   /* a pointer, size or parameter is invalid   */
#define STB_ERR_BAD_MESH (-2)      /* not a closed oriented manifold / degenerate */
#define STB_ERR_NOMEM (-3)         /* a library allocation failed                */
#define STB_ERR_CUDA (-4)          /* a CUDA runtime call failed                 */
#define STB_ERR_NOT_SPD (-5)       /* V^0 has a non-positive pivot               */
#define STB_ERR_NOT_CONVERGED (-6) /* iterative refinement did not converge      */
#define STB_ERR_TIMEOUT (-7)       /* a bounded device-side wait expired         */
#define STB_ERR_WORKSPACE (-8)     /* workspace missing, too small or misaligned */

/* Arithmetic of the assembly. */
#define STB_PREC_FP64 0  /* every quadrature point and time level in FP64 (the paper's) */
#define STB_PREC_MIXED 1 /* FP32 quadrature points in cancellation-free forms (block error
                            <= 2e-6 stated), FP32 solve inside iterative refinement whose
                            residual products run on the tensor cores with split operands */

/* Element type of V/K storage. */
#define STB_STORE_F64 0
#define STB_STORE_F32 1

/* Flags (stb_params.flags).
 * STB_FLAG_NO_SYNC: the call only enqueues device work.  No host
 *   synchronisation and no copy from pageable host memory (host arrays such
 *   as the sources must then be page-locked), so a sequence of such calls
 *   can be captured into a CUDA graph and replayed.  The mixed solve then
 *   runs a fixed number of refinement steps, STB_FLAG_REFINE(n) (n = 1..15,
 *   default 1), e.g. the count a synchronous solve of the same problem
 *   reported, and writes its convergence into the workspace status word
 *   (STB_ERR_NOT_CONVERGED if ||f - V_h w|| > 1e-10 ||f||), read afterwards by
 *   stb_workspace_status or stb_solve_report.  stb_assemble uploads its
 *   tables from pageable host memory and does not take the flag; graphs
 *   capture stb_batch_launch after stb_batch_prepare instead. */
#define STB_FLAG_NO_SYNC 1
#define STB_FLAG_REFINE(n) (((n) & 15) << 8)

typedef struct stb_params {
    double alpha;          /* heat capacity constant alpha > 0 (eq. heat_eq)           */
    double T;              /* end time T > 0                                            */
    int32_t n_steps;       /* E_t >= 1 uniform time steps                               */
    int32_t quad_regular;  /* q: q x q conical product rule per triangle (eq. st), 1..16 */
    int32_t quad_singular; /* m: m^4 Gauss points per sub-domain (eq. ss), 1..12         */
    int32_t precision;     /* STB_PREC_*                                                */
    int32_t storage;       /* STB_STORE_*                                               */
    int32_t flags;         /* STB_FLAG_* bits, 0 = none                                  */
} stb_params;

/* Default parameters (q = 3, m = 4, FP64, F64 storage) for given alpha, T, E_t. */
stb_params stb_default_params(double alpha, double T, int32_t n_steps);

const char *stb_status_string(stb_status status);
/* Message of the last error raised on the calling thread ("" if none). */
const char *stb_last_error_message(void);
/* Number of kernels this library has launched in the process so far. */
int64_t stb_launch_count(void);

/* ---- mesh (Sec. 3: the spatial mesh Gamma_h of flat triangles) ---------------
 * Validates the surface, copies nodes and tris to device memory owned by the
 * mesh object (O(E) bytes on the current device) and counts the touching
 * triangle pairs.  Synchronous.  Errors: INVALID_ARG, BAD_MESH, NOMEM, CUDA. */
typedef struct stb_mesh stb_mesh;
stb_status stb_mesh_create(const double *nodes, int64_t n_nodes, const int32_t *tris,
                           int64_t n_tris, stb_mesh **out);
void stb_mesh_destroy(stb_mesh *mesh);
/* Counts: nodes, triangles, and unordered touching pairs (a <= b sharing at
 * least one vertex, the identical pairs included). */
stb_status stb_mesh_info(const stb_mesh *mesh, int64_t *n_nodes, int64_t *n_tris,
                         int64_t *n_touching_pairs);

/* ---- assembly of V_h and K_h (Sec. 3.1-3.2, Sec. 5) ------------------------------
 * Writes all blocks V^d and K^d, d = 0..n_steps-1, each E x E, in the layout
 * above (element type per params->storage).  Every entry is
 *   V^d[l][j] = int_{gamma_l} int_{gamma_j} V^d(x - y) ds_y ds_x
 * with V^d(r) from eq. vd (d >= 1) and eq. V0 (d = 0), K^d likewise from
 * eq. K_d / eq. K0, computed as second differences of the time-level sums
 * S_i = int int G^{dtau dt}(x - y, i h) (each level evaluated once, Table
 * deltad); separated pairs use the regular rule (eq. quad_reg, eq. st),
 * pairs sharing a vertex, an edge or the whole triangle the regularised rules
 * (eq. quad_duffy, eq. ss) at every time level.  K may be NULL (V only).
 * The kernels compute triangle geometry and the pair classification in the
 * workspace first.  Asynchronous on `stream`. */
stb_status stb_assemble_workspace_size(const stb_mesh *mesh, const stb_params *params,
                                       size_t *bytes);
stb_status stb_assemble(const stb_mesh *mesh, const stb_params *params, void *V, void *K,
                        void *workspace, size_t workspace_bytes, stb_stream stream);

/* ---- many problems in one launch (no counterpart in the paper) -------------------
 * Mixed-precision assembly (eq. V_mat / eq. K_mat blocks, as stb_assemble with
 * STB_PREC_MIXED and STB_STORE_F32) of n independent problems, each with its
 * own mesh, parameters (alpha, T, n_steps, quadrature orders) and output
 * blocks.  All pair classes of all problems run in one persistent launch
 * whose CTAs claim work items from a device counter: first every touching
 * pair (identical, shared edge, shared vertex; one item each), then the
 * separated pairs as (problem, row, block of `tile` columns), so meshes of
 * uneven size and step count share the SMs.  Per problem there are in
 * addition three small set-up launches (geometry, classification).
 * tile: columns per work item (= threads per CTA), 128 or 256; the touching
 * pairs run on 128 threads of a CTA either way, so every tile writes the
 * same blocks as stb_assemble; 0 = the value stb_batch_tune
 * chose on this device for a batch of the same shape (128 if none).
 * The workspace is shared by all items (stb_batch_workspace_size). */
typedef struct {
    const stb_mesh *mesh;
    stb_params params; /* precision STB_PREC_MIXED, storage STB_STORE_F32 */
    float *V;          /* device [params.n_steps][E][E] */
    float *K;          /* device, same shape; NULL: V only */
} stb_batch_item;
stb_status stb_batch_workspace_size(const stb_batch_item *items, int32_t n, size_t *bytes);
/* = stb_batch_prepare + stb_batch_launch. */
stb_status stb_batch_assemble(const stb_batch_item *items, int32_t n, int32_t tile,
                              void *workspace, size_t workspace_bytes, stb_stream stream);
/* Set-up: uploads every problem's tables and the work-item descriptors for
 * this tile from host memory, then computes geometry and pair classes.  Not
 * capturable into a CUDA graph; call once for a workspace. */
stb_status stb_batch_prepare(const stb_batch_item *items, int32_t n, int32_t tile,
                             void *workspace, size_t workspace_bytes, stb_stream stream);
/* The batched launches only (same items, tile and workspace as the preceding
 * stb_batch_prepare): a device memset and two kernels, no host
 * synchronisation and no host copy, so the call can be captured into a CUDA
 * graph and replayed. */
stb_status stb_batch_launch(const stb_batch_item *items, int32_t n, int32_t tile,
                            void *workspace, size_t workspace_bytes, stb_stream stream);
/* Tile autotuner: times the separated-pair launch of this batch on a sample
 * (every 16th work item) for tile = 64, 128 and 256 with CUDA events, keeps
 * the fastest for batches of the same shape on this device (used by tile = 0)
 * and returns it in *tile.  It writes into the items' blocks (assemble
 * afterwards) and synchronises `stream`. */
stb_status stb_batch_tune(const stb_batch_item *items, int32_t n, void *workspace,
                          size_t workspace_bytes, stb_stream stream, int32_t *tile);

/* ---- double layer with piecewise-linear trial functions (Sec. 3.2) -------------
 * K1: device [n_steps][E][n_nodes] of params->storage (the caller's buffer,
 * overwritten).  K1^d[l][i] is the block-d entry of K_h between the constant
 * test function of triangle l and the nodal hat function phi_i of X_h^{1,0}
 * (continuous, piecewise linear in space): the K integrand of stb_assemble
 * weighted by the barycentric coordinate of node i at the trial point, by the
 * same rules (regular Gauss for separated pairs, the regularised rules for
 * touching pairs; identical pairs give zero since r . n_y = 0) and the same
 * second differences in time (eq. K0, eq. K_d).  Needs STB_PREC_FP64.  The
 * contributions of the triangles around node i are added with atomics, so
 * two runs may differ in the last bits.  Workspace from
 * stb_assemble_k1_workspace_size; the device status word reports as for
 * stb_assemble. */
stb_status stb_assemble_k1_workspace_size(const stb_mesh *mesh, const stb_params *params,
                                          size_t *bytes);
stb_status stb_assemble_k1(const stb_mesh *mesh, const stb_params *params, void *K1,
                           void *workspace, size_t workspace_bytes, stb_stream stream);

/* ---- Dirichlet data (Sec. 3.4, Sec. 6.1) --------------------------------------
 * sources: HOST array [nrhs][n_src][5] of (y1, y2, y3, t0, weight); right-hand
 * side r has the Dirichlet datum g_r(x,t) = sum_s weight_s G_alpha(x - y_s, t - t0_s)
 * (the exterior-source exact solution of Sec. 6.1).  g (device, [nrhs][n_steps][E])
 * receives its L2 projection into piecewise constants (element means) by a
 * q_space x q_space conical rule and n_time Gauss points per step, in FP64
 * (STB_PREC_FP64) or FP32 arithmetic (STB_PREC_MIXED). */
stb_status stb_project_workspace_size(const stb_mesh *mesh, int32_t nrhs, int32_t n_src,
                                      int32_t q_space, int32_t n_time, size_t *bytes);
stb_status stb_project_dirichlet(const stb_mesh *mesh, const stb_params *params,
                                 const double *sources, int32_t nrhs, int32_t n_src,
                                 int32_t q_space, int32_t n_time, double *g, void *workspace,
                                 size_t workspace_bytes, stb_stream stream);

/* ---- piecewise-linear Dirichlet data (Sec. 3.4) ---------------------------------
 * g1 (device FP64 [nrhs][n_steps][n_nodes]) receives the L2(Sigma_h)
 * projection of g_r (sources as for stb_project_dirichlet) into
 * X_h^{1,0} x (piecewise constants in time): per step k, M1 g1^k = b^k with
 * the hat-function mass matrix M1[i][i'] = sum over the triangles j holding
 * both nodes of Delta_j (1 + [i = i']) / 12 and the moments
 * b^k_i = h^{-1} int_{t_k}^{t_{k+1}} int_Gamma g_r phi_i (q_space x q_space
 * conical rule, n_time Gauss points; FP64, or FP32 moments with
 * STB_PREC_MIXED).  M1 is inverted densely in FP64 (n_nodes <= 65535; every
 * node must belong to a triangle, else STB_ERR_INVALID_ARG).  The moments
 * are added with atomics (last bits may differ between runs). */
stb_status stb_project_p1_workspace_size(const stb_mesh *mesh, const stb_params *params,
                                         int32_t nrhs, int32_t n_src, int32_t q_space,
                                         int32_t n_time, size_t *bytes);
stb_status stb_project_dirichlet_p1(const stb_mesh *mesh, const stb_params *params,
                                    const double *sources, int32_t nrhs, int32_t n_src,
                                    int32_t q_space, int32_t n_time, double *g1, void *workspace,
                                    size_t workspace_bytes, stb_stream stream);
/* f (device FP64 [nrhs][n_steps][E], overwritten) = (1/2 M_h + K_h) g1 with
 * piecewise-linear data: K_h = K1 of stb_assemble_k1 (params->storage) as a
 * block-Toeplitz product with E x n_nodes blocks, and the p0 x p1 mass
 * M_h = h blockdiag(M01), M01[l][i] = int_{gamma_l} phi_i = Delta_l / 3 for
 * the three nodes i of triangle l.  FP64 arithmetic for either storage. */
stb_status stb_rhs_p1_workspace_size(const stb_mesh *mesh, const stb_params *params, int32_t nrhs,
                                     size_t *bytes);
stb_status stb_dirichlet_rhs_p1(const stb_mesh *mesh, const stb_params *params, const void *K1,
                                const double *g1, int32_t nrhs, double *f, void *workspace,
                                size_t workspace_bytes, stb_stream stream);

/* ---- potentials: the representation formula at points off Gamma (Sec. 3.5) --------
 * u_h(x,t) = V~ w_h(x,t) - W u_h(x,t) (eq. repr).  points: device FP64
 * [n_pts][4] = (x1, x2, x3, t) with 0 <= t <= T and x off Gamma_h (a point on
 * Gamma_h divides by zero); a time outside [0, T] leaves STB_ERR_INVALID_ARG
 * in the workspace status word and that point's outputs at zero.
 * w: device FP64 [nrhs][n_steps][E] (piecewise constant, e.g. the solution
 * of stb_dirichlet_solve); u1: device FP64 [nrhs][n_steps][n_nodes] (piecewise
 * linear in space, e.g. the data of stb_project_dirichlet_p1).
 * slp = V~ w_h, dlp = W u_h: device FP64 [nrhs][n_pts]; either may be NULL
 * (then its density is not read).  With t = t_k + eps, k = min(floor(t/h),
 * E_t - 1), both are the paper's sums over the past steps of antiderivative
 * differences (eq. G_dtau, eq. dn_G_dtau and their delta = 0 limits), formed
 * in FP64 with a q_space x q_space conical rule per triangle
 * (1 <= q_space <= 5); params->precision = STB_PREC_MIXED forms the
 * antiderivative values from FP32 rule points (x - P0 of each triangle in
 * FP64, rounded once) and sums them over the levels in FP64. */
stb_status stb_potentials_workspace_size(const stb_mesh *mesh, const stb_params *params,
                                         int32_t nrhs, int64_t n_pts, int32_t q_space,
                                         size_t *bytes);
stb_status stb_potentials(const stb_mesh *mesh, const stb_params *params, const double *points,
                          int64_t n_pts, const double *w, const double *u1, int32_t nrhs,
                          int32_t q_space, double *slp, double *dlp, void *workspace,
                          size_t workspace_bytes, stb_stream stream);
/* The same potentials at every step for fixed points: points3 device FP64
 * [n_pts][3] (n_pts <= 65535 per call), times t_k + eps for k = 0..n_steps-1
 * with one 0 <= eps <= T/n_steps; slp, dlp: device FP64 [nrhs][n_steps][n_pts].
 * The antiderivative at level d h + eps does not depend on k, so it is
 * evaluated once per (point, triangle, rule point, level) into level blocks
 * of n_steps x n_pts x E (single layer) and n_steps x n_pts x n_nodes (double
 * layer, accumulated per node with atomics) in the workspace, and the
 * potentials are block-Toeplitz products of these blocks with the backward
 * differences of the densities in time (FP64).  params->precision =
 * STB_PREC_MIXED evaluates the level blocks from FP32 quadrature points
 * (distances and weights formed in FP64; FP32 blocks, FP32 atomics for the
 * double layer; the products in double-float arithmetic, FP64 results).
 * Workspace from
 * stb_potentials_grid_workspace_size (about 8 n_steps n_pts (E + n_nodes)
 * bytes). */
stb_status stb_potentials_grid_workspace_size(const stb_mesh *mesh, const stb_params *params,
                                              int32_t nrhs, int64_t n_pts, int32_t q_space,
                                              size_t *bytes);
stb_status stb_potentials_grid(const stb_mesh *mesh, const stb_params *params,
                               const double *points3, int64_t n_pts, double eps, const double *w,
                               const double *u1, int32_t nrhs, int32_t q_space, double *slp,
                               double *dlp, void *workspace, size_t workspace_bytes,
                               stb_stream stream);

/* ---- hypersingular operator and the Neumann problem (Sec. 3.3, Sec. 3.4) ----------
 * D: device [n_steps][n_nodes][n_nodes] of params->storage (overwritten) receives
 * D_h = D_h^1 + D_h^2 on X_h^{1,0}: D^{1,d} = T^T (alpha^2 V^d (x) I_3) T
 * (eq. D_1_sp_trafo, T the surface curls of the hat functions on every
 * triangle) from the caller's single-layer blocks V (device [n_steps][E][E],
 * same storage, as assembled by stb_assemble), and D^{2,d} (eq. D2d: second
 * differences in time of G^{dtau}, weighted by n_x . n_y phi_i(x) phi_j(y)) by
 * the rules of stb_assemble.  Needs STB_PREC_FP64, n_nodes <= 65535 and at most
 * 32 triangles per node; the D^2 contributions are added with atomics (last
 * bits may differ between runs). */
stb_status stb_assemble_d_workspace_size(const stb_mesh *mesh, const stb_params *params,
                                         size_t *bytes);
stb_status stb_assemble_d(const stb_mesh *mesh, const stb_params *params, const void *V, void *D,
                          void *workspace, size_t workspace_bytes, stb_stream stream);
/* hd (device FP64 [nrhs][n_steps][E], overwritten): the L2 projection of the
 * Neumann datum w_r = alpha du_r/dn of the sources (as for
 * stb_project_dirichlet, whose workspace size it shares) into X_h^{0,0}. */
stb_status stb_project_neumann(const stb_mesh *mesh, const stb_params *params,
                               const double *sources, int32_t nrhs, int32_t n_src,
                               int32_t q_space, int32_t n_time, double *hd, void *workspace,
                               size_t workspace_bytes, stb_stream stream);
/* f (device FP64 [nrhs][n_steps][n_nodes], overwritten) = (1/2 M_h^{T_x} -
 * K_h^{T_x}) hd: K1 of stb_assemble_k1 transposed blockwise (Sec. 3.2's
 * remark) as a block-Toeplitz product, and the transposed p0 x p1 mass
 * (Delta_l / 3 to each node of l).  FP64 arithmetic for either storage. */
stb_status stb_neumann_rhs_workspace_size(const stb_mesh *mesh, const stb_params *params,
                                          int32_t nrhs, size_t *bytes);
stb_status stb_neumann_rhs(const stb_mesh *mesh, const stb_params *params, const void *K1,
                           const double *hd, int32_t nrhs, double *f, void *workspace,
                           size_t workspace_bytes, stb_stream stream);
/* D_h u = f by the block forward substitution of stb_dirichlet_solve with
 * n_nodes x n_nodes blocks (D^0 symmetric positive definite): u, f device FP64
 * [nrhs][n_steps][n_nodes]; same precisions, flags and reports. */
stb_status stb_neumann_solve_workspace_size(const stb_mesh *mesh, const stb_params *params,
                                            int32_t nrhs, size_t *bytes);
stb_status stb_neumann_solve(const stb_mesh *mesh, const stb_params *params, const void *D,
                             const double *f, int32_t nrhs, double *u, void *workspace,
                             size_t workspace_bytes, stb_stream stream);
/* out[0] = sum_r ||g_r - u_h,r||^2, out[1] = sum_r ||g_r||^2 in L2(Sigma_h) for
 * piecewise-linear u1 (device FP64 [nrhs][n_steps][n_nodes]) against the
 * Dirichlet datum of the sources; workspace of stb_error_workspace_size. */
stb_status stb_dirichlet_error_p1(const stb_mesh *mesh, const stb_params *params,
                                  const double *sources, int32_t nrhs, int32_t n_src,
                                  const double *u1, int32_t q_space, int32_t n_time, double *out,
                                  void *workspace, size_t workspace_bytes, stb_stream stream);

/* ---- V_h and the right-hand side without storing K_h (matrix-free K g) ----------
 * For the Dirichlet problem with piecewise-constant data: V (device FP32
 * [n_steps][E][E], overwritten) as stb_assemble writes it, and f (device FP64
 * [nrhs][n_steps][E], overwritten) = (1/2 M_h + K_h) g for g (device FP64
 * [nrhs][n_steps][E]), the blocks of K_h contracted with g as they are formed
 * (never stored: half the memory of the assembly).  Needs STB_PREC_MIXED,
 * STB_STORE_F32 and nrhs * n_steps <= 128.  The products of K with g are
 * summed in FP32 per CTA of 128 columns and added in FP64 (relative error of
 * the order of the mixed block error); atomics: last bits may differ between
 * runs. */
stb_status stb_assemble_vrhs_workspace_size(const stb_mesh *mesh, const stb_params *params,
                                            int32_t nrhs, size_t *bytes);
stb_status stb_assemble_vrhs(const stb_mesh *mesh, const stb_params *params, void *V,
                             const double *g, int32_t nrhs, double *f, void *workspace,
                             size_t workspace_bytes, stb_stream stream);

/* ---- non-uniform time grids (Sec. 7: the antiderivatives carry over) ------------
 * times: HOST FP64 [n_steps + 1], times[0] = 0, strictly increasing
 * (params->n_steps steps; params->T is not used).  The matrices stay block
 * lower triangular but are not Toeplitz: blocks A^{k,i}, k >= i, packed at
 * b(k,i) = k(k+1)/2 + i, each E x E FP64 row-major.
 * stb_assemble_nu: V, K (device FP64 [n_steps(n_steps+1)/2][E][E],
 *   overwritten): A^{k,i} = S(t_{k+1}-t_{i+1}) - S(t_k-t_{i+1}) - S(t_{k+1}-t_i)
 *   + S(t_k-t_i) for k > i and h_k S_*(0) - S(h_k) + S(0) on the diagonal
 *   (eq. V0 / eq. K0 with the local step), S the pair's spatial sum of
 *   G^{dtau dt} (or its scaled normal derivative) by the rules of
 *   stb_assemble; every distinct time difference is evaluated once per
 *   point.  STB_PREC_MIXED: the same blocks from FP32 quadrature points,
 *   written as the time integral of the pair's kernel against the overlap
 *   weight of the two intervals (closed forms where the weight reaches lag
 *   0, Gauss-Legendre nodes on its linear pieces elsewhere; stated bound as
 *   for stb_assemble's mixed path: relative Frobenius error per block
 *   <= 2e-6 against FP64), still stored FP64.  Needs STB_STORE_F64,
 *   n_steps <= 256.
 * stb_matvec_nu: y^k = sum_{i <= k} A^{k,i} x^i (x, y device FP64
 *   [nrhs][n_steps][E]).
 * stb_solve_nu: w^k = (V^{k,k})^{-1} (f^k - sum_{i<k} V^{k,i} w^i), every
 *   diagonal block inverted (blocked Cholesky); synchronises `stream`.
 * stb_project_dirichlet_nu / stb_neumann_error_nu / stb_dirichlet_rhs_nu:
 *   the data projection, the L2(Sigma_h) error and f = (1/2 M_h + K_h) g
 *   (M_h = blockdiag(h_k diag(Delta_l))) on the grid; sources as for
 *   stb_project_dirichlet; the first two share stb_project_nu_workspace_size.
 * stb_assemble_nu_mixed_counts: host only (no device work): the sizes of the
 *   STB_PREC_MIXED tables for params and times -- closed-form evaluations
 *   (corner differences t with delta_t > 0, summed over the distinct
 *   closed-form blocks), Gauss nodes (over the distinct node lists, no
 *   padding) and blocks with any closed-form part; each output may be NULL.
 *   Equal differences (to 2^-44 times[n_steps]) share one evaluation. */
stb_status stb_assemble_nu_mixed_counts(const stb_params *params, const double *times,
                                        int64_t *closed_form_terms, int64_t *gauss_nodes,
                                        int64_t *closed_form_blocks);
stb_status stb_assemble_nu_workspace_size(const stb_mesh *mesh, const stb_params *params,
                                          const double *times, size_t *bytes);
stb_status stb_assemble_nu(const stb_mesh *mesh, const stb_params *params, const double *times,
                           double *V, double *K, void *workspace, size_t workspace_bytes,
                           stb_stream stream);
stb_status stb_matvec_nu(const double *A, int64_t E, int32_t n_steps, int32_t nrhs,
                         const double *x, double *y, stb_stream stream);
stb_status stb_solve_nu_workspace_size(int64_t E, int32_t n_steps, int32_t nrhs, size_t *bytes);
stb_status stb_solve_nu(const double *V, int64_t E, int32_t n_steps, int32_t nrhs,
                        const double *f, double *w, void *workspace, size_t workspace_bytes,
                        stb_stream stream);
stb_status stb_project_nu_workspace_size(const stb_mesh *mesh, const stb_params *params,
                                         int32_t nrhs, int32_t n_src, int32_t q_space,
                                         int32_t n_time, size_t *bytes);
stb_status stb_project_dirichlet_nu(const stb_mesh *mesh, const stb_params *params,
                                    const double *times, const double *sources, int32_t nrhs,
                                    int32_t n_src, int32_t q_space, int32_t n_time, double *g,
                                    void *workspace, size_t workspace_bytes, stb_stream stream);
stb_status stb_neumann_error_nu(const stb_mesh *mesh, const stb_params *params,
                                const double *times, const double *sources, int32_t nrhs,
                                int32_t n_src, const double *w, int32_t q_space, int32_t n_time,
                                double *out, void *workspace, size_t workspace_bytes,
                                stb_stream stream);
stb_status stb_dirichlet_rhs_nu_workspace_size(const stb_mesh *mesh, const stb_params *params,
                                               size_t *bytes);
stb_status stb_dirichlet_rhs_nu(const stb_mesh *mesh, const stb_params *params,
                                const double *times, const double *K, const double *g,
                                int32_t nrhs, double *f, void *workspace, size_t workspace_bytes,
                                stb_stream stream);

/* ---- block-Toeplitz matrix-vector product (eq. V_mat) ---------------------------
 *   y_r^k = beta y_r^k + sum_{d=0}^{k} A^d x_r^{k-d},  k = 0..n_steps-1,
 * A: device [n_steps][E][E] of `a_storage`; x, y: device FP64
 * [nrhs][n_steps][E], not overlapping.  FP64 arithmetic. */
stb_status stb_toeplitz_workspace_size(int64_t E, int32_t n_steps, int32_t nrhs, size_t *bytes);
stb_status stb_toeplitz_matvec(const void *A, int32_t a_storage, int64_t E, int32_t n_steps,
                               int32_t nrhs, const double *x, double beta, double *y,
                               void *workspace, size_t workspace_bytes, stb_stream stream);

/* ---- the same product in a chosen arithmetic (eq. V_mat) --------------------------
 * Same y, A, x, beta as stb_toeplitz_matvec; `arith` selects how it is formed:
 *   STB_ARITH_FP64  FP64 FMA, blocks of either storage (= stb_toeplitz_matvec);
 *   STB_ARITH_DF    STB_STORE_F32 blocks, exact FP32 products with a two-float
 *                   split of x summed in FP32 pairs (about 44 significant bits);
 *   STB_ARITH_TF32  STB_STORE_F32 blocks on the tensor cores: blocks read as
 *                   TF32 (10 stored mantissa bits), x rounded to TF32, FP32
 *                   accumulation over slices of blocks, slices added in FP64.
 *                   Needs E % 4 == 0 and A 16-byte aligned.  Error per entry
 *                   <= (2^-10 + 2^-11) sum_d |A^d| |x^{k-d}| plus the FP32
 *                   accumulation error.
 *   STB_ARITH_SPLIT STB_STORE_F32 blocks on the tensor cores with split
 *                   operands: per row and 64-column chunk j0..j0+63 of a block,
 *                   and per step vector and chunk of x, a power-of-two scale
 *                   above the chunk's largest magnitude and five bf16 slices of
 *                   9-bit digits (44 bits); the slice products of each level
 *                   are summed exactly in FP32 over a chunk, the chunks in
 *                   FP32 pairs, the slices of blocks in FP64.  Any E.  Error
 *                   per entry about 2^-44 sum_{d,chunks} 64 max|A^d_chunk|
 *                   max|x^{k-d}_chunk| (relative to the chunk maxima, not to
 *                   |A||x| entrywise).  Block entries below 2^126 in magnitude.
 * Workspace from stb_toeplitz_ex_workspace_size (same arith).  STB_ARITH_TF32
 * and STB_ARITH_SPLIT bound every device wait (2 s); an expired wait leaves
 * STB_ERR_TIMEOUT in the workspace status word (stb_workspace_status). */
#define STB_ARITH_FP64 0
#define STB_ARITH_DF 1
#define STB_ARITH_TF32 2
#define STB_ARITH_SPLIT 3
stb_status stb_toeplitz_ex_workspace_size(int64_t E, int32_t n_steps, int32_t nrhs, int32_t arith,
                                          size_t *bytes);
stb_status stb_toeplitz_matvec_ex(const void *A, int32_t a_storage, int64_t E, int32_t n_steps,
                                  int32_t nrhs, const double *x, double beta, double *y,
                                  int32_t arith, void *workspace, size_t workspace_bytes,
                                  stb_stream stream);

/* ---- self-test of the bounded device waits (no counterpart in the paper) ---------
 * The tensor-core kernels never wait without a limit: each mbarrier wait gives
 * up after a time limit, records STB_ERR_TIMEOUT in the status word and lets
 * the kernel wind down.  This call exercises that path without any fault: one
 * CTA copies the first 256 bytes of `probe` (device, 16-byte aligned) into
 * shared memory with a bulk copy, waits for it to land with the library's
 * bounded wait, then waits on a second mbarrier with a limit of `limit_ns`
 * nanoseconds (1000 .. 10^10).  With `arrive` == 0 nothing ever arrives on
 * that barrier, the wait expires and the status word of `workspace` (at least
 * 256 bytes) receives STB_ERR_TIMEOUT; with `arrive` != 0 the kernel arrives
 * first and the status stays STB_OK.  Asynchronous on `stream`; read the
 * result with stb_workspace_status. */
stb_status stb_selftest_bounded_wait(const void *probe, int64_t limit_ns, int32_t arrive,
                                     void *workspace, size_t workspace_bytes, stb_stream stream);

/* Self test of the grid barrier of the cooperative kernels (the march of a
 * panel, the blocked Cholesky): one cooperative launch of n_cta CTAs (at most
 * one per SM) in which every CTA but `skip` (-1: none) waits on one grid
 * barrier with a limit of limit_ns nanoseconds (1e3 .. 1e10).  With a CTA
 * skipping, the other CTAs' waits expire and the workspace status word
 * receives STB_ERR_TIMEOUT; with skip = -1 it stays STB_OK.  Workspace: at
 * least 512 + 4 n_cta bytes; bytes [512, 512 + 4 n_cta) receive one int32 per
 * CTA (1: passed, 0: gave up, 2: skipped).  Asynchronous on `stream`; read
 * the result with stb_workspace_status. */
stb_status stb_selftest_grid_barrier(int32_t n_cta, int32_t skip, int64_t limit_ns, void *workspace,
                                     size_t workspace_bytes, stb_stream stream);

/* ---- the same product without any allocation (no counterpart in the paper) -------
 * For callers that cannot allocate device memory at the point of the call:
 * code running while a CUDA stream is being captured into a graph (where
 * cudaMalloc is not permitted), plugins that live inside a host framework
 * owning all device memory, or real-time code that forbids allocation after
 * start-up.  Identical arguments and result as stb_toeplitz_matvec, but the
 * partial sums live in a scratch array inside this library, of fixed size
 * STB_TOEPLITZ_STATIC_SCRATCH_BYTES on every device that loads the library,
 * held until the process exits.  Problems needing more scratch
 * (8 * ceil(n_steps/8) * nrhs * n_steps * E bytes) are rejected with
 * STB_ERR_INVALID_ARG.  The call allocates nothing: the first call on a
 * device looks up the scratch's device address (make that first call before
 * any stream capture).  All calls on one device share its scratch, which
 * keeps the last call's contents: calls that overlap on the GPU (for example
 * on two streams of the same device) race and must be serialised by the
 * caller, e.g. by issuing them on one stream.  The looked-up address is kept
 * for the life of the process: after cudaDeviceReset (or any teardown of the
 * device's primary context) the library must not be called on that device
 * again in the same process. */
#define STB_TOEPLITZ_STATIC_SCRATCH_BYTES ((size_t)16 << 20)
stb_status stb_toeplitz_matvec_static(const void *A, int32_t a_storage, int64_t E, int32_t n_steps,
                                      int32_t nrhs, const double *x, double beta, double *y,
                                      stb_stream stream);

/* ---- right-hand side f = (1/2 M_h + K_h) g, M_h = h blockdiag(diag(Delta_l)) --
 * (Sec. 3.4).  K g in FP64 for STB_PREC_FP64; for STB_PREC_MIXED (FP32 blocks)
 * on the tensor cores with split operands (STB_ARITH_SPLIT).  An expired
 * bounded wait leaves STB_ERR_TIMEOUT in the workspace status word. */
stb_status stb_rhs_workspace_size(const stb_mesh *mesh, const stb_params *params, int32_t nrhs,
                                  size_t *bytes);
stb_status stb_dirichlet_rhs(const stb_mesh *mesh, const stb_params *params, const void *K,
                             const double *g, int32_t nrhs, double *f, void *workspace,
                             size_t workspace_bytes, stb_stream stream);

/* ---- forward-substitution solve of V_h w = f (eq. V_mat) --------------------------
 * Factorises V^0 = L L^T (blocked Cholesky of its lower triangle; V^0 is
 * symmetric positive definite), inverts L, then marches in time:
 *   w^k = (V^0)^{-1} (f^k - sum_{d=1}^{k} V^d w^{k-d}).
 * V: device [n_steps][E][E] (params->storage), f, w: device FP64
 * [nrhs][n_steps][E].  STB_PREC_FP64: every step in FP64.  STB_PREC_MIXED
 * (needs STB_STORE_F32 blocks): FP32 factorisation and march inside
 * iterative refinement w <- w + march(f - V_h w) with the residual products
 * V_h delta formed on the tensor cores with split operands (STB_ARITH_SPLIT,
 * about 2^-44 of the chunk magnitudes) and summed in FP64, until
 * ||f - V_h w|| <= 1e-10 ||f||
 * (at most 8 refinements, else STB_ERR_NOT_CONVERGED).  Synchronises `stream`
 * at the end and returns STB_ERR_NOT_SPD if a pivot was not positive. */
stb_status stb_solve_workspace_size(const stb_mesh *mesh, const stb_params *params, int32_t nrhs,
                                    size_t *bytes);
stb_status stb_dirichlet_solve(const stb_mesh *mesh, const stb_params *params, const void *V,
                               const double *f, int32_t nrhs, double *w, void *workspace,
                               size_t workspace_bytes, stb_stream stream);
/* Refinement count and final ||f - V_h w|| / ||f|| of the last solve that used
 * this workspace (0 and 0.0 after an FP64 solve).  Synchronises `stream`. */
stb_status stb_solve_report(const void *workspace, stb_stream stream, int32_t *refinements,
                            double *rel_residual);

/* ---- error of the Neumann datum (Sec. 6.1, relative L2(Sigma_h) error) -------------
 * out[0] = sum_r || w_r - w_{h,r} ||^2_{L2(Sigma_h)},  out[1] = sum_r || w_r ||^2
 * for the exact w_r = alpha du_r/dn of the sources (HOST array as above),
 * by the same product rule as the projection.  out: device FP64 [2]. */
stb_status stb_error_workspace_size(const stb_mesh *mesh, const stb_params *params, int32_t nrhs,
                                    int32_t n_src, int32_t q_space, int32_t n_time, size_t *bytes);
stb_status stb_neumann_error(const stb_mesh *mesh, const stb_params *params,
                             const double *sources, int32_t nrhs, int32_t n_src,
                             const double *w, int32_t q_space, int32_t n_time, double *out,
                             void *workspace, size_t workspace_bytes, stb_stream stream);

/* Device status word of a workspace (STB_OK or the first device-side error);
 * synchronises `stream`. */
stb_status stb_workspace_status(const void *workspace, stb_stream stream);

/* ---- pipe throughput probes (no counterpart in the paper) ---------------------
 * Measures, on the current device, the FP64 FMA, FP32 FMA and MUFU exp2 rates
 * (operations per second; one FMA counts as one operation) with eight
 * independent chains per thread on 4 CTAs of 256 threads per SM, about 10 ms
 * of work each; allocates and frees a small scratch buffer and synchronises
 * `stream`.  These are the denominators of the arithmetic rooflines. */
stb_status stb_measure_peaks(double *fp64_fma_per_s, double *fp32_fma_per_s, double *ex2_per_s,
                             stb_stream stream);

/* ---- kernel tracing (no counterpart in the paper; timing of the kernels) ------
 * While enabled, every kernel the library launches is bracketed by two CUDA
 * events recorded on its launch stream.  stb_trace_read synchronises those
 * events and returns, per kernel name, the number of launches and the summed
 * device time since the last reset.  Process-wide; not for concurrent use from
 * several threads while enabled. */
typedef struct stb_trace_entry {
    char name[48];
    int64_t launches;
    double total_ms;
} stb_trace_entry;
stb_status stb_trace_enable(int32_t on);
stb_status stb_trace_reset(void);
stb_status stb_trace_read(stb_trace_entry *out, int32_t max_entries, int32_t *n_entries);

#ifdef __cplusplus
}
#endif
#endif /* STBEM_H */
