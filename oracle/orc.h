/*
 * orc.h -- FP64 CPU oracle for the space-time Galerkin BEM of the 3D heat
 * equation (Zapletal, Watschinger, Of, Merta, "Semi-analytic integration for
 * a parallel space-time boundary element method modeling the heat equation").
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that
 * the GPU path is checked against.  Only tests/, __graft_entry__.smoke() and
 * the cpu_baseline / reference legs of bench.py may load it.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * Conventions (all arrays row-major, host memory, caller-owned):
 *   nodes  [n_nodes][3]  double   vertex coordinates
 *   tris   [E][3]        int32    vertex indices, counter-clockwise seen from
 *                                 outside (outward normal by the right hand)
 *   r = x - y with x on the test triangle (row l), y on the trial triangle
 *   (column j); n = n_y is the trial triangle's outward unit normal (Sec. 2).
 *   Time grid t_i = i*h, h = T/E_t (Sec. 3); time level i_t = delta/h.
 *   Block d of a lower-triangular block-Toeplitz matrix: A^d[l][j]
 *   (eq. V_mat, eq. K_mat).
 *
 * Return codes: 0 ok, -1 invalid argument, -5 not SPD.
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- pair classes (Sec. 3.1, "Computation of the Galerkin weights") ---- */
enum { ORC_DISJOINT = 0, ORC_VERTEX = 1, ORC_EDGE = 2, ORC_IDENTICAL = 3 };

/* ---- heat kernel and its temporal antiderivatives (Sec. 2, Sec. 3, Sec. 4) */
double orc_heat_kernel(double rho, double delta, double alpha);
double orc_dn_heat_kernel(double rn, double rho, double delta, double alpha);
double orc_G_dtau(double rho, double delta, double alpha);
double orc_G_dtau_dt(double rho, double delta, double alpha);
double orc_dn_G_dtau_dt(double rn, double rho, double delta, double alpha);
double orc_dn_G_dtau(double rn, double rho, double delta, double alpha);
double orc_V_d(double rho, int d, double h, double alpha);
double orc_K_d(double rn, double rho, int d, double h, double alpha);
/* small-argument series of the bracket of eq. dG (reading of the stable
 * evaluation, x = rho / (2 sqrt(alpha delta)) below ORC_SERIES_X) */
double orc_psi_series(double x);
double orc_psi_direct(double x);
#define ORC_SERIES_X 0.5

/* ---- quadrature rules ---------------------------------------------------- */
int orc_gauss_legendre01(int n, double *x, double *w);
int orc_gauss_jacobi01(int n, double *x, double *w);           /* weight x on [0,1] */
int orc_triangle_rule(int q, double *s1, double *s2, double *w);
int orc_ss_rule_size(int cls, int m);
int orc_ss_rule(int cls, int m, double *s1, double *s2, double *t1, double *t2,
                double *w);

/* ---- mesh geometry and pair classification -------------------------------- */
int orc_triangle_geometry(const double *nodes, int64_t n_nodes,
                          const int32_t *tris, int64_t E, double *area,
                          double *normal);
int orc_pair_class(const int32_t *tl, const int32_t *tj, int32_t *ol,
                   int32_t *oj);

/* ---- assembly ---------------------------------------------------------------
 * Spatial sums of one pair, scaled by 4*Delta_l*Delta_j:
 *   SV[i] = sum_q w_q G^{dtau dt}(r_q, i h)          i = 0..n_levels-1
 *   SK[i] = sum_q w_q alpha dG^{dtau dt}/dn_y(r_q, i h)
 *   SV[n_levels] = sum_q w_q G^{dtau}(r_q, 0)
 *   SK[n_levels] = sum_q w_q alpha dG^{dtau}/dn_y(r_q, 0)                     */
int orc_pair_sums(const double *nodes, int64_t n_nodes, const int32_t *tris,
                  int64_t E, int64_t l, int64_t j, double alpha, double h,
                  int n_levels, int q_reg, int m_ss, double *SV, double *SK);

/* Rows `rows[0..n_rows)` of all blocks V^d, K^d, d = 0..n_steps-1.
 * V, K: [n_rows][n_steps][E].  SV, SK (may be NULL): [n_rows][n_steps+2][E]
 * with level i_t = 0..n_steps in slots 0..n_steps and the delta = 0 singular
 * sum in slot n_steps+1.                                                       */
int orc_assemble_rows(const double *nodes, int64_t n_nodes,
                      const int32_t *tris, int64_t E, double alpha, double T,
                      int32_t n_steps, int32_t q_reg, int32_t m_ss,
                      const int64_t *rows, int64_t n_rows, double *V,
                      double *K, double *SV, double *SK);

/* ---- Dirichlet data, right-hand side, solve, error --------------------------
 * sources [nrhs][n_src][5] = (y1, y2, y3, t0, weight); the Dirichlet datum of
 * right-hand side r is g_r(x,t) = sum_s weight_s G_alpha(x - y_s, t - t0_s).
 * Vectors are laid out [nrhs][n_steps][E].                                    */
int orc_project_dirichlet(const double *nodes, int64_t n_nodes,
                          const int32_t *tris, int64_t E, double alpha,
                          double T, int32_t n_steps, const double *sources,
                          int32_t n_src, int32_t nrhs, int32_t q_space,
                          int32_t n_time, double *g);
int orc_project_neumann(const double *nodes, int64_t n_nodes,
                        const int32_t *tris, int64_t E, double alpha, double T,
                        int32_t n_steps, const double *sources, int32_t n_src,
                        int32_t nrhs, int32_t q_space, int32_t n_time,
                        double *wproj);
int orc_toeplitz_matvec(const double *A, int64_t E, int32_t n_steps,
                        int32_t nrhs, const double *x, double *y);
int orc_dirichlet_rhs(const double *area, const double *K, int64_t E,
                      double T, int32_t n_steps, int32_t nrhs,
                      const double *g, double *f);
int orc_dirichlet_solve(const double *V, int64_t E, int32_t n_steps,
                        int32_t nrhs, const double *f, double *w);
int orc_neumann_error(const double *nodes, int64_t n_nodes,
                      const int32_t *tris, int64_t E, double alpha, double T,
                      int32_t n_steps, const double *sources, int32_t n_src,
                      int32_t nrhs, const double *w, int32_t q_space,
                      int32_t n_time, double *err2, double *ref2);

/* ---- piecewise-linear trial space in space (Sec. 3.2, Sec. 3.4) -----------
 * K1 [n_rows][n_steps][n_nodes]: rows of the blocks of K_h with the trial
 * functions phi_i (nodal hat functions); g1 [nrhs][n_steps][n_nodes]: the
 * L2(Sigma_h) projection of the Dirichlet datum into X_h^{1,0}; the
 * right-hand side (1/2 M_h + K_h) g1 with the p0 x p1 mass matrix.           */
int orc_assemble_k1_rows(const double *nodes, int64_t n_nodes,
                         const int32_t *tris, int64_t E, double alpha, double T,
                         int32_t n_steps, int32_t q_reg, int32_t m_ss,
                         const int64_t *rows, int64_t n_rows, double *K1);
int orc_project_dirichlet_p1(const double *nodes, int64_t n_nodes,
                             const int32_t *tris, int64_t E, double alpha,
                             double T, int32_t n_steps, const double *sources,
                             int32_t n_src, int32_t nrhs, int32_t q_space,
                             int32_t n_time, double *g1);
int orc_toeplitz_matvec_rect(const double *A, int64_t E, int64_t N, int32_t n_steps,
                             int32_t nrhs, const double *x, double *y);
int orc_dirichlet_rhs_p1(const double *area, const int32_t *tris, const double *K1,
                         int64_t E, int64_t N, double T, int32_t n_steps, int32_t nrhs,
                         const double *g1, double *f);

/* ---- hypersingular operator and the Neumann problem (Sec. 3.3, Sec. 3.4) ----
 * D_h = D_h^1 + D_h^2, blocks [n_steps][N][N]: D2 from the test triangles
 * test_tris (added into D2), D1 = T^T (alpha^2 V^d (x) I_3) T from the
 * single-layer blocks V [n_steps][E][E] (overwritten), the surface curls of
 * the hat functions curl [E][3 vertices][3]; the Neumann right-hand side
 * (1/2 M_h^{T_x} - K_h^{T_x}) h (h [nrhs][n_steps][E] -> f [nrhs][n_steps][N])
 * and the L2(Sigma_h) error of piecewise-linear Dirichlet data.            */
int orc_assemble_d2_tris(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t E,
                         double alpha, double T, int32_t n_steps, int32_t q_reg, int32_t m_ss,
                         const int64_t *test_tris, int64_t n_test, double *D2);
int orc_surface_curls(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t E,
                      double *curl);
int orc_assemble_d1(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t E,
                    double alpha, int32_t n_steps, const double *V, double *D1);
int orc_neumann_rhs(const double *area, const int32_t *tris, const double *K1, int64_t E,
                    int64_t N, double T, int32_t n_steps, int32_t nrhs, const double *hd,
                    double *f);
int orc_dirichlet_error_p1(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t E,
                           double alpha, double T, int32_t n_steps, const double *sources,
                           int32_t n_src, int32_t nrhs, const double *u1, int32_t q_space,
                           int32_t n_time, double *err2, double *ref2);

/* ---- non-uniform time grids (Sec. 7) ----------------------------------------
 * times [n_steps + 1] strictly increasing from 0; blocks A^{k,i}, k >= i,
 * packed at b(k,i) = k(k+1)/2 + i: V, K rows [n_rows][n_blocks][E]; matrices
 * [n_blocks][E][E] for the product and the solve.                          */
int orc_assemble_rows_nu(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t E,
                         double alpha, const double *times, int32_t n_steps, int32_t q_reg,
                         int32_t m_ss, const int64_t *rows, int64_t n_rows, double *V, double *K);
int orc_matvec_nu(const double *A, int64_t E, int32_t n_steps, int32_t nrhs, const double *x,
                  double *y);
int orc_solve_nu(const double *V, int64_t E, int32_t n_steps, int32_t nrhs, const double *f,
                 double *w);
int orc_project_dirichlet_nu(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t E,
                             double alpha, const double *times, int32_t n_steps,
                             const double *sources, int32_t n_src, int32_t nrhs, int32_t q_space,
                             int32_t n_time, double *g);
int orc_dirichlet_rhs_nu(const double *area, const double *K, int64_t E, const double *times,
                         int32_t n_steps, int32_t nrhs, const double *g, double *f);
int orc_neumann_error_nu(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t E,
                         double alpha, const double *times, int32_t n_steps,
                         const double *sources, int32_t n_src, int32_t nrhs, const double *w,
                         int32_t q_space, int32_t n_time, double *err2, double *ref2);

/* ---- potentials: the discretised representation formula (Sec. 3.5) --------
 * At points (x, t) off Gamma_h, points [n_pts][4] = (x1, x2, x3, t),
 * 0 <= t <= T: slp [nrhs][n_pts] = V~ w_h (w [nrhs][n_steps][E], piecewise
 * constant), dlp [nrhs][n_pts] = W u_h (u1 [nrhs][n_steps][n_nodes],
 * piecewise linear in space); either output may be NULL.  The q x q conical
 * rule on every triangle, exact temporal antiderivatives.                   */
int orc_potentials(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t E,
                   double alpha, double T, int32_t n_steps, const double *w, const double *u1,
                   int32_t nrhs, const double *points, int64_t n_pts, int32_t q,
                   double *slp, double *dlp);

#ifdef __cplusplus
}
#endif
#endif
