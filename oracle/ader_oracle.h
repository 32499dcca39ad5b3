/*
 * ader_oracle.h -- plain, slow, FP64 CPU oracle for the 1D ADER-DG and
 * ADER-WENO finite-volume schemes (Popov, arXiv 2409.12483), Euler equations.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the tests, the smoke check of the graft entry point and
 * the CPU-baseline leg of bench.py use it.  It shares no code with the CUDA
 * library; the two meet only through the seeded input generators.
 *
 * Notation follows the paper: n = N+1 Gauss-Legendre nodes xi_k on [0,1],
 * weights w_k, Lagrange basis phi_k, psi_k = phi_k(0), psi~_k = phi_k(1),
 * mass Lambda, stiffness Xi, Upsilon, kappa~ = Upsilon^-1 Lambda,
 * k~ = Lambda^-1 Xi, D~_kl = w_l Dphi_kl, subcell projection P.
 * Space-time coefficients are AoS: q[p0][p1][r] (tau node, xi node, variable).
 *
 * Parity pins: every function here is pinned by tests/test_oracle_*.py
 * against closed forms, invariants, textbook special cases and brute force.
 */
#ifndef ADER_ORACLE_H
#define ADER_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OB_MAXDEG 9
#define OB_MAXN 10            /* nodes = N+1 */
#define OB_MAXNS 19           /* subcells = 2N+1 */
#define OB_M 3                /* conserved variables of 1D Euler */

enum { OB_OK = 0, OB_ERR_ARG = 1, OB_ERR_NOT_CONVERGED = 4, OB_ERR_NONPHYSICAL = 5 };

typedef struct {
  int N, n, Ns;
  double xi[OB_MAXN];               /* GL nodes on [0,1], ascending (Sec. 1.1, eq. gl_rule) */
  double w[OB_MAXN];                /* GL weights, sum = 1 */
  double psi0[OB_MAXN];             /* phi_k(0) */
  double psi1[OB_MAXN];             /* phi_k(1) */
  double dphi[OB_MAXN][OB_MAXN];    /* dphi[k][l] = phi_k'(xi_l) */
  double lam[OB_MAXN][OB_MAXN];     /* Lambda_kl = int phi_k phi_l */
  double xi_m[OB_MAXN][OB_MAXN];    /* Xi_kl = int phi_k phi_l' */
  double ups[OB_MAXN][OB_MAXN];     /* Upsilon_kl = phi_k(1)phi_l(1) - Xi_lk */
  double kap[OB_MAXN][OB_MAXN];     /* kappa~ = Upsilon^-1 Lambda */
  double kt[OB_MAXN][OB_MAXN];      /* k~ = Lambda^-1 Xi */
  double dt_m[OB_MAXN][OB_MAXN];    /* D~_kl = w_l dphi_kl */
  double P[OB_MAXNS][OB_MAXN];      /* P_jk = Ns int_{j/Ns}^{(j+1)/Ns} phi_k */
} ob_basis;

typedef struct {
  double gamma;     /* adiabatic index */
  double cfl;       /* Courant number */
  double tol;       /* Picard tolerance eps_0 (relative to max(1, max|q|)) */
  int max_iter;     /* Picard iteration cap (tolerance mode) */
  int fixed_iter;   /* >0: exactly this many Picard iterations, no early exit */
  int cfl_mode;     /* DG time step: 0 = lambda over the 2N+1 subcell averages (Sec. 1.4,
                       1.5), 1 = over the nodal values themselves */
} ob_params;

/* WENO reconstruction tables for odd order N+1 (N even): three stencils. */
typedef struct {
  int N, n;
  int shift[3];                       /* first cell of each stencil, relative to i */
  double lin[3];                      /* linear weights lambda_S */
  double eps;                         /* epsilon in (sigma+eps)^r */
  int r;                              /* power r */
  double ainv[3][OB_MAXN][OB_MAXN];   /* c^S = ainv[S] v_S (nodal values in cell i) */
  double sig[OB_MAXN][OB_MAXN];       /* smoothness matrix Sigma (sigma = c^T Sigma c) */
  double dal[OB_MAXN][OB_MAXN][OB_MAXN]; /* dal[a-1][q][k] = a-th xi-derivative of phi_k at xi_q */
  double wq[OB_MAXN];                 /* GL weights used to integrate the squared derivatives */
} ob_weno;

typedef struct {
  int64_t cells;
  int max_iters, min_iters;
  double mean_iters;
  int status;
} ob_stats;

/* ---- basis and operators ---- */
int ob_basis_build(int N, ob_basis* b);
/* phi_k(x) for all k at one point x (reference coords, any real x) */
void ob_basis_eval(const ob_basis* b, double x, double* phi_out);

/* ---- pointwise physics ---- */
void ob_euler_flux(double gamma, const double* U, double* F);
double ob_wave_speed(double gamma, const double* U);
void ob_rusanov(double gamma, const double* a, const double* b, double* G);

/* ---- LST-DG predictor (Sec. 1.1, eq. lst_dg_predictor_picard) ---- */
int ob_predict_cell(const ob_basis* b, const ob_params* p, double lam,
                    const double* u, double* q, int* iters);
/* Literal nested-loop form of Algorithm lst_dg_predictor with s = b = 0. */
int ob_predict_cell_nested(const ob_basis* b, const ob_params* p, double lam,
                           const double* u, double* q, int* iters);

/* ---- CFL (Sec. 1.5) ---- */
double ob_dg_lambda_max(const ob_basis* b, double gamma, int64_t ncells, const double* u);
/* lambda = max over every cell and node of |u| + c at the nodal values u[cell][k][r] */
double ob_dg_lambda_max_nodal(const ob_basis* b, double gamma, int64_t ncells, const double* u);
double ob_fv_lambda_max(double gamma, int64_t ncells, const double* v);
double ob_dg_dt(const ob_basis* b, const ob_params* p, double dx, int64_t ncells, const double* u);
double ob_fv_dt(const ob_params* p, double dx, int64_t ncells, const double* v);

/* ---- ADER-DG corrector and step (Sec. 1.2, eq. ader_dg_method_full) ---- */
int ob_dg_correct(const ob_basis* b, const ob_params* p, int64_t ncells, double dx, double dt,
                  const double* u, const double* q, double* u_new);
int ob_dg_step(const ob_basis* b, const ob_params* p, int64_t ncells, double dx, double dt,
               const double* u, double* u_new, double* q_out, ob_stats* st);
/* u_new only at the listed cells (needs predictors of i-1, i, i+1). */
int ob_dg_step_cells(const ob_basis* b, const ob_params* p, int64_t ncells, double dx, double dt,
                     const double* u, const int64_t* cells, int64_t count, double* u_new_sel);

/* ---- WENO reconstruction and ADER-WENO FV step (Sec. 1.3, eq. weno_reconstr) ---- */
int ob_weno_build(int N, const ob_basis* b, ob_weno* wt);
/* sigma = sum_{a=1..N} int_0^1 (p^(a))^2 for p = sum_k c_k phi_k, evaluated as
 * sum_a sum_q w_q (sum_k dal[a-1][q][k] c_k)^2 (exact: degree 2N-2a <= 2N+1). */
double ob_weno_sigma(const ob_weno* wt, const double* c);
int ob_weno_reconstruct(const ob_weno* wt, int64_t ncells, const double* v, double* w);
int ob_weno_cell(const ob_weno* wt, int64_t ncells, const double* v, int64_t i, double* w_i,
                 double* omega /* [3][M] or NULL */);
int ob_fv_step(const ob_basis* b, const ob_weno* wt, const ob_params* p, int64_t ncells, double dx,
               double dt, const double* v, double* v_new, ob_stats* st);
int ob_fv_step_cells(const ob_basis* b, const ob_weno* wt, const ob_params* p, int64_t ncells,
                     double dx, double dt, const double* v, const int64_t* cells, int64_t count,
                     double* v_new_sel);

/* ---- time loop (steps of Sec. 1 in sequence; dt clipped to t_end) ----
 * scheme 0 = DG (u is [cell][k][r]), 1 = WENO-FV (u is [cell][r]).
 * Stops when t reaches t_end (t_end > 0) or after max_steps steps. */
int ob_solve(int scheme, const ob_basis* b, const ob_weno* wt, const ob_params* p, int64_t ncells,
             double dx, double* u, double t_end, int64_t max_steps, int64_t* steps_out,
             double* t_out);

/* ------------------------------------------------------------------------
 * Systems with algebraic source terms (ader_oracle_src.c).
 *
 * The 1D reduction of the paper's two-component reacting flow (Sec. 2,
 * eq. pdes_2_comps): U = (rho, m, E, rho c1, rho c2), Euler fluxes plus the
 * advected species, F = (m, m u + p, (E + p) u, rho c1 u, rho c2 u), and the
 * "reaction rates" S = (0, 0, 0, rho c2, -omega^2 rho c1).  The predictor is
 * the nested Picard iteration of eq. lst_dg_predictor_nested_picards (outer
 * loop: fluxes; inner loop: sources, L^sigma = kappa~ (x) I acting on the
 * rescaled source s = dt S); the corrector adds the space-time integral of s
 * (last term of eq. ader_dg_method_full).  DG only.
 * ---------------------------------------------------------------------- */
#define OB_MRS 5

typedef struct {
  double gamma;
  double omega;     /* reaction frequency of S */
  double cfl;
  double tol;       /* eps_0 for both loops (relative to max(1, max|q|)) */
  int max_iter;     /* cap of each loop */
  int fixed_iter;   /* >0: exactly this many outer iterations (inner loops still converge) */
} ob_rs_params;

void ob_rs_flux(double gamma, const double* U, double* F);
void ob_rs_source(double omega, const double* U, double* S);
void ob_rs_rusanov(double gamma, const double* a, const double* b, double* G);
/* nested Picard; iters: outer count, inner_total: inner iterations summed over
 * the outer ones (either may be NULL) */
int ob_rs_predict_cell(const ob_basis* b, const ob_rs_params* p, double lam, double dt,
                       const double* u, double* q, int* iters, int* inner_total);
/* one Picard loop updating flux and source together (test variant) */
int ob_rs_predict_cell_direct(const ob_basis* b, const ob_rs_params* p, double lam, double dt,
                              const double* u, double* q, int* iters);
double ob_rs_dg_dt(const ob_basis* b, const ob_rs_params* p, double dx, int64_t ncells,
                   const double* u);
int ob_rs_dg_step(const ob_basis* b, const ob_rs_params* p, int64_t ncells, double dx, double dt,
                  const double* u, double* u_new, double* q_out, ob_stats* st);
int ob_rs_dg_step_cells(const ob_basis* b, const ob_rs_params* p, int64_t ncells, double dx,
                        double dt, const double* u, const int64_t* cells, int64_t count,
                        double* u_new_sel);
/* time loop: dt_fixed > 0 gives uniform steps (clipped to t_end), else the CFL
 * rule of Sec. 1.5 over the Euler part of the state */
int ob_rs_solve(const ob_basis* b, const ob_rs_params* p, int64_t ncells, double dx, double* u,
                double t_end, int64_t max_steps, double dt_fixed, int64_t* steps_out,
                double* t_out);

/* ------------------------------------------------------------------------
 * Boundaries and the a posteriori subcell limiter (ader_oracle_lim.c), DG, Euler.
 *
 * bc: 0 periodic, 1 outflow (free outflow: the ghost side of a boundary face
 * holds the boundary cell's mean state of u^n; a first reading, with the
 * interior trace on both sides, made the high-order boundary cells unstable --
 * rounding noise of a uniform state grew without bound at N = 5).  For the
 * limiter's subcell fluxes the ghost subcells are the boundary subcell.
 * limiter 1 (N >= 1): the candidate u* of eq.
 * ader_dg_method_full is checked cell by cell on its 2N+1 subcell averages
 * P u* (Sec. 1.4, eq. p_operator) by the physical admissibility detector
 * (rho > 0, e > 0) and the relaxed discrete maximum principle of eq. nad_ineq
 * against the subcell averages P u^n of the cell and its neighbours
 * (delta = max(delta0, eps (max - min))); troubled cells are recomputed by the
 * finite-volume ADER-WENO2 scheme (WENO reconstruction of degree 1, LST-DG
 * predictor of degree 1, Rusanov flux) on their 2N+1 subcells, from the subcell
 * averages P u^n, and reconstructed with the pseudo-inverse R = (P^T P)^-1 P^T
 * (eq. r_operator); faces next to a troubled cell carry the subcell flux on
 * both sides (the DG neighbour's update is corrected with it), so the step
 * stays conservative.  If R v has an inadmissible subcell average, the cell
 * takes the mean of v.  limiter 2: every cell is troubled (the ADER-WENO2
 * scheme on the subgrid, with the projection P R after each step).
 * ---------------------------------------------------------------------- */
typedef struct {
  int bc;          /* 0 periodic, 1 outflow */
  int limiter;     /* 0 off, 1 on, 2 every cell recomputed on its subcells */
  double delta0;   /* NAD absolute tolerance (1e-4) */
  double eps;      /* NAD relative tolerance (1e-3) */
} ob_lim_params;

/* degree-1 WENO nodal values w[2][3] at the nodes xi[2] of a subcell with
 * averages v0 and neighbours vm (left), vp (right) */
void ob_lim_weno2(const double* vm, const double* v0, const double* vp, const double* xi,
                  double* w);
/* R = (P^T P)^-1 P^T, [n][Ns] row-major */
int ob_r_matrix(const ob_basis* b, double* R);
int ob_dgl_step(const ob_basis* b, const ob_params* p, const ob_lim_params* lp, int64_t ncells,
                double dx, double dt, const double* u, double* u_new, int* troubled,
                ob_stats* st);
int ob_dgl_solve(const ob_basis* b, const ob_params* p, const ob_lim_params* lp, int64_t ncells,
                 double dx, double* u, double t_end, int64_t max_steps, int64_t* steps_out,
                 double* t_out, int64_t* troubled_total);

/* ------------------------------------------------------------------------
 * 2D Euler on a periodic Cartesian mesh (ader_oracle_2d.c): state
 * u[cell][k1][k2][r], cell = iy nx + ix, r = (rho, m_x, m_y, E); predictor
 * q[p0][p1][p2][r]; the tensor-product predictor of Sec. 1.1 (L^xi = kappa~ (x)
 * k~ (x) I, L^eta = kappa~ (x) I (x) k~), the corrector of Sec. 1.2 with x- and
 * y-faces, dt = CFL / (2 (2N+1)) min(dx / lambda_x, dy / lambda_y) over the
 * Ns x Ns subcell averages (Sec. 1.5, d = 2).
 * ---------------------------------------------------------------------- */
#define OB2_M 4
void ob2_flux(double gamma, const double* U, double* F, double* G);
double ob2_speed(double gamma, const double* U, int dir);
void ob2_rusanov(double gamma, int dir, const double* a, const double* b, double* H);
int ob2_predict_cell(const ob_basis* b, const ob_params* p, double lx, double ly, const double* u,
                     double* q, int* iters);
int ob2_dg_step(const ob_basis* b, const ob_params* p, int64_t nx, int64_t ny, double dx,
                double dy, double dt, const double* u, double* u_new, ob_stats* st);
int ob2_dg_step_cells(const ob_basis* b, const ob_params* p, int64_t nx, int64_t ny, double dx,
                      double dy, double dt, const double* u, const int64_t* cells, int64_t count,
                      double* out);
double ob2_dt(const ob_basis* b, const ob_params* p, int64_t nx, int64_t ny, double dx, double dy,
              const double* u);
int ob2_solve(const ob_basis* b, const ob_params* p, int64_t nx, int64_t ny, double dx, double dy,
              double* u, double t_end, int64_t max_steps, int64_t* steps_out, double* t_out);

/* ------------------------------------------------------------------------
 * 3D Euler on a periodic Cartesian mesh (ader_oracle_3d.c): state
 * u[cell][k1][k2][k3][r], cell = (iz ny + iy) nx + ix, r = (rho, m_x, m_y,
 * m_z, E); predictor q[p0][p1][p2][p3][r]; L^xi = kappa~ (x) k~ (x) I (x) I and
 * likewise along eta and zeta; faces in x, y and z; dt = CFL / (3 (2N+1))
 * min_d (h_d / lambda_d) over the Ns^3 subcell averages.
 * ---------------------------------------------------------------------- */
#define OB3_M 5
void ob3_flux(double gamma, const double* U, double* F);  /* F[3][5]: x-, y-, z-fluxes */
double ob3_speed(double gamma, const double* U, int dir);
void ob3_rusanov(double gamma, int dir, const double* a, const double* b, double* H);
int ob3_predict_cell(const ob_basis* b, const ob_params* p, double lx, double ly, double lz,
                     const double* u, double* q, int* iters);
int ob3_dg_step(const ob_basis* b, const ob_params* p, int64_t nx, int64_t ny, int64_t nz,
                double dx, double dy, double dz, double dt, const double* u, double* u_new,
                ob_stats* st);
int ob3_dg_step_cells(const ob_basis* b, const ob_params* p, int64_t nx, int64_t ny, int64_t nz,
                      double dx, double dy, double dz, double dt, const double* u,
                      const int64_t* cells, int64_t count, double* out);
double ob3_dt(const ob_basis* b, const ob_params* p, int64_t nx, int64_t ny, int64_t nz, double dx,
              double dy, double dz, const double* u);
int ob3_solve(const ob_basis* b, const ob_params* p, int64_t nx, int64_t ny, int64_t nz, double dx,
              double dy, double dz, double* u, double t_end, int64_t max_steps, int64_t* steps_out,
              double* t_out);

/* ------------------------------------------------------------------------
 * Non-conservative product (ader_oracle_nc.c): 1D Euler with a passive tracer
 * phi in non-conservative form, U = (rho, m, E, phi), B(U) dU/dx = (0, 0, 0,
 * u dphi/dx); nested Picard predictor with the b term in the inner loop, the B
 * volume term and a path-conservative Rusanov face (G +- Bt/2, 3-point GL path
 * integral along the straight segment).  State u[cell][k][4].
 * ---------------------------------------------------------------------- */
#define OB_NC_M 4
void ob_nc_flux(double gamma, const double* U, double* F);
void ob_nc_face(double gamma, const double* a, const double* b, double* G, double* Bt);
int ob_nc_predict_cell(const ob_basis* b, const ob_params* p, double lam, const double* u,
                       double* q, int* iters);
int ob_nc_step(const ob_basis* b, const ob_params* p, int64_t ncells, double dx, double dt,
               const double* u, double* u_new, ob_stats* st);
int ob_nc_solve(const ob_basis* b, const ob_params* p, int64_t ncells, double dx, double* u,
                double t_end, int64_t max_steps, int64_t* steps_out, double* t_out);

#ifdef __cplusplus
}
#endif
#endif
