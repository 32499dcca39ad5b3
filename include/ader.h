/*
 * ader.h -- C ABI of the GB300 (sm_103a) ADER-DG / ADER-WENO library for the
 * 1D Euler equations (gamma-law gas, M = 3 conserved variables rho, rho u, E).
 *
 * Method: Popov, "The effective use of BLAS interface for implementation of
 * finite-element ADER-DG and finite-volume ADER-WENO methods" (arXiv 2409.12483):
 *   - LST-DG predictor, Picard iteration of Sec. 1.1 eq. lst_dg_predictor_picard
 *     with the Kronecker-factored operators kappa~ (x) k~ (eq. m_and_kappa_matrices
 *     and the Kronecker forms below it), initialised by eq. ind_prop;
 *   - ADER-DG corrector, Sec. 1.2 eq. ader_dg_method_full reduced to 1D;
 *   - ADER-WENO finite-volume corrector, Sec. 1.3 eq. ader_weno_fv_method_full,
 *     fed by the WENO reconstruction of eq. weno_reconstr;
 *   - time step constraint of Sec. 1.5 with the subcell averages of Sec. 1.4.
 * The Riemann solver is Rusanov (local Lax-Friedrichs); the paper leaves it open.
 *
 * Conventions (every entry point):
 *   - returns an ader_status; nothing aborts or exits; ader_last_error() holds a
 *     message for the last failure on that context;
 *   - "device" pointers are CUDA device addresses owned by the caller (for
 *     example torch tensors); "host" pointers are ordinary host memory;
 *   - work is enqueued on the stream given to ader_bind() (NULL = legacy default
 *     stream) and is asynchronous unless the entry point says it synchronises;
 *   - a context is not thread-safe: use one context per host thread;
 *   - layouts are AoS, variable fastest (M = 3 for the Euler system, 5 for the
 *     reacting system, see ader_system):
 *       DG state      u[cell][k][r]        k < N+1 GL nodes, r < M
 *       FV state      v[cell][r]
 *       predictor     q[cell][p0][p1][r]   p0 = tau node, p1 = xi node
 *     cell i covers [x0 + i dx, x0 + (i+1) dx], dx = (x1 - x0) / n_cells, periodic.
 */
#ifndef ADER_GB300_H
#define ADER_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ADER_OK = 0,
  ADER_ERR_ARG = 1,            /* invalid argument, size or layout */
  ADER_ERR_NOMEM = 2,          /* workspace missing or too small */
  ADER_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  ADER_ERR_NOT_CONVERGED = 4,  /* some cell hit the Picard iteration cap (result still written) */
  ADER_ERR_NONPHYSICAL = 5,    /* rho <= 0 or p <= 0 (or non-finite) met by the CFL rule */
  ADER_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
  ADER_ERR_STATE = 7           /* call out of order (e.g. no workspace bound) */
} ader_status;

typedef enum { ADER_SCHEME_DG = 0, ADER_SCHEME_WENO_FV = 1 } ader_scheme;

typedef enum {
  ADER_PREC_FP64 = 0,            /* whole path in FP64 */
  ADER_PREC_FP32_PREDICTOR = 1,  /* Picard in FP32, then fp64_sweeps FP64 sweeps; rest FP64 */
  ADER_PREC_FF_PREDICTOR = 2,    /* Picard and predictor epilogue in float-float (~48 bits,
                                    FP32 pipes); corrector and CFL in FP64 */
  ADER_PREC_FP32_FF_SWEEPS = 3,  /* Picard in FP32 (to fp32_tol), then fp64_sweeps sweeps and
                                    the predictor epilogue in float-float (FP64-grade accuracy
                                    on the FP32 pipes); corrector and CFL in FP64 */
  ADER_PREC_FP32_INCREMENT = 4   /* increment form: with q = u + d, the tau-independent first
                                    iteration d1 = -(dt/dx) tau (x) k~ F(u) and the terms of u
                                    in float-float; the Picard iterations on d - d1 in FP32 with
                                    F(u + d) - F(u) as exact differences, so FP32 rounding is
                                    relative to the correction, not the state; stops at the FP64
                                    tolerance or the FP32 resolution of the correction.  Euler
                                    system only; corrector and CFL in FP64 */
} ader_precision;

/* The system of conservation laws.
 * ADER_SYSTEM_EULER: 1D Euler, M = 3 variables (rho, rho u, E).
 * ADER_SYSTEM_REACTING: the paper's two-component reacting flow in 1D (Sec. 2,
 *   eq. pdes_2_comps), M = 5 variables (rho, rho u, E, rho c1, rho c2), species
 *   advected with the flow and the source S = (0, 0, 0, rho c2, -omega^2 rho c1);
 *   predictor by the nested Picard iteration of eq.
 *   lst_dg_predictor_nested_picards, corrector with the source term of eq.
 *   ader_dg_method_full.  DG scheme and ADER_PREC_FP64 only.
 * ADER_SYSTEM_TRACER: a non-conservative product (eq. pde_src with B != 0): 1D
 *   Euler carrying a passive tracer in non-conservative form, M = 4 variables
 *   (rho, rho u, E, phi), B(U) dU/dx = (0, 0, 0, u dphi/dx); predictor by the
 *   nested Picard iteration with b = (dt/dx) B(q) D^xi q in the inner loop,
 *   corrector with the B volume term and a path-conservative Rusanov face (the
 *   minus-side cell takes G + Bt/2, the plus side G - Bt/2, Bt the integral of B
 *   along the straight segment, 3-point Gauss-Legendre).  DG, ADER_PREC_FP64,
 *   periodic only; it runs through ader_step / ader_solve (ader_predict and
 *   ader_correct return ADER_ERR_ARG). */
typedef enum { ADER_SYSTEM_EULER = 0, ADER_SYSTEM_REACTING = 1, ADER_SYSTEM_TRACER = 2 } ader_system;

/* Boundary condition of the mesh ends.  ADER_BC_OUTFLOW (DG only): free outflow;
 * the ghost side of a boundary face holds the boundary cell's mean state of the
 * step's initial data (a uniform state passes unchanged; the Rusanov
 * dissipation damps trace-mean differences at the boundary). */
typedef enum { ADER_BC_PERIODIC = 0, ADER_BC_OUTFLOW = 1 } ader_bc;

/* Uniform periodic mesh on [x0, x1]. */
typedef struct {
  int64_t n_cells;
  double x0, x1;
} ader_mesh;

typedef struct {
  double gamma;           /* adiabatic index (1.4) */
  double cfl;             /* Courant number of Sec. 1.5 (0.4) */
  double picard_tol;      /* eps_0: stop when max|q'-q| <= tol * max(1, max|q'|) (1e-13) */
  int picard_max_iter;    /* iteration cap in tolerance mode; 0 = 4(N+1)+8 */
  int picard_fixed_iter;  /* > 0: exactly this many iterations, no early exit */
  int precision;          /* ader_precision */
  int fp64_sweeps;        /* sweeps after the FP32 stage (>= 1): FP64 sweeps for
                             ADER_PREC_FP32_PREDICTOR, float-float sweeps for
                             ADER_PREC_FP32_FF_SWEEPS */
  double fp32_tol;        /* FP32 stage tolerance (relative, as picard_tol) (1e-6) */
  int profile;            /* 1: ader_solve records CUDA events around every kernel of every
                             step on the stream it launches them on (graph event nodes) and
                             waits for each graph, so per-kernel times land in ader_stats */
  int system;             /* ader_system (ADER_SYSTEM_EULER) */
  double omega;           /* reaction frequency of ADER_SYSTEM_REACTING (1.0) */
  int bc;                 /* ader_bc (ADER_BC_PERIODIC) */
  int limiter;            /* 1: a posteriori subcell limiter (DG, Euler, N >= 1; 0): the
                             candidate of eq. ader_dg_method_full is checked on its 2N+1 subcell
                             averages (Sec. 1.4) by the physical admissibility detector (rho > 0,
                             e > 0) and the relaxed discrete maximum principle of eq. nad_ineq
                             against the cell and its neighbours; troubled cells are recomputed
                             from the subcell averages of u^n by the finite-volume ADER-WENO2
                             scheme (degree-1 WENO, degree-1 LST-DG predictor, Rusanov flux) on
                             their subcells and reconstructed with R = (P^T P)^-1 P^T
                             (eq. r_operator), the faces next to them carrying the subcell flux
                             on both sides.  2: every cell is recomputed on its subcells. */
  double nad_delta0;      /* NAD: delta = max(nad_delta0, nad_eps (max - min)) (1e-4) */
  double nad_eps;         /* (1e-3) */
  int cfl_mode;           /* where lambda_max of the CFL rule (Sec. 1.5) is taken:
                             0 = over the 2N+1 subcell averages P u of Sec. 1.4 (the
                             finite-volume subcell representation; default);
                             1 = over the nodal values u_k (1D DG, Euler system, no
                             limiter; ADER_ERR_ARG elsewhere).  dt = CFL / (2N+1) dx /
                             lambda_max in both. */
} ader_options;

typedef struct {
  int64_t steps;          /* time steps taken by the last ader_solve* call */
  double t;               /* simulated time reached */
  int64_t cells;          /* cells that ran the predictor in the last call */
  int max_iters;          /* max Picard iterations over those cells (FP64 + FP32 stages) */
  double mean_iters;      /* mean Picard iterations per cell */
  int status;             /* sticky device status (ader_status) */
  int64_t profiled_steps; /* steps timed by the profile option (0 when it is off) */
  double weno_ms;         /* summed CUDA-event times of the WENO kernel over profiled steps */
  double predict_ms;      /* ... of the predictor kernel */
  double face_ms;         /* ... of the interface-flux + update kernel */
  int64_t kernel_launches;/* kernels the last call launched (including no-op steps after 'done') */
  int64_t troubled_cells; /* cells the limiter recomputed, summed over the steps of the last call */
} ader_stats;

typedef struct ader_ctx ader_ctx;

/* Defaults listed above.  opt: host pointer, written. */
ader_status ader_default_options(ader_options* opt);

/* Create a context for a mesh, a degree N and a scheme.
 *   degree: DG 0..7; WENO-FV 2 or 4 (WENO order N+1 feeding an LST-DG predictor of degree N).
 *   opt: NULL for defaults.  Builds the operator tables of Sec. 1.1 (GL nodes,
 *   kappa~, k~, D~, psi, psi~, P of Sec. 1.4, WENO tables) on the host; allocates
 *   no device memory.  *out owns host memory only; free with ader_destroy(). */
ader_status ader_init(const ader_mesh* mesh, int degree, int scheme, const ader_options* opt,
                      ader_ctx** out);
/* The 2D Euler equations on a periodic Cartesian mesh (Sec. 1.1 tensor-product
 * predictor with L^xi = kappa~ (x) k~ (x) I and L^eta = kappa~ (x) I (x) k~,
 * Sec. 1.2 corrector with x- and y-faces, Sec. 1.5 time step with d = 2):
 *   mesh: nx x ny cells on [x0, x1] x [y0, y1] (host pointer, read);
 *   state u[cell][k1][k2][r], cell = iy nx + ix, k1 the xi node, k2 the eta
 *   node, r = (rho, m_x, m_y, E), FP64, n_cells = nx ny (ader_state_count);
 *   degree 0..7; options: DG, Euler, FP64 predictor, periodic, no limiter
 *   (anything else: ADER_ERR_ARG).
 * The context works with ader_workspace_bytes, ader_bind, ader_step,
 * ader_solve, ader_solve_from, ader_solve_host, ader_compute_dt,
 * ader_get_stats, ader_get_table and ader_destroy; the 1D-only calls
 * (ader_predict, ader_correct, ader_node_coords, ader_step_noalloc,
 * ader_autotune, ader_get_troubled) return ADER_ERR_ARG. */
typedef struct {
  int64_t nx, ny;
  double x0, x1, y0, y1;
} ader_mesh2d;
ader_status ader_init_2d(const ader_mesh2d* mesh, int degree, const ader_options* opt,
                         ader_ctx** out);

/* The 3D Euler equations on a periodic Cartesian mesh (the same predictor with
 * L^zeta = kappa~ (x) I (x) I (x) k~ added, x-, y- and z-faces, d = 3):
 *   mesh: nx x ny x nz cells on [x0, x1] x [y0, y1] x [z0, z1];
 *   state u[cell][k1][k2][k3][r], cell = (iz ny + iy) nx + ix, r = (rho, m_x,
 *   m_y, m_z, E), FP64; degree 0..7 (N <= 4: one GPU thread per space-time
 *   node; N = 5, 6: one thread per spatial node holding its tau column; N = 7:
 *   a cluster of two CTAs per cell, each holding half of every tau column); the
 *   options and the entry points that accept the context are those of
 *   ader_init_2d. */
typedef struct {
  int64_t nx, ny, nz;
  double x0, x1, y0, y1, z0, z1;
} ader_mesh3d;
ader_status ader_init_3d(const ader_mesh3d* mesh, int degree, const ader_options* opt,
                         ader_ctx** out);

void ader_destroy(ader_ctx* ctx);
const char* ader_last_error(const ader_ctx* ctx);
const char* ader_status_string(int status);

/* Sizes (in doubles / bytes) the caller must provide. */
int64_t ader_state_count(const ader_ctx* ctx);      /* DG: n_cells (N+1) M; FV: n_cells 3 */
int64_t ader_predictor_count(const ader_ctx* ctx);  /* n_cells (N+1)^2 M */
size_t ader_workspace_bytes(const ader_ctx* ctx);   /* device scratch for ader_bind() */

/* Physical coordinates of the state's points: DG: the GL nodes x0 + dx (i + xi_k)
 * ([cell][k], count = n_cells (N+1)); FV: the cell centres (count = n_cells).
 * x_host: host array, written. */
ader_status ader_node_coords(const ader_ctx* ctx, double* x_host, int64_t count);

/* Operator tables (host copies, row-major), for inspection:
 * name: "xi","w","psi0","psi1" (N+1), "kt","kap","dphi","dtil" ((N+1)^2), "P" ((2N+1)(N+1)),
 * "R" ((N+1)(2N+1): (P^T P)^-1 P^T, the reconstruction of eq. r_operator),
 * "ksa","ksb" (H^2, H = (N+2)/2: k~ in even/odd form, used by the predictor for
 * N >= 4; with h = (N+1)/2, ksa[p][q] = (k~[p][q] + k~[p][N-q])/2 for p, q < h and
 * ksa[p][h] = k~[p][h] for odd N+1; ksb[p][q] = (k~[p][q] - k~[p][N-q])/2 for
 * p < H, q < h; other entries 0); WENO contexts only: "wamono" (3 (N+1)^2:
 * [S][j][k], the coefficient a_j of stencil S's polynomial in t = 2 xi - 1 from
 * its k-th cell average, S = central, left, right), "wvnod" ((N+1)^2: [q][j] =
 * t_q^j, nodal values from monomial coefficients).  count must equal the
 * table's size; a wrong count or an unknown name returns ADER_ERR_ARG. */
ader_status ader_get_table(const ader_ctx* ctx, const char* name, double* out_host, int64_t count);

/* Bind caller-owned device scratch (>= ader_workspace_bytes, 256-byte aligned)
 * and a CUDA stream (cudaStream_t, NULL = default stream).  The library never
 * allocates device memory; the workspace must outlive every call that uses it. */
ader_status ader_bind(ader_ctx* ctx, void* workspace_dev, size_t bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Hot path.  All state pointers are device pointers of ader_state_count()
 * doubles (q: ader_predictor_count()).  dt > 0 is used as given; dt <= 0 means
 * "CFL time step of Sec. 1.5 for the input state" (computed on the device).
 * ------------------------------------------------------------------------- */

/* CFL time step (Sec. 1.5): DG: CFL/(2N+1) dx / lambda_max over the 2N+1 subcell
 * averages of Sec. 1.4 in every cell; FV: CFL dx / lambda_max over the cell
 * averages; lambda = |u| + c.  Clipped to t_end - t when t_end > 0.  Synchronises
 * the stream and returns the value in *dt_host.  ADER_ERR_NONPHYSICAL when some
 * subcell state has rho <= 0 or p <= 0. */
ader_status ader_compute_dt(ader_ctx* ctx, const double* u_dev, double t, double t_end,
                            double* dt_host);

/* LST-DG predictor for every cell: q for the state u (DG) or for the WENO
 * reconstruction of v (FV).  Algorithm lst_dg_predictor with S = B = 0. */
ader_status ader_predict(ader_ctx* ctx, const double* u_dev, double dt, double* q_dev);

/* Corrector that consumes a predictor result q (DG: eq. ader_dg_method_full;
 * FV: eq. ader_weno_fv_method_full): u_new from u and q.  dt must be > 0. */
ader_status ader_correct(ader_ctx* ctx, const double* u_dev, const double* q_dev, double dt,
                         double* u_new_dev);

/* One time step (predictor fused with its trace/volume epilogue, then the fused
 * interface-flux and update kernel).  u_dev and u_new_dev must not alias. */
ader_status ader_step(ader_ctx* ctx, const double* u_dev, double* u_new_dev, double dt);

/* WENO reconstruction only (FV contexts): nodal values w[cell][k][r] of eq. weno_reconstr. */
ader_status ader_weno_reconstruct(ader_ctx* ctx, const double* v_dev, double* w_dev);

/* Time loop with a device-resident time step: repeat {CFL dt, predictor,
 * corrector} until t = t_end (t_end > 0; the last step is clipped) or until
 * max_steps steps (max_steps > 0).  The state is updated in place (u_dev);
 * steps run as CUDA graphs of a fixed number of steps, the host polls the
 * device 'done' flag once per graph.  Synchronises before returning. */
ader_status ader_solve(ader_ctx* ctx, double* u_dev, double t_end, int64_t max_steps,
                       int64_t* steps_out, double* t_out);

/* ader_solve starting from simulated time t0 (0 <= t0 < t_end when t_end > 0):
 * resumes a solve from a checkpoint (the caller's state u_dev and the t reached).
 * A solve split as ader_solve(max_steps = k) then ader_solve_from(t_k, t_end)
 * gives the same steps and state bit for bit as one ader_solve(t_end). */
ader_status ader_solve_from(ader_ctx* ctx, double* u_dev, double t0, double t_end,
                            int64_t max_steps, int64_t* steps_out, double* t_out);

/* ader_solve on a HOST state: copies u_host to the device (workspace), solves,
 * copies the result back to u_host.  Synchronises. */
ader_status ader_solve_host(ader_ctx* ctx, double* u_host, double t_end, int64_t max_steps,
                            int64_t* steps_out, double* t_out);

/* ---------------------------------------------------------------------------
 * Context-resident state: the mesh-level form of the paper's interface, which
 * hands the previous solution to get_cell_local_solution(u_prev) (the LST-DG
 * predictor of one cell, Sec. 1.1, algorithm lst_dg_predictor) and to
 * get_dg_solution(u_prev) / get_fv_solution(v_prev) (the corrector of Sec. 1.2 /
 * Sec. 1.3, algorithms ader_dg and ader_weno_fv).  The state lives in the bound
 * workspace (one more state-sized region, counted by ader_workspace_bytes); a
 * simulated time t travels with it.  These calls take no state pointers; the
 * pointer-taking calls above stay the zero-copy path and do not touch it.
 * ader_bind() of a new workspace forgets the resident state.
 * ------------------------------------------------------------------------- */

/* Copy a state (ader_state_count() doubles, layout of this header) into the
 * context and set its time to 0.  on_device = 1: u is a device pointer, copied
 * on the context's stream (asynchronous); 0: a host pointer (synchronises, so the
 * buffer may be reused on return).  count must equal ader_state_count(). */
ader_status ader_set_state(ader_ctx* ctx, const double* u, int64_t count, int on_device);
/* Copy the resident state out (same conventions; a host copy synchronises).
 * ADER_ERR_STATE before ader_set_state. */
ader_status ader_get_state(ader_ctx* ctx, double* u, int64_t count, int on_device);
/* Simulated time of the resident state (host pointer, written). */
ader_status ader_get_state_time(ader_ctx* ctx, double* t);
/* The LST-DG predictor q[cell][p0][p1][r] of the resident state (the
 * mesh-level get_cell_local_solution): q_dev is a caller-owned DEVICE buffer
 * of count = ader_predictor_count() doubles; dt > 0 as given, dt <= 0 the CFL
 * step of Sec. 1.5.  The resident state is not changed.  1D only. */
ader_status ader_get_predictor(ader_ctx* ctx, double dt, double* q_dev, int64_t count);
/* Advance the resident state by one time step (predictor, corrector; the
 * limiter when enabled): dt > 0 as given; dt <= 0 the CFL step of Sec. 1.5 for
 * the resident state (computed on the device and read back: synchronises).
 * *dt_out (may be NULL) receives the step used; the resident time advances by
 * it.  Otherwise asynchronous; the step's status bits land in ader_get_stats. */
ader_status ader_state_step(ader_ctx* ctx, double dt, double* dt_out);
/* ader_solve_from on the resident state, from its current time: CFL steps until
 * t_end (t_end > 0, clipped) or max_steps.  The resident time becomes the time
 * reached (also on ADER_ERR_NOT_CONVERGED / NONPHYSICAL / TIMEOUT).  Synchronises. */
ader_status ader_state_solve(ader_ctx* ctx, double t_end, int64_t max_steps, int64_t* steps_out,
                             double* t_out);

/* ---------------------------------------------------------------------------
 * Domain decomposition of one periodic 1D mesh over several contexts (one per
 * GPU or process).  A shard holds the contiguous cells [first_cell, first_cell +
 * n_local) of the global mesh plus halo_cells copies of its neighbours' cells on
 * each side, as one array of n_local + 2 halo_cells cells:
 *   [ left halo | local cells | right halo ],  local cells at cell offset halo_cells.
 * Halo width: DG 1 (the face neighbour's traces come from its own cell-local
 * predictor, recomputed here); WENO-FV N + 1 (the neighbour's reconstruction
 * reaches N cells further).  One time step of the global scheme is then:
 *   1. fill the halos: the first halo_cells local cells go to the left
 *      neighbour's right halo, the last ones to the right neighbour's left halo
 *      (periodic: shard 0's left neighbour is the last shard);
 *   2. dt = min over shards of ader_compute_dt(ctx, u, t, 0, &dt_shard) (an
 *      8-byte min-reduction), clipped on the host to t_end - t when t + dt >=
 *      t_end;
 *   3. ader_step(ctx, u, u_new, dt) on the whole array.
 * The local cells of u_new then equal the single-mesh step (same kernels on the
 * same inputs); the halo cells of u_new are stale until the next fill.  The
 * device-resident time loops (ader_solve*, ader_state_solve) return
 * ADER_ERR_ARG on a shard: their time step needs every shard's lambda_max.
 * Periodic global mesh, no limiter; n_local >= 1 (DG) or >= N (WENO-FV).
 * ------------------------------------------------------------------------- */
typedef struct {
  int64_t first_cell;       /* global index of the first local cell */
  int64_t n_local;          /* cells this shard advances */
  int64_t n_global;         /* cells of the global mesh */
  int64_t halo_cells;       /* halo cells on each side */
  int64_t values_per_cell;  /* doubles per cell in the state array */
} ader_shard;
ader_status ader_init_shard(const ader_mesh* global_mesh, int64_t first_cell, int64_t n_local,
                            int degree, int scheme, const ader_options* opt, ader_ctx** out);
/* Layout of a shard context (ADER_ERR_ARG for a context from ader_init). */
ader_status ader_shard_info(const ader_ctx* ctx, ader_shard* out);

/* Statistics of the last predictor/solve call (synchronises). */
ader_status ader_get_stats(ader_ctx* ctx, ader_stats* out);

/* Troubled-cell flags of the last limited step (Sec. 1.6: the cells whose
 * candidate failed PAD or NAD, or every cell in limiter mode 2), one int32 per
 * cell (1 troubled, 0 not), copied into the DEVICE buffer flags_dev of n_cells
 * entries (caller-owned) on the context's stream order.  ADER_ERR_ARG without
 * the limiter, for a null pointer or count != n_cells. */
ader_status ader_get_troubled(ader_ctx* ctx, int32_t* flags_dev, int64_t count);

/* ---------------------------------------------------------------------------
 * Autotuning of launch shapes (no counterpart in the paper).
 * ------------------------------------------------------------------------- */
typedef struct {
  int predict_cells_per_block;  /* predictor tile: 16, 32 or 64 cells x (N+1) threads */
  int face_cells_per_block;     /* interface/update tile: 32 or 64 cells per 256 threads */
  int graph_steps;              /* time steps per CUDA-graph replay in ader_solve (even, 2..64) */
  double predict_ms;            /* measured per launch for the chosen shape (autotune only) */
  double face_ms;
  double solve_ms_per_step;     /* measured ader_solve time per step with graph_steps */
} ader_tuning;

/* Time every valid predictor tile shape, interface tile shape and graph length on
 * the state u_dev (not modified; the solve trials run on a workspace copy) with
 * `reps` repetitions each (the tile shapes in three interleaved rounds, each
 * keeping its fastest), keep the fastest, and report them.  Valid predictor
 * shapes have (N+1) * cells a multiple of 32 and at most 512 threads (32 cells
 * at most for N > 5).  Synchronises. */
ader_status ader_autotune(ader_ctx* ctx, const double* u_dev, int reps, ader_tuning* out);
/* Current launch shapes (defaults: 32, 64, mesh-size rule for graph_steps). */
ader_status ader_get_tuning(const ader_ctx* ctx, ader_tuning* out);
/* Set launch shapes (e.g. from an earlier autotune); invalid shapes give ADER_ERR_ARG. */
ader_status ader_set_tuning(ader_ctx* ctx, const ader_tuning* in);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of independent ADER-DG solves (no counterpart in
 * the paper; its single-mesh step is what every solve runs).
 *
 * A server owns a caller-provided device pool, admits queued requests in arrival
 * order when a slot and enough pool memory are free (admission by device
 * memory), keeps every admitted solve's state resident, and advances all of them
 * together: each tick launches, per degree present, one batched predictor and
 * one batched interface/update kernel over a work list of (solve, tile) items;
 * every solve keeps its own device-resident time step, CFL rule and stop time.
 * Ticks run as CUDA graphs of `ticks_per_round` steps; between rounds the host
 * retires finished solves (copying their state back), admits new ones and
 * rebuilds the work lists.  Requests that arrive while others run join at the
 * next round: their work overlaps on the device with the running solves.
 * A solve's result is the same as running it alone (same kernels per cell).
 * ------------------------------------------------------------------------- */
typedef struct ader_server ader_server;

typedef struct {
  void* pool_dev;           /* caller-owned device memory, 256-byte aligned */
  size_t pool_bytes;
  int max_slots;            /* solves resident at once (>= 1) */
  int ticks_per_round;      /* time steps per graph replay (even, >= 2) */
  int precision;            /* ader_precision of every solve's predictor */
  int fp64_sweeps;          /* sweeps after the FP32 stage (precision 1: FP64, 3: float-float) */
  double gamma, cfl;        /* shared physics / CFL (1.4, 0.4) */
  double picard_tol;        /* 0 = 1e-13 */
  void* stream;             /* cudaStream_t the server works on (NULL = default) */
} ader_server_opts;

typedef struct {
  int degree;               /* DG degree 0..7 */
  int64_t n_cells;
  double x0, x1;
  double t_end;             /* > 0 */
  double arrival;           /* server-clock time before which it is not admitted */
  const double* u0_host;    /* initial DG state [cell][k][r]; copied by ader_server_submit */
} ader_request;

enum { ADER_REQ_QUEUED = 0, ADER_REQ_RUNNING = 1, ADER_REQ_DONE = 2, ADER_REQ_FAILED = 3 };

typedef struct {
  int state;                /* ADER_REQ_* */
  int status;               /* ader_status of the solve once done/failed */
  int64_t steps;
  double t;                 /* simulated time reached */
  double arrival, admitted, finished;  /* server-clock times (finished: result on the host) */
  int64_t n_cells;
  int degree;
} ader_result;

/* Defaults (pool and stream NULL). */
ader_status ader_server_default_options(ader_server_opts* opt);
ader_status ader_server_create(const ader_server_opts* opt, ader_server** out);
void ader_server_destroy(ader_server* srv);
const char* ader_server_last_error(const ader_server* srv);
/* Device bytes one request needs in the pool (state x2, traces, alignment). */
size_t ader_server_request_bytes(int degree, int64_t n_cells);
/* Queue a request (copies u0_host).  ADER_ERR_NOMEM if it could never fit the pool. */
ader_status ader_server_submit(ader_server* srv, const ader_request* req, uint64_t* id_out);
/* One round at server-clock time `now`: retire finished solves (their results
 * reach host memory), admit arrived requests while slots and pool memory allow,
 * then run ticks_per_round steps of every running solve and wait for them.
 * Reports the running and queued counts afterwards.  Synchronises. */
ader_status ader_server_progress(ader_server* srv, double now, int* running, int* queued);
/* State of a request; when done and u_host != NULL, copies its final state
 * (n_cells (N+1) 3 doubles) to u_host. */
ader_status ader_server_poll(ader_server* srv, uint64_t id, ader_result* out, double* u_host);
/* Forget a finished request (frees its host copy). */
ader_status ader_server_release(ader_server* srv, uint64_t id);
/* Totals since creation: cell-updates, ticks, rounds, kernel launches. */
ader_status ader_server_totals(const ader_server* srv, int64_t* cell_updates, int64_t* ticks,
                               int64_t* rounds, int64_t* launches);

/* ---------------------------------------------------------------------------
 * One time step that allocates nothing (no counterpart in the paper: it exists
 * for callers that cannot allocate device memory -- code running where
 * cudaMalloc is not allowed or not wanted, e.g. inside a host that owns every
 * device allocation itself, or a caller with no allocator at hand -- and so
 * cannot provide the workspace ader_bind() needs).
 *
 * Same result as ader_step(ctx, u, u_new, dt) with dt > 0 (same kernels), but
 * the predictor's trace/volume scratch, the WENO reconstruction (FV) and the
 * small control block live in one file-scope static device array of
 * ADER_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the library keeps
 * until the process exits.  The caller passes only the input state u_dev and
 * the output u_new_dev (device pointers, ader_state_count() doubles each, not
 * aliased), dt > 0, and a CUDA stream (NULL = legacy default stream).  ctx comes
 * from ader_init(); ader_bind() is not needed.
 *
 *   - needs 256 bytes plus n_cells * 9 (N+1) doubles (DG: traces and volume
 *     term; FV: traces and reconstruction); larger meshes return ADER_ERR_ARG
 *     with a message naming the limit (38835 cells at N = 5, 29126 at N = 7,
 *     46602 for WENO5);
 *   - calls no cudaMalloc, cudaFree, cudaMallocHost or any other allocating
 *     routine, and creates no stream or event;
 *   - the first call on a device sets that device up (looks up the array's
 *     device address with cudaGetSymbolAddress and raises the kernels' shared
 *     memory limit): make that first call before any stream capture;
 *   - every call shares the one array and leaves its contents behind; the
 *     control block is cleared on the stream at the start of each call, but
 *     calls whose work overlaps on the GPU (other streams, other threads) race
 *     on the array: serialise them;
 *   - synchronises the stream before returning: it reads back the step's status
 *     bits from the array and returns ADER_ERR_NOT_CONVERGED when some cell hit
 *     the Picard iteration cap, ADER_ERR_NONPHYSICAL when some subcell average
 *     of u_new has rho <= 0 or p <= 0 or is not finite (u_new is written in both
 *     cases); launch errors return ADER_ERR_CUDA. */
#define ADER_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
ader_status ader_step_noalloc(ader_ctx* ctx, const double* u_dev, double* u_new_dev, double dt,
                              void* stream);

#ifdef __cplusplus
}
#endif
#endif
