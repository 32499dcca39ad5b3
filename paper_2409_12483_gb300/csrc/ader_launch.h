// ader_launch.h -- launch parameter blocks and per-degree launchers of the
// sm_103a kernels (one translation unit per degree N, see ader_deg.cu).
#pragma once

#include <cuda_runtime.h>

#include "ader_device.cuh"
#include "ader_ops.h"

namespace ader {

enum : int { kOutQ = 0, kOutTrace = 1 };
enum : int { kSysEuler = 0, kSysReacting = 1, kSysTracer = 2 };
enum : int { kBcPeriodic = 0, kBcOutflow = 1 };

// LST-DG predictor (Algorithm lst_dg_predictor, S = B = 0) with its epilogue.
struct PredictParams {
  const double* u;       // nodal initial data [cell][n][3]: DG u^n, FV WENO reconstruction
  double* q_out;         // kOutQ: q[cell][p0][p1][3]
  const double* q_in;    // from_q: q is given, only the epilogue runs
  double* trace;         // kOutTrace: DG [cell][qR(3n) | qL(3n) | u + volume(3n)], FV [cell][qR | qL]
  long long ncells;
  int out_mode;
  int from_q;
  int dg;
  int prec;              // 0 FP64, 1 FP32 Picard + `sweeps` FP64 sweeps
  int sweeps;
  int max_iter;
  int fixed_iter;
  int cpb;               // predictor cells per block (16, 32, 64; tuned), 0 = 32
  int sys;               // kSysEuler, kSysReacting (ader_source.cuh), kSysTracer (ader_tracer.cuh)
  float tol32;
  double tol;
  double gamma, gm1;
  // FP32 constants of the increment form: gamma, gamma - 1, (3 - gamma)/2,
  // (gamma - 1)/2, tol (rounded once on the host)
  float gamf, gm1f, c1f, c2f, tolf;
  double om2;            // omega^2 of the reacting system's source
  StepParams sp;
  OpsD ops;
  OpsF opf;
};

// Interface flux (Rusanov at every tau node, GL-weighted in time) fused with the
// DG / FV update and, optionally, the lambda_max reduction for the next step.
struct FaceParams {
  const double* trace;
  const double* v_old;   // FV: previous cell averages; DG: u^n (outflow ghost states)
  double* u_new;
  long long ncells;
  int dg;
  int want_lambda;
  int cpf;               // interface/update cells per block (32, 64; tuned), 0 = 64
  int sys;               // kSysEuler or kSysReacting
  int bc;                // kBcPeriodic or kBcOutflow
  int Ns;
  int nodal;             // DG: lambda_max over the nodal values (cfl_mode 1), not the subcells
  double gamma, gm1;
  StepParams sp;
  OpsD ops;
};

// lambda_max over subcell (DG) or cell (FV) averages into ctl->lam[slot].
struct CflParams {
  const double* u;
  long long ncells;
  int vars;              // values per node record (3 Euler, 5 reacting); Euler variables first
  int dg;
  int slot;
  int Ns;
  int nodal;             // DG: over the nodal values (cfl_mode 1), not the subcells
  double gamma, gm1;
  DevCtl* ctl;
  OpsD ops;
};

// Continuous batching: a work list of tiles over many independent solves of the
// same degree; each solve has its own state buffers, trace buffer and control block.
struct SlotDesc {
  const double* u[2];   // ping-pong state: step with parity p reads u[p], writes u[p ^ 1]
  double* trace;
  long long ncells;
  int par0;             // parity offset: the solve's first step ran at tick parity par0
  int degree;
  StepParams sp;        // mode kDtSolve, t_end, max_steps, cfl_factor, inv_dx, ctl
};

struct TileItem {
  int slot;
  int tile;  // predictor or face tile index within the solve (tile sizes below)
};

// Tile sizes of the batched (server) kernels: 16-cell predictor tiles (32 for
// N = 0, whose 16-cell tile would be half a warp) and 32-cell face tiles, so a
// lone large solve spreads over twice as many SMs as with the single-solve
// kernels' default tiles.
constexpr int server_pred_cells(int N) { return N == 0 ? 32 : 16; }
constexpr int kServerFaceCells = 32;

struct MultiArgs {
  const SlotDesc* slots;
  const TileItem* items;
  long long nitems;
  int tick_par;
};

struct WenoParams {
  const double* v;
  double* w;
  long long ncells;
  WenoOps wo;
};

// A posteriori subcell limiter of the DG scheme (ader_limiter.cuh).
// Degree-1 operators of the limiter's subcell ADER-WENO2 scheme (GL nodes and
// weights, phi_k(0), phi_k(1), k~ = Lambda^-1 Xi, kappa~ = Upsilon^-1 Lambda).
struct Sub1Ops {
  double xi[2], w[2], psi0[2], psi1[2];
  double kt[2][2], kap[2][2];
};

struct LimParams {
  const double* u_old;   // u^n, [cell][n][3]
  double* u;             // in: candidate u*, out: u^{n+1} (same layout)
  const double* trace;   // predictor traces [cell][qR(3n) | qL(3n) | u + volume(3n)]
  float* mmf;            // [cell][9]: FP32 min (3), max (3) of the subcell averages of
                         // u^n and a bound (3) on their distance from the FP64 ones
  int* troubled;         // [cell]
  long long* list;       // [cell]: the troubled cells of the step (first ctl->lim_n entries)
  double* gface;         // [cell][2][3]: subcell fluxes of a troubled cell's left / right face
  long long ncells;
  int bc;                // kBcPeriodic or kBcOutflow
  int Ns;
  int mode;              // 1: detect troubled cells, 2: every cell troubled
  int want_lambda;       // lambda_max of the limited state into ctl->lam[par ^ 1]
  int max_iter, fixed_iter;  // Picard of the subcell predictor (as the DG predictor's)
  double tol;
  double gamma, gm1;
  double delta0, eps;    // NAD tolerances
  StepParams sp;
  OpsD ops;
  Sub1Ops s1;
  double R[kMaxN][kMaxNs];  // reconstruction from subcell averages
  float Pf[kMaxNs][kMaxN];  // P in FP32 (the screening passes)
  float pabs;               // max_j sum_k |P_jk|
};

// 2D Euler (ader_kernels2d.cuh): state [cell][k1][k2][4], cell = iy nx + ix.
struct Predict2DParams {
  const double* u;
  double* trace;         // [cell][xR | xL | yR | yL | volume], each [n][n][4]
  long long ncells;
  int max_iter, fixed_iter;
  double tol;
  double gamma, gm1;
  double inv_dy;         // 1 / dy (1 / dx travels in sp)
  StepParams sp;
  OpsD ops;
};

struct Face2DParams {
  const double* trace;
  double* gface;         // [cell][dir][k][4]: fluxes of the left x-face and bottom y-face
  double* u_new;
  long long ncells, nx, ny;
  int want_lambda;       // the update also reduces lambda_max of u_new into ctl->lam[par ^ 1]
  double gamma, gm1;
  double inv_dy;
  StepParams sp;
  OpsD ops;
  float Pf[kMaxNs][kMaxN];  // P in FP32 (the screening pass of lambda_max)
};

struct Cfl2DParams {
  const double* u;
  long long ncells;
  double gamma, gm1;
  double inv_dx, inv_dy;
  DevCtl* ctl;
  int slot;
  double P[kMaxNs][kMaxN];
  float Pf[kMaxNs][kMaxN];
};

// 3D Euler (ader_kernels3d.cuh): state [cell][k1][k2][k3][5], cell = (iz ny + iy) nx + ix.
struct Predict3DParams {
  const double* u;
  double* trace;         // [cell][d][side][l0][a][c][5] (six faces), then the volume term
  long long ncells;
  int max_iter, fixed_iter;
  double tol;
  double gamma, gm1;
  double inv_dy, inv_dz;  // 1 / dx travels in sp
  StepParams sp;
  OpsD ops;
};

struct Face3DParams {
  const double* trace;
  double* gface;         // [cell][d][a][c][5]: fluxes of the low face per direction
  double* u_new;
  const double* u_cfl;   // non-null: lambda_max of this state only (no update) into lam[cfl_slot]
  int cfl_slot;
  long long ncells, nx, ny, nz;
  int want_lambda;       // the update also reduces lambda_max of u_new into ctl->lam[par ^ 1]
  double gamma, gm1;
  double inv_dy, inv_dz;
  StepParams sp;
  OpsD ops;
  float Pf[kMaxNs][kMaxN];  // P in FP32 (the screening pass of lambda_max)
};

struct Cfl3DParams {
  const double* u;
  long long ncells;
  double gamma, gm1;
  double inv_dx, inv_dy, inv_dz;
  DevCtl* ctl;
  int slot;
  double P[kMaxNs][kMaxN];
  float Pf[kMaxNs][kMaxN];
};

// Per-degree entry points (defined in ader_deg.cu compiled once per degree).
#define ADER_DECLARE_DEGREE(D)                                                         \
  cudaError_t launch_predict_##D(const PredictParams& p, cudaStream_t s);              \
  cudaError_t launch_face_update_##D(const FaceParams& p, cudaStream_t s);             \
  cudaError_t launch_cfl_##D(const CflParams& p, cudaStream_t s);                      \
  cudaError_t launch_weno_##D(const WenoParams& p, cudaStream_t s);                    \
  cudaError_t launch_predict_multi_##D(const PredictParams& p, const MultiArgs& m, int grid,  \
                                       cudaStream_t s);                                 \
  cudaError_t launch_face_multi_##D(const FaceParams& p, const MultiArgs& m, int grid,     \
                                    cudaStream_t s);                                    \
  cudaError_t launch_limiter_##D(const LimParams& p, cudaStream_t s);                   \
  cudaError_t launch_predict2d_##D(const Predict2DParams& p, cudaStream_t s);           \
  cudaError_t launch_face2d_##D(const Face2DParams& p, cudaStream_t s);                 \
  cudaError_t launch_cfl2d_##D(const Cfl2DParams& p, cudaStream_t s);                   \
  cudaError_t launch_predict3d_##D(const Predict3DParams& p, cudaStream_t s);           \
  cudaError_t launch_face3d_##D(const Face3DParams& p, cudaStream_t s);                 \
  cudaError_t launch_cfl3d_##D(const Cfl3DParams& p, cudaStream_t s);                   \
  cudaError_t prepare_degree_##D();

ADER_DECLARE_DEGREE(0)
ADER_DECLARE_DEGREE(1)
ADER_DECLARE_DEGREE(2)
ADER_DECLARE_DEGREE(3)
ADER_DECLARE_DEGREE(4)
ADER_DECLARE_DEGREE(5)
ADER_DECLARE_DEGREE(6)
ADER_DECLARE_DEGREE(7)

}  // namespace ader
