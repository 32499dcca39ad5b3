// ader_capi.cu -- the C ABI of include/ader.h: contexts, caller-owned device
// workspace, kernel sequencing, the device-resident time loop under CUDA graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/ader.h"
#include "ader_dispatch.h"
#include "ader_launch.h"
#include "ader_ops.h"

using namespace ader;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct HostFlags {
  int done;
  int status;
  long long steps;
  unsigned long long lam;
  double t;
};

}  // namespace

struct ader_ctx {
  Basis basis{};
  ader_mesh mesh{};
  ader_options opt{};
  int N = 0, n = 1, scheme = 0;
  int M = kM;  // variables per node: 3 (Euler) or kMR (reacting system)
  double dx = 0.0;
  int dims = 1;                   // 2 / 3: the meshes of ader_init_2d / ader_init_3d
  long long nx = 0, ny = 0, nz = 1;  // cells per direction (mesh.n_cells = nx ny nz)
  double dy = 0.0, dz = 0.0;
  double* gface2 = nullptr;       // 2D: face fluxes [cell][dir][k][4]; 3D: [cell][d][a][c][5]
  // workspace (caller-owned)
  char* ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t user_stream = nullptr;
  cudaStream_t stream = nullptr;  // private stream for work and graph capture
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_poll[2] = {nullptr, nullptr};
  HostFlags* hflags = nullptr;    // pinned, 2 entries
  DevCtl* ctl = nullptr;
  double* trace = nullptr;
  double* wrec = nullptr;
  double* ubuf = nullptr;
  double* hbuf = nullptr;
  double* sbuf = nullptr;         // the context-resident state (ader_set_state)
  bool state_set = false;
  double state_t = 0.0;           // simulated time of the resident state
  // shard of a periodic global mesh (ader_init_shard): local cells
  // [shard_first, shard_first + shard_local) held at offset shard_halo
  long long shard_first = -1, shard_local = 0, shard_global = 0;
  int shard_halo = 0;
  float* lim_mmf = nullptr;   // limiter: FP32 subcell extrema of u^n and bounds [cell][9]
  Sub1Ops sub1{};             // limiter: degree-1 operators of the subcell scheme
  int* lim_flag = nullptr;    // limiter: troubled flags [cell]
  long long* lim_list = nullptr;  // limiter: troubled-cell list [cell]
  double* lim_gface = nullptr;    // limiter: subcell fluxes of troubled cells' faces [cell][6]
  // cached solve graph
  cudaGraphExec_t gexec = nullptr;
  const double* g_u = nullptr;
  double g_tend = 0.0;
  long long g_maxsteps = 0;
  int g_steps = 0;
  bool prepared = false;
  char err[512] = {0};
  // profiling: 4 timing events per graph step (start, predictor start, predictor end, end)
  static constexpr int kMaxGraphSteps = 64;
  cudaEvent_t pev[kMaxGraphSteps][4] = {};
  bool pev_ready = false;
  long long prof_steps = 0;
  double prof_ms[3] = {0, 0, 0};  // weno, predict, face
  long long launches = 0;         // kernels launched by the last call
  ader_tuning tune{32, 64, 0, 0.0, 0.0, 0.0};  // graph_steps 0 = mesh-size rule
};

namespace {

ader_status fail(ader_ctx* c, ader_status st, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(ctx, ADER_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

bool is_weno_degree(int N) { return N == 2 || N == 4; }

int64_t state_count(const ader_ctx* c) {
  if (c->dims == 2) return c->mesh.n_cells * c->n * c->n * kM2;
  if (c->dims == 3) return c->mesh.n_cells * c->n * c->n * c->n * kM3;
  return c->scheme == ADER_SCHEME_DG ? c->mesh.n_cells * c->n * c->M : c->mesh.n_cells * kM;
}

// DG: [cell][qR | qL | u + volume (+ source)], M n doubles each; FV: [cell][qR | qL]
size_t trace_doubles(const ader_ctx* c) {
  if (c->dims == 2) return (size_t)c->mesh.n_cells * 5 * c->n * c->n * kM2;  // xR xL yR yL volume
  if (c->dims == 3) return (size_t)c->mesh.n_cells * 7 * c->n * c->n * c->n * kM3;  // 6 faces, volume
  return (size_t)c->mesh.n_cells * (c->scheme == ADER_SCHEME_DG ? 3 : 2) * c->M * c->n;
}

size_t workspace_bytes(const ader_ctx* c) {
  size_t b = align_up(sizeof(DevCtl));
  b += align_up(trace_doubles(c) * sizeof(double));
  if (c->scheme == ADER_SCHEME_WENO_FV) b += align_up((size_t)c->mesh.n_cells * c->n * kM * 8);
  b += 3 * align_up((size_t)state_count(c) * sizeof(double));  // ubuf, hbuf, sbuf
  if (c->dims == 2) b += align_up((size_t)c->mesh.n_cells * 2 * c->n * kM2 * sizeof(double));
  if (c->dims == 3) b += align_up((size_t)c->mesh.n_cells * 3 * c->n * c->n * kM3 * sizeof(double));
  if (c->opt.limiter)
    b += align_up((size_t)c->mesh.n_cells * 9 * sizeof(float)) +
         align_up((size_t)c->mesh.n_cells * 6 * sizeof(double)) +
         align_up((size_t)c->mesh.n_cells * sizeof(long long)) +
         align_up((size_t)c->mesh.n_cells * sizeof(int));
  return b;
}

int kernels_per_step(const ader_ctx* c) {
  if (c->dims >= 2) return 3;  // predictor, face fluxes, update with lambda_max
  int k = c->scheme == ADER_SCHEME_WENO_FV ? 3 : 2;
  if (c->opt.limiter) k += 4;
  return k;
}

StepParams make_step(const ader_ctx* c, int mode, int par, double dt, double t_end,
                     long long max_steps) {
  StepParams sp{};
  sp.mode = mode;
  sp.par = par;
  sp.dt_fixed = dt;
  sp.t_end = t_end;
  sp.max_steps = max_steps;
  sp.cfl_factor = c->scheme == ADER_SCHEME_DG ? c->opt.cfl * c->dx / (double)(2 * c->N + 1)
                                              : c->opt.cfl * c->dx;
  // 2D: dt = CFL / (d (2N+1)) / max(lambda_x / dx, lambda_y / dy), d = 2 (Sec. 1.5)
  if (c->dims >= 2) sp.cfl_factor = c->opt.cfl / ((double)c->dims * (double)(2 * c->N + 1));
  sp.inv_dx = 1.0 / c->dx;
  sp.ctl = c->ctl;
  return sp;
}

PredictParams make_predict(const ader_ctx* c, const double* u_nodal, const StepParams& sp) {
  PredictParams p{};
  p.u = u_nodal;
  p.ncells = c->mesh.n_cells;
  p.out_mode = kOutTrace;
  p.trace = c->trace;
  p.dg = c->scheme == ADER_SCHEME_DG;
  p.prec = c->opt.precision;
  p.sweeps = c->opt.fp64_sweeps;
  p.max_iter = c->opt.picard_max_iter;
  p.fixed_iter = c->opt.picard_fixed_iter;
  p.cpb = c->tune.predict_cells_per_block;
  p.sys = c->opt.system;
  p.om2 = c->opt.omega * c->opt.omega;
  p.tol = c->opt.picard_tol;
  p.tol32 = (float)c->opt.fp32_tol;
  p.gamma = c->opt.gamma;
  p.gm1 = c->opt.gamma - 1.0;
  p.gamf = (float)p.gamma;
  p.gm1f = (float)p.gm1;
  p.c1f = (float)(0.5 * (3.0 - p.gamma));
  p.c2f = (float)(0.5 * p.gm1);
  p.tolf = (float)p.tol;
  p.sp = sp;
  p.ops = c->basis.d;
  p.opf = c->basis.f;
  return p;
}

FaceParams make_face(const ader_ctx* c, const double* v_old, double* u_new, const StepParams& sp,
                     int want_lambda) {
  FaceParams f{};
  f.trace = c->trace;
  f.v_old = v_old;
  f.u_new = u_new;
  f.ncells = c->mesh.n_cells;
  f.dg = c->scheme == ADER_SCHEME_DG;
  f.want_lambda = want_lambda;
  f.cpf = c->tune.face_cells_per_block;
  f.sys = c->opt.system;
  f.bc = c->opt.bc;
  f.Ns = c->basis.Ns;
  f.nodal = c->opt.cfl_mode == 1;
  f.gamma = c->opt.gamma;
  f.gm1 = c->opt.gamma - 1.0;
  f.sp = sp;
  f.ops = c->basis.d;
  return f;
}

ader_status need_bound(ader_ctx* ctx) {
  if (!ctx) return ADER_ERR_ARG;
  if (!ctx->ws) return fail(ctx, ADER_ERR_STATE, "no workspace bound (call ader_bind first)");
  return ADER_OK;
}

CflParams make_cfl(const ader_ctx* ctx, const double* u, int slot) {
  CflParams p{};
  p.u = u;
  p.ncells = ctx->mesh.n_cells;
  p.vars = ctx->scheme == ADER_SCHEME_DG ? ctx->M : kM;
  p.dg = ctx->scheme == ADER_SCHEME_DG;
  p.slot = slot;
  p.Ns = ctx->basis.Ns;
  p.nodal = ctx->opt.cfl_mode == 1;
  p.gamma = ctx->opt.gamma;
  p.gm1 = ctx->opt.gamma - 1.0;
  p.ctl = ctx->ctl;
  p.ops = ctx->basis.d;
  return p;
}

Cfl2DParams make_cfl2d(const ader_ctx* ctx, const double* u, int slot) {
  Cfl2DParams p{};
  p.u = u;
  p.ncells = ctx->mesh.n_cells;
  p.gamma = ctx->opt.gamma;
  p.gm1 = ctx->opt.gamma - 1.0;
  p.inv_dx = 1.0 / ctx->dx;
  p.inv_dy = 1.0 / ctx->dy;
  p.ctl = ctx->ctl;
  p.slot = slot;
  for (int j = 0; j < kMaxNs; ++j)
    for (int k = 0; k < kMaxN; ++k) {
      p.P[j][k] = ctx->basis.d.P[j][k];
      p.Pf[j][k] = (float)ctx->basis.d.P[j][k];
    }
  return p;
}

Cfl3DParams make_cfl3d(const ader_ctx* ctx, const double* u, int slot) {
  Cfl3DParams p{};
  p.u = u;
  p.ncells = ctx->mesh.n_cells;
  p.gamma = ctx->opt.gamma;
  p.gm1 = ctx->opt.gamma - 1.0;
  p.inv_dx = 1.0 / ctx->dx;
  p.inv_dy = 1.0 / ctx->dy;
  p.inv_dz = 1.0 / ctx->dz;
  p.ctl = ctx->ctl;
  p.slot = slot;
  for (int j = 0; j < kMaxNs; ++j)
    for (int k = 0; k < kMaxN; ++k) {
      p.P[j][k] = ctx->basis.d.P[j][k];
      p.Pf[j][k] = (float)ctx->basis.d.P[j][k];
    }
  return p;
}

// enqueue the CFL kernel into lam[slot] (resets the slot first)
ader_status enqueue_cfl(ader_ctx* ctx, const double* u, int slot) {
  CK(cudaMemsetAsync(&ctx->ctl->lam[slot], 0, sizeof(unsigned long long), ctx->stream));
  if (ctx->dims == 2) {
    Cfl2DParams p = make_cfl2d(ctx, u, slot);
    CK(do_cfl2d(ctx->N, p, ctx->stream));
    ctx->launches += 1;
    return ADER_OK;
  }
  if (ctx->dims == 3) {
    Cfl3DParams p = make_cfl3d(ctx, u, slot);
    CK(do_cfl3d(ctx->N, p, ctx->stream));
    ctx->launches += 1;
    return ADER_OK;
  }
  CflParams p = make_cfl(ctx, u, slot);
  CK(do_cfl(ctx->N, p, ctx->stream));
  ctx->launches += 1;
  return ADER_OK;
}

// the a posteriori subcell limiter on the candidate in dst (u^n in src)
ader_status enqueue_limiter(ader_ctx* ctx, const double* src, double* dst, const StepParams& sp,
                            int want_lambda) {
  LimParams l{};
  l.u_old = src;
  l.u = dst;
  l.trace = ctx->trace;
  l.mmf = ctx->lim_mmf;
  l.troubled = ctx->lim_flag;
  l.list = ctx->lim_list;
  l.gface = ctx->lim_gface;
  l.ncells = ctx->mesh.n_cells;
  l.bc = ctx->opt.bc;
  l.Ns = ctx->basis.Ns;
  l.mode = ctx->opt.limiter;
  l.want_lambda = want_lambda;
  l.max_iter = ctx->opt.picard_max_iter;
  l.fixed_iter = ctx->opt.picard_fixed_iter;
  l.tol = ctx->opt.picard_tol;
  l.s1 = ctx->sub1;
  l.gamma = ctx->opt.gamma;
  l.gm1 = ctx->opt.gamma - 1.0;
  l.delta0 = ctx->opt.nad_delta0;
  l.eps = ctx->opt.nad_eps;
  l.sp = sp;
  l.ops = ctx->basis.d;
  std::memcpy(l.R, ctx->basis.R, sizeof(l.R));
  double pabs = 0.0;
  for (int j = 0; j < kMaxNs; ++j) {
    double a = 0.0;
    for (int k = 0; k < kMaxN; ++k) {
      l.Pf[j][k] = (float)ctx->basis.d.P[j][k];
      a += std::fabs(ctx->basis.d.P[j][k]);
    }
    pabs = std::max(pabs, a);
  }
  l.pabs = (float)(pabs * (1.0 + 1e-6));  // rounded up
  CK(do_limiter(ctx->N, l, ctx->stream));
  ctx->launches += 4;
  return ADER_OK;
}

// one step from src to dst with the given step parameters; ev (4 events or
// null) are recorded around the kernels as external event nodes when captured
// one 2D step: predictor, face fluxes + update, lambda_max of the new state
ader_status enqueue_step2d(ader_ctx* ctx, const double* src, double* dst, const StepParams& sp,
                           int want_lambda, cudaEvent_t* ev) {
  if (ev) CK(cudaEventRecordWithFlags(ev[0], ctx->stream, cudaEventRecordExternal));
  if (ev) CK(cudaEventRecordWithFlags(ev[1], ctx->stream, cudaEventRecordExternal));
  Predict2DParams p{};
  p.u = src;
  p.trace = ctx->trace;
  p.ncells = ctx->mesh.n_cells;
  p.max_iter = ctx->opt.picard_max_iter;
  p.fixed_iter = ctx->opt.picard_fixed_iter;
  p.tol = ctx->opt.picard_tol;
  p.gamma = ctx->opt.gamma;
  p.gm1 = ctx->opt.gamma - 1.0;
  p.inv_dy = 1.0 / ctx->dy;
  p.sp = sp;
  p.ops = ctx->basis.d;
  CK(do_predict2d(ctx->N, p, ctx->stream));
  if (ev) CK(cudaEventRecordWithFlags(ev[2], ctx->stream, cudaEventRecordExternal));
  Face2DParams f{};
  f.trace = ctx->trace;
  f.gface = ctx->gface2;
  f.u_new = dst;
  f.ncells = ctx->mesh.n_cells;
  f.nx = ctx->nx;
  f.ny = ctx->ny;
  f.gamma = ctx->opt.gamma;
  f.gm1 = ctx->opt.gamma - 1.0;
  f.inv_dy = 1.0 / ctx->dy;
  f.want_lambda = want_lambda;  // the predictor of this step has reset the slot
  f.sp = sp;
  f.ops = ctx->basis.d;
  for (int j = 0; j < kMaxNs; ++j)
    for (int k = 0; k < kMaxN; ++k) f.Pf[j][k] = (float)ctx->basis.d.P[j][k];
  CK(do_face2d(ctx->N, f, ctx->stream));
  ctx->launches += 3;
  if (ev) CK(cudaEventRecordWithFlags(ev[3], ctx->stream, cudaEventRecordExternal));
  return ADER_OK;
}

// one 3D step: predictor, face fluxes + update, lambda_max of the new state
ader_status enqueue_step3d(ader_ctx* ctx, const double* src, double* dst, const StepParams& sp,
                           int want_lambda, cudaEvent_t* ev) {
  if (ev) CK(cudaEventRecordWithFlags(ev[0], ctx->stream, cudaEventRecordExternal));
  if (ev) CK(cudaEventRecordWithFlags(ev[1], ctx->stream, cudaEventRecordExternal));
  Predict3DParams p{};
  p.u = src;
  p.trace = ctx->trace;
  p.ncells = ctx->mesh.n_cells;
  p.max_iter = ctx->opt.picard_max_iter;
  p.fixed_iter = ctx->opt.picard_fixed_iter;
  p.tol = ctx->opt.picard_tol;
  p.gamma = ctx->opt.gamma;
  p.gm1 = ctx->opt.gamma - 1.0;
  p.inv_dy = 1.0 / ctx->dy;
  p.inv_dz = 1.0 / ctx->dz;
  p.sp = sp;
  p.ops = ctx->basis.d;
  CK(do_predict3d(ctx->N, p, ctx->stream));
  if (ev) CK(cudaEventRecordWithFlags(ev[2], ctx->stream, cudaEventRecordExternal));
  Face3DParams f{};
  f.trace = ctx->trace;
  f.gface = ctx->gface2;
  f.u_new = dst;
  f.ncells = ctx->mesh.n_cells;
  f.nx = ctx->nx;
  f.ny = ctx->ny;
  f.nz = ctx->nz;
  f.gamma = ctx->opt.gamma;
  f.gm1 = ctx->opt.gamma - 1.0;
  f.inv_dy = 1.0 / ctx->dy;
  f.inv_dz = 1.0 / ctx->dz;
  f.want_lambda = want_lambda;  // the predictor of this step has reset the slot
  f.sp = sp;
  f.ops = ctx->basis.d;
  for (int j = 0; j < kMaxNs; ++j)
    for (int k = 0; k < kMaxN; ++k) f.Pf[j][k] = (float)ctx->basis.d.P[j][k];
  CK(do_face3d(ctx->N, f, ctx->stream));
  ctx->launches += 3;
  if (ev) CK(cudaEventRecordWithFlags(ev[3], ctx->stream, cudaEventRecordExternal));
  return ADER_OK;
}

ader_status enqueue_step(ader_ctx* ctx, const double* src, double* dst, const StepParams& sp,
                         int want_lambda, cudaEvent_t* ev = nullptr) {
  if (ctx->dims == 2) return enqueue_step2d(ctx, src, dst, sp, want_lambda, ev);
  if (ctx->dims == 3) return enqueue_step3d(ctx, src, dst, sp, want_lambda, ev);
  const double* nodal = src;
  if (ev) CK(cudaEventRecordWithFlags(ev[0], ctx->stream, cudaEventRecordExternal));
  if (ctx->scheme == ADER_SCHEME_WENO_FV) {
    WenoParams w{};
    w.v = src;
    w.w = ctx->wrec;
    w.ncells = ctx->mesh.n_cells;
    w.wo = ctx->basis.weno;
    CK(do_weno(ctx->N, w, ctx->stream));
    nodal = ctx->wrec;
  }
  if (ev) CK(cudaEventRecordWithFlags(ev[1], ctx->stream, cudaEventRecordExternal));
  PredictParams p = make_predict(ctx, nodal, sp);
  CK(do_predict(ctx->N, p, ctx->stream));
  if (ev) CK(cudaEventRecordWithFlags(ev[2], ctx->stream, cudaEventRecordExternal));
  FaceParams f = make_face(ctx, src, dst, sp, ctx->opt.limiter ? 0 : want_lambda);
  CK(do_face(ctx->N, f, ctx->stream));
  ctx->launches += ctx->scheme == ADER_SCHEME_WENO_FV ? 3 : 2;
  if (ctx->opt.limiter) {
    // with lambda_max of the limited state for the next step (the predictor of
    // this step has reset the slot)
    ader_status st = enqueue_limiter(ctx, src, dst, sp, want_lambda);
    if (st != ADER_OK) return st;
  }
  if (ev) CK(cudaEventRecordWithFlags(ev[3], ctx->stream, cudaEventRecordExternal));
  return ADER_OK;
}

// fork the private stream from the caller's stream / join back
ader_status fork_in(ader_ctx* ctx) {
  CK(cudaEventRecord(ctx->ev_fork, ctx->user_stream));
  CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_fork, 0));
  return ADER_OK;
}
ader_status join_out(ader_ctx* ctx) {
  CK(cudaEventRecord(ctx->ev_join, ctx->stream));
  CK(cudaStreamWaitEvent(ctx->user_stream, ctx->ev_join, 0));
  return ADER_OK;
}

ader_status reset_ctl(ader_ctx* ctx) {
  CK(cudaMemsetAsync(ctx->ctl, 0, sizeof(DevCtl), ctx->stream));
  ctx->launches = 0;
  return ADER_OK;
}

ader_status status_from_flags(ader_ctx* ctx, int st) {
  if (st & kStNonPhysical)
    return fail(ctx, ADER_ERR_NONPHYSICAL, "non-physical state (rho <= 0, p <= 0 or non-finite)");
  if (st & kStNotConverged)
    return fail(ctx, ADER_ERR_NOT_CONVERGED, "Picard iteration cap reached in some cell");
  return ADER_OK;
}

bool valid_cpb(int N, int cpb) {
  const int threads = cpb * (N + 1);
  return (cpb == 16 || cpb == 32 || cpb == 64) && (threads % 32 == 0 || cpb == 16) &&
         threads <= 512 && (N <= 5 || cpb <= 32);
}

int graph_steps_for(int64_t ncells) {
  if (ncells <= 4096) return 64;
  if (ncells <= 65536) return 16;
  if (ncells <= 524288) return 8;
  return 4;
}

}  // namespace

extern "C" {

const char* ader_status_string(int s) {
  switch (s) {
    case ADER_OK: return "ok";
    case ADER_ERR_ARG: return "invalid argument";
    case ADER_ERR_NOMEM: return "workspace missing or too small";
    case ADER_ERR_CUDA: return "CUDA error";
    case ADER_ERR_NOT_CONVERGED: return "Picard iteration did not converge";
    case ADER_ERR_NONPHYSICAL: return "non-physical state";
    case ADER_ERR_TIMEOUT: return "device wait timed out";
    case ADER_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

ader_status ader_default_options(ader_options* o) {
  if (!o) return ADER_ERR_ARG;
  o->gamma = 1.4;
  o->cfl = 0.4;
  o->picard_tol = 1e-13;
  o->picard_max_iter = 0;
  o->picard_fixed_iter = 0;
  o->precision = ADER_PREC_FP64;
  o->fp64_sweeps = 1;
  o->fp32_tol = 1e-6;
  o->profile = 0;
  o->system = ADER_SYSTEM_EULER;
  o->omega = 1.0;
  o->bc = ADER_BC_PERIODIC;
  o->limiter = 0;
  o->nad_delta0 = 1e-4;
  o->nad_eps = 1e-3;
  o->cfl_mode = 0;
  return ADER_OK;
}

ader_status ader_init(const ader_mesh* mesh, int degree, int scheme, const ader_options* opt,
                      ader_ctx** out) {
  if (!out) return ADER_ERR_ARG;
  *out = nullptr;
  if (!mesh || mesh->n_cells <= 0 || !(mesh->x1 > mesh->x0)) return ADER_ERR_ARG;
  if (scheme != ADER_SCHEME_DG && scheme != ADER_SCHEME_WENO_FV) return ADER_ERR_ARG;
  if (degree < 0 || degree > kMaxDeg) return ADER_ERR_ARG;
  if (scheme == ADER_SCHEME_WENO_FV && !is_weno_degree(degree)) return ADER_ERR_ARG;
  // every per-cell index fits in int64 with room for the 9 (N+1) 3 doubles per cell
  if (mesh->n_cells > (int64_t)1 << 36) return ADER_ERR_ARG;
  ader_ctx* c = new (std::nothrow) ader_ctx();
  if (!c) return ADER_ERR_NOMEM;
  c->mesh = *mesh;
  c->N = degree;
  c->n = degree + 1;
  c->scheme = scheme;
  c->dx = (mesh->x1 - mesh->x0) / (double)mesh->n_cells;
  // default tiles: half-size below two blocks per SM, so that a small mesh
  // spreads over more SMs (autotuning or ader_set_tuning replaces them)
  if (mesh->n_cells < 152LL * 2 * 32) c->tune.predict_cells_per_block = 16;
  if (mesh->n_cells < 152LL * 2 * 64) c->tune.face_cells_per_block = 32;
  if (opt) {
    c->opt = *opt;
  } else {
    ader_default_options(&c->opt);
  }
  ader_options& o = c->opt;
  if (o.picard_max_iter <= 0) o.picard_max_iter = 4 * c->n + 8;
  if (!(o.gamma > 1.0) || !(o.cfl > 0.0) || !(o.picard_tol >= 0.0) || o.picard_fixed_iter < 0 ||
      (o.precision != ADER_PREC_FP64 && o.precision != ADER_PREC_FP32_PREDICTOR &&
       o.precision != ADER_PREC_FF_PREDICTOR && o.precision != ADER_PREC_FP32_FF_SWEEPS &&
       o.precision != ADER_PREC_FP32_INCREMENT) ||
      ((o.precision == ADER_PREC_FP32_PREDICTOR || o.precision == ADER_PREC_FP32_FF_SWEEPS) &&
       o.fp64_sweeps < 1) || o.picard_max_iter > 10000 ||
      (o.system != ADER_SYSTEM_EULER && o.system != ADER_SYSTEM_REACTING &&
       o.system != ADER_SYSTEM_TRACER) ||
      (o.system == ADER_SYSTEM_TRACER &&
       (scheme != ADER_SCHEME_DG || o.precision != ADER_PREC_FP64 || o.bc != ADER_BC_PERIODIC)) ||
      (o.system == ADER_SYSTEM_REACTING &&
       (scheme != ADER_SCHEME_DG || o.precision != ADER_PREC_FP64 || !std::isfinite(o.omega))) ||
      (o.bc != ADER_BC_PERIODIC && o.bc != ADER_BC_OUTFLOW) ||
      (o.bc == ADER_BC_OUTFLOW && scheme != ADER_SCHEME_DG) || (o.limiter < 0 || o.limiter > 2) ||
      (o.limiter && (scheme != ADER_SCHEME_DG || o.system != ADER_SYSTEM_EULER || degree < 1)) ||
      !(o.nad_delta0 >= 0.0) || !(o.nad_eps >= 0.0) || (o.cfl_mode != 0 && o.cfl_mode != 1) ||
      (o.cfl_mode == 1 &&
       (scheme != ADER_SCHEME_DG || o.system != ADER_SYSTEM_EULER || o.limiter != 0))) {
    delete c;
    return ADER_ERR_ARG;
  }
  c->M = o.system == ADER_SYSTEM_REACTING ? kMR : (o.system == ADER_SYSTEM_TRACER ? kMN : kM);
  if (build_basis(degree, scheme == ADER_SCHEME_WENO_FV, &c->basis) != 0) {
    delete c;
    return ADER_ERR_ARG;
  }
  if (o.limiter) {
    Basis b1;
    if (build_basis(1, false, &b1) != 0) {
      delete c;
      return ADER_ERR_ARG;
    }
    for (int k = 0; k < 2; ++k) {
      c->sub1.xi[k] = b1.d.xi[k];
      c->sub1.w[k] = b1.d.w[k];
      c->sub1.psi0[k] = b1.d.psi0[k];
      c->sub1.psi1[k] = b1.d.psi1[k];
      for (int l = 0; l < 2; ++l) {
        c->sub1.kt[k][l] = b1.d.kt[k][l];
        c->sub1.kap[k][l] = b1.d.kap[k][l];
      }
    }
  }
  *out = c;
  return ADER_OK;
}

ader_status ader_init_2d(const ader_mesh2d* mesh, int degree, const ader_options* opt,
                         ader_ctx** out) {
  if (!out) return ADER_ERR_ARG;
  *out = nullptr;
  if (!mesh || mesh->nx <= 0 || mesh->ny <= 0 || !(mesh->x1 > mesh->x0) || !(mesh->y1 > mesh->y0))
    return ADER_ERR_ARG;
  if (degree < 0 || degree > kMaxDeg) return ADER_ERR_ARG;
  if (mesh->nx > ((int64_t)1 << 30) / mesh->ny) return ADER_ERR_ARG;
  ader_options o;
  if (opt) {
    o = *opt;
  } else {
    ader_default_options(&o);
  }
  // the 2D path: DG, Euler, FP64 predictor, periodic, no limiter, subcell CFL
  if (o.system != ADER_SYSTEM_EULER || o.precision != ADER_PREC_FP64 || o.bc != ADER_BC_PERIODIC ||
      o.limiter != 0 || o.cfl_mode != 0)
    return ADER_ERR_ARG;
  ader_mesh m1{mesh->nx * mesh->ny, mesh->x0, mesh->x1};
  ader_ctx* c = nullptr;
  ader_status st = ader_init(&m1, degree, ADER_SCHEME_DG, &o, &c);
  if (st != ADER_OK) return st;
  c->dims = 2;
  c->nx = mesh->nx;
  c->ny = mesh->ny;
  c->dx = (mesh->x1 - mesh->x0) / (double)mesh->nx;
  c->dy = (mesh->y1 - mesh->y0) / (double)mesh->ny;
  *out = c;
  return ADER_OK;
}

ader_status ader_init_3d(const ader_mesh3d* mesh, int degree, const ader_options* opt,
                         ader_ctx** out) {
  if (!out) return ADER_ERR_ARG;
  *out = nullptr;
  if (!mesh || mesh->nx <= 0 || mesh->ny <= 0 || mesh->nz <= 0 || !(mesh->x1 > mesh->x0) ||
      !(mesh->y1 > mesh->y0) || !(mesh->z1 > mesh->z0))
    return ADER_ERR_ARG;
  if (degree < 0 || degree > kMax3DDegree) return ADER_ERR_ARG;
  if (mesh->nx > ((int64_t)1 << 28) / mesh->ny / mesh->nz) return ADER_ERR_ARG;
  ader_options o;
  if (opt) {
    o = *opt;
  } else {
    ader_default_options(&o);
  }
  if (o.system != ADER_SYSTEM_EULER || o.precision != ADER_PREC_FP64 || o.bc != ADER_BC_PERIODIC ||
      o.limiter != 0 || o.cfl_mode != 0)
    return ADER_ERR_ARG;
  ader_mesh m1{mesh->nx * mesh->ny * mesh->nz, mesh->x0, mesh->x1};
  ader_ctx* c = nullptr;
  ader_status st = ader_init(&m1, degree, ADER_SCHEME_DG, &o, &c);
  if (st != ADER_OK) return st;
  c->dims = 3;
  c->nx = mesh->nx;
  c->ny = mesh->ny;
  c->nz = mesh->nz;
  c->dx = (mesh->x1 - mesh->x0) / (double)mesh->nx;
  c->dy = (mesh->y1 - mesh->y0) / (double)mesh->ny;
  c->dz = (mesh->z1 - mesh->z0) / (double)mesh->nz;
  *out = c;
  return ADER_OK;
}

void ader_destroy(ader_ctx* c) {
  if (!c) return;
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->stream) cudaStreamDestroy(c->stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  for (auto& e : c->ev_poll)
    if (e) cudaEventDestroy(e);
  if (c->hflags) cudaFreeHost(c->hflags);
  if (c->pev_ready)
    for (auto& row : c->pev)
      for (auto& e : row)
        if (e) cudaEventDestroy(e);
  delete c;
}

const char* ader_last_error(const ader_ctx* c) { return c ? c->err : "null context"; }

int64_t ader_state_count(const ader_ctx* c) { return c ? state_count(c) : -1; }
int64_t ader_predictor_count(const ader_ctx* c) {
  if (c && c->dims == 2) return c->mesh.n_cells * c->n * c->n * c->n * kM2;
  if (c && c->dims == 3) return c->mesh.n_cells * c->n * c->n * c->n * c->n * kM3;
  return c ? c->mesh.n_cells * c->n * c->n * c->M : -1;
}
size_t ader_workspace_bytes(const ader_ctx* c) { return c ? workspace_bytes(c) : 0; }

ader_status ader_node_coords(const ader_ctx* c, double* x, int64_t count) {
  if (!c || !x || c->dims != 1) return ADER_ERR_ARG;
  const int per = c->scheme == ADER_SCHEME_DG ? c->n : 1;
  if (count != c->mesh.n_cells * per) return ADER_ERR_ARG;
  for (int64_t i = 0; i < c->mesh.n_cells; ++i)
    for (int k = 0; k < per; ++k)
      x[i * per + k] = c->mesh.x0 + c->dx * ((double)i + (per == 1 ? 0.5 : c->basis.d.xi[k]));
  return ADER_OK;
}

ader_status ader_get_table(const ader_ctx* c, const char* name, double* out, int64_t count) {
  if (!c || !name || !out) return ADER_ERR_ARG;
  const int n = c->n;
  const OpsD& d = c->basis.d;
  auto vec = [&](const double* src, int m) -> ader_status {
    if (count != m) return ADER_ERR_ARG;
    std::memcpy(out, src, sizeof(double) * m);
    return ADER_OK;
  };
  auto mat = [&](const double (*src)[kMaxN], int rows) -> ader_status {
    if (count != (int64_t)rows * n) return ADER_ERR_ARG;
    for (int i = 0; i < rows; ++i)
      for (int j = 0; j < n; ++j) out[i * n + j] = src[i][j];
    return ADER_OK;
  };
  if (!strcmp(name, "xi")) return vec(d.xi, n);
  if (!strcmp(name, "w")) return vec(d.w, n);
  if (!strcmp(name, "psi0")) return vec(d.psi0, n);
  if (!strcmp(name, "psi1")) return vec(d.psi1, n);
  if (!strcmp(name, "kt")) return mat(d.kt, n);
  if (!strcmp(name, "kap")) return mat(d.kap, n);
  if (!strcmp(name, "dphi")) return mat(c->basis.dphi, n);
  if (!strcmp(name, "dtil")) return mat(c->basis.dtil, n);
  if (!strcmp(name, "P")) return mat(d.P, c->basis.Ns);
  if (!strcmp(name, "R")) {  // [n][Ns]
    const int Ns = c->basis.Ns;
    if (count != (int64_t)n * Ns) return ADER_ERR_ARG;
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < Ns; ++j) out[k * Ns + j] = c->basis.R[k][j];
    return ADER_OK;
  }
  const int H = (n + 1) / 2;
  auto half = [&](const double (*src)[kMaxH]) -> ader_status {
    if (count != (int64_t)H * H) return ADER_ERR_ARG;
    for (int i = 0; i < H; ++i)
      for (int j = 0; j < H; ++j) out[i * H + j] = src[i][j];
    return ADER_OK;
  };
  if (!strcmp(name, "ksa")) return half(d.ksa);
  if (!strcmp(name, "ksb")) return half(d.ksb);
  if (c->scheme == ADER_SCHEME_WENO_FV) {
    const WenoOps& wo = c->basis.weno;
    if (!strcmp(name, "wvnod")) return mat(wo.vnod, n);
    if (!strcmp(name, "wamono")) {
      if (count != (int64_t)3 * n * n) return ADER_ERR_ARG;
      for (int S = 0; S < 3; ++S)
        for (int j = 0; j < n; ++j)
          for (int k = 0; k < n; ++k) out[(S * n + j) * n + k] = wo.amono[S][j][k];
      return ADER_OK;
    }
  }
  return ADER_ERR_ARG;
}

ader_status ader_bind(ader_ctx* ctx, void* ws, size_t bytes, void* stream) {
  if (!ctx || !ws) return ADER_ERR_ARG;
  if (bytes < workspace_bytes(ctx))
    return fail(ctx, ADER_ERR_NOMEM, "workspace %zu bytes < required %zu", bytes,
                workspace_bytes(ctx));
  if (reinterpret_cast<uintptr_t>(ws) % kAlign)
    return fail(ctx, ADER_ERR_ARG, "workspace must be %zu-byte aligned", kAlign);
  if (!ctx->prepared) {
    CK(dispatch_prepare(ctx->N));
    CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->ev_poll[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->ev_poll[1], cudaEventDisableTiming));
    CK(cudaMallocHost(&ctx->hflags, 2 * sizeof(HostFlags)));
    ctx->prepared = true;
  }
  if (ctx->gexec) {
    cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
  }
  ctx->ws = static_cast<char*>(ws);
  ctx->ws_bytes = bytes;
  ctx->user_stream = static_cast<cudaStream_t>(stream);
  char* p = ctx->ws;
  ctx->ctl = reinterpret_cast<DevCtl*>(p);
  p += align_up(sizeof(DevCtl));
  ctx->trace = reinterpret_cast<double*>(p);
  p += align_up(trace_doubles(ctx) * sizeof(double));
  if (ctx->scheme == ADER_SCHEME_WENO_FV) {
    ctx->wrec = reinterpret_cast<double*>(p);
    p += align_up((size_t)ctx->mesh.n_cells * ctx->n * kM * 8);
  }
  ctx->ubuf = reinterpret_cast<double*>(p);
  p += align_up((size_t)state_count(ctx) * sizeof(double));
  ctx->hbuf = reinterpret_cast<double*>(p);
  p += align_up((size_t)state_count(ctx) * sizeof(double));
  ctx->sbuf = reinterpret_cast<double*>(p);
  p += align_up((size_t)state_count(ctx) * sizeof(double));
  ctx->state_set = false;  // a new workspace holds no resident state
  if (ctx->dims == 2) {
    ctx->gface2 = reinterpret_cast<double*>(p);
    p += align_up((size_t)ctx->mesh.n_cells * 2 * ctx->n * kM2 * sizeof(double));
  }
  if (ctx->dims == 3) {
    ctx->gface2 = reinterpret_cast<double*>(p);
    p += align_up((size_t)ctx->mesh.n_cells * 3 * ctx->n * ctx->n * kM3 * sizeof(double));
  }
  if (ctx->opt.limiter) {
    ctx->lim_mmf = reinterpret_cast<float*>(p);
    p += align_up((size_t)ctx->mesh.n_cells * 9 * sizeof(float));
    ctx->lim_gface = reinterpret_cast<double*>(p);
    p += align_up((size_t)ctx->mesh.n_cells * 6 * sizeof(double));
    ctx->lim_list = reinterpret_cast<long long*>(p);
    p += align_up((size_t)ctx->mesh.n_cells * sizeof(long long));
    ctx->lim_flag = reinterpret_cast<int*>(p);
  }
  return ADER_OK;
}

ader_status ader_compute_dt(ader_ctx* ctx, const double* u, double t, double t_end,
                            double* dt_host) {
  ader_status st = need_bound(ctx);
  if (st != ADER_OK) return st;
  if (!u || !dt_host) return fail(ctx, ADER_ERR_ARG, "null pointer");
  if ((st = fork_in(ctx)) != ADER_OK) return st;
  if ((st = reset_ctl(ctx)) != ADER_OK) return st;
  if ((st = enqueue_cfl(ctx, u, 0)) != ADER_OK) return st;
  CK(cudaMemcpyAsync(&ctx->hflags[0].lam, &ctx->ctl->lam[0], sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hflags[0].status, &ctx->ctl->status, sizeof(int),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if ((st = join_out(ctx)) != ADER_OK) return st;
  double lam;
  std::memcpy(&lam, &ctx->hflags[0].lam, sizeof(lam));
  if ((ctx->hflags[0].status & kStNonPhysical) || !(lam > 0.0) || !std::isfinite(lam))
    return fail(ctx, ADER_ERR_NONPHYSICAL, "non-physical state in the CFL reduction");
  const StepParams sp = make_step(ctx, kDtCfl, 0, 0.0, 0.0, 0);
  double dt = sp.cfl_factor / lam;
  if (t_end > 0.0 && t + dt >= t_end) dt = t_end - t;
  *dt_host = dt;
  return ADER_OK;
}

ader_status ader_predict(ader_ctx* ctx, const double* u, double dt, double* q) {
  ader_status st = need_bound(ctx);
  if (st != ADER_OK) return st;
  if (ctx->dims != 1) return fail(ctx, ADER_ERR_ARG, "ader_predict is 1D only");
  if (ctx->opt.system == ADER_SYSTEM_TRACER)
    return fail(ctx, ADER_ERR_ARG, "the tracer system's predictor runs inside ader_step / ader_solve");
  if (!u || !q) return fail(ctx, ADER_ERR_ARG, "null pointer");
  if (std::isnan(dt)) return fail(ctx, ADER_ERR_ARG, "dt is NaN");
  if ((st = fork_in(ctx)) != ADER_OK) return st;
  if ((st = reset_ctl(ctx)) != ADER_OK) return st;
  int mode = kDtFixed;
  if (!(dt > 0.0)) {
    if ((st = enqueue_cfl(ctx, u, 0)) != ADER_OK) return st;
    mode = kDtCfl;
  }
  const StepParams sp = make_step(ctx, mode, 0, dt, 0.0, 0);
  const double* nodal = u;
  if (ctx->scheme == ADER_SCHEME_WENO_FV) {
    WenoParams w{};
    w.v = u;
    w.w = ctx->wrec;
    w.ncells = ctx->mesh.n_cells;
    w.wo = ctx->basis.weno;
    CK(do_weno(ctx->N, w, ctx->stream));
    nodal = ctx->wrec;
  }
  PredictParams p = make_predict(ctx, nodal, sp);
  p.out_mode = kOutQ;
  p.q_out = q;
  CK(do_predict(ctx->N, p, ctx->stream));
  return join_out(ctx);
}

ader_status ader_correct(ader_ctx* ctx, const double* u, const double* q, double dt,
                         double* u_new) {
  ader_status st = need_bound(ctx);
  if (st != ADER_OK) return st;
  if (ctx->dims != 1) return fail(ctx, ADER_ERR_ARG, "ader_correct is 1D only");
  if (ctx->opt.system == ADER_SYSTEM_TRACER)
    return fail(ctx, ADER_ERR_ARG, "the tracer system's corrector runs inside ader_step / ader_solve");
  if (!u || !q || !u_new) return fail(ctx, ADER_ERR_ARG, "null pointer");
  if (!(dt > 0.0)) return fail(ctx, ADER_ERR_ARG, "ader_correct needs dt > 0");
  if (u == u_new) return fail(ctx, ADER_ERR_ARG, "u and u_new must not alias");
  if ((st = fork_in(ctx)) != ADER_OK) return st;
  if ((st = reset_ctl(ctx)) != ADER_OK) return st;
  const StepParams sp = make_step(ctx, kDtFixed, 0, dt, 0.0, 0);
  PredictParams p = make_predict(ctx, u, sp);
  p.from_q = 1;
  p.q_in = q;
  CK(do_predict(ctx->N, p, ctx->stream));
  FaceParams f = make_face(ctx, u, u_new, sp, 0);
  CK(do_face(ctx->N, f, ctx->stream));
  if (ctx->opt.limiter && (st = enqueue_limiter(ctx, u, u_new, sp, 0)) != ADER_OK) return st;
  return join_out(ctx);
}

ader_status ader_step(ader_ctx* ctx, const double* u, double* u_new, double dt) {
  ader_status st = need_bound(ctx);
  if (st != ADER_OK) return st;
  if (!u || !u_new) return fail(ctx, ADER_ERR_ARG, "null pointer");
  if (u == u_new) return fail(ctx, ADER_ERR_ARG, "u and u_new must not alias");
  if (std::isnan(dt)) return fail(ctx, ADER_ERR_ARG, "dt is NaN");
  if ((st = fork_in(ctx)) != ADER_OK) return st;
  if ((st = reset_ctl(ctx)) != ADER_OK) return st;
  int mode = kDtFixed;
  if (!(dt > 0.0)) {
    if ((st = enqueue_cfl(ctx, u, 0)) != ADER_OK) return st;
    mode = kDtCfl;
  }
  const StepParams sp = make_step(ctx, mode, 0, dt, 0.0, 0);
  if ((st = enqueue_step(ctx, u, u_new, sp, 0)) != ADER_OK) return st;
  return join_out(ctx);
}

ader_status ader_weno_reconstruct(ader_ctx* ctx, const double* v, double* w) {
  ader_status st = need_bound(ctx);
  if (st != ADER_OK) return st;
  if (ctx->scheme != ADER_SCHEME_WENO_FV)
    return fail(ctx, ADER_ERR_ARG, "WENO reconstruction needs a WENO-FV context");
  if (!v || !w) return fail(ctx, ADER_ERR_ARG, "null pointer");
  if ((st = fork_in(ctx)) != ADER_OK) return st;
  WenoParams p{};
  p.v = v;
  p.w = w;
  p.ncells = ctx->mesh.n_cells;
  p.wo = ctx->basis.weno;
  CK(do_weno(ctx->N, p, ctx->stream));
  return join_out(ctx);
}

static ader_status solve_impl(ader_ctx* ctx, double* u, double t0, double t_end,
                              int64_t max_steps, int64_t* steps_out, double* t_out) {
  ader_status st = need_bound(ctx);
  if (st != ADER_OK) return st;
  if (!u) return fail(ctx, ADER_ERR_ARG, "null pointer");
  if (ctx->shard_first >= 0)
    return fail(ctx, ADER_ERR_ARG,
                "a shard's time step needs every shard's lambda_max: advance it with "
                "ader_compute_dt, a min over shards and ader_step");
  if (!(t_end > 0.0) && max_steps <= 0)
    return fail(ctx, ADER_ERR_ARG, "need t_end > 0 or max_steps > 0");
  if (std::isnan(t_end) || max_steps < 0) return fail(ctx, ADER_ERR_ARG, "bad t_end / max_steps");
  if (!(t0 >= 0.0) || !std::isfinite(t0) || (t_end > 0.0 && !(t0 < t_end)))
    return fail(ctx, ADER_ERR_ARG, "need 0 <= t0 < t_end");
  if (!(t_end > 0.0)) t_end = 0.0;
  if ((st = fork_in(ctx)) != ADER_OK) return st;
  if ((st = reset_ctl(ctx)) != ADER_OK) return st;
  if (t0 != 0.0) {  // resume: the device clock starts at t0
    ctx->hflags[1].t = t0;
    CK(cudaMemcpyAsync(&ctx->ctl->t, &ctx->hflags[1].t, sizeof(double), cudaMemcpyHostToDevice,
                       ctx->stream));
  }
  if ((st = enqueue_cfl(ctx, u, 0)) != ADER_OK) return st;

  const int K = ctx->tune.graph_steps > 0 ? ctx->tune.graph_steps : graph_steps_for(ctx->mesh.n_cells);
  const bool prof = ctx->opt.profile != 0;
  if (prof && !ctx->pev_ready) {
    for (int j = 0; j < ader_ctx::kMaxGraphSteps; ++j)
      for (int e = 0; e < 4; ++e) CK(cudaEventCreate(&ctx->pev[j][e]));
    ctx->pev_ready = true;
  }
  ctx->prof_steps = 0;
  ctx->prof_ms[0] = ctx->prof_ms[1] = ctx->prof_ms[2] = 0.0;
  if (!ctx->gexec || ctx->g_u != u || ctx->g_tend != t_end || ctx->g_maxsteps != max_steps ||
      ctx->g_steps != K) {
    if (ctx->gexec) {
      cudaGraphExecDestroy(ctx->gexec);
      ctx->gexec = nullptr;
    }
    cudaGraph_t g;
    const long long before = ctx->launches;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    ader_status cst = ADER_OK;
    for (int j = 0; j < K && cst == ADER_OK; ++j) {
      const StepParams sp = make_step(ctx, kDtSolve, j & 1, 0.0, t_end, max_steps);
      const double* src = (j & 1) ? ctx->ubuf : u;
      double* dst = (j & 1) ? u : ctx->ubuf;
      cst = enqueue_step(ctx, src, dst, sp, 1, prof ? ctx->pev[j] : nullptr);
    }
    cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
    if (cst != ADER_OK) {
      if (ce == cudaSuccess) cudaGraphDestroy(g);
      return cst;
    }
    if (ce != cudaSuccess)
      return fail(ctx, ADER_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&ctx->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess)
      return fail(ctx, ADER_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ce));
    ctx->launches = before;  // capture launches nothing; replays are counted below
    ctx->g_u = u;
    ctx->g_tend = t_end;
    ctx->g_maxsteps = max_steps;
    ctx->g_steps = K;
  }
  // Replay K-step graphs; keep two in flight and poll the 'done' flag of the
  // older one.  Steps after 'done' are no-ops on the device.
  const long long max_launches =
      max_steps > 0 ? (max_steps + K - 1) / K + 1 : (long long)4e9 / K;
  long long launches = 0;
  bool finished = false;
  long long steps_seen = 0;
  while (prof && !finished) {
    // one graph at a time: read the K step timings before the events are re-recorded
    CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
    CK(cudaMemcpyAsync(&ctx->hflags[0].done, &ctx->ctl->done, sizeof(int), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaMemcpyAsync(&ctx->hflags[0].steps, &ctx->ctl->steps, sizeof(long long),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ++launches;
    const long long active = ctx->hflags[0].steps - steps_seen;
    steps_seen = ctx->hflags[0].steps;
    for (long long j = 0; j < active && j < K; ++j) {
      float ms[3];
      for (int e = 0; e < 3; ++e) CK(cudaEventElapsedTime(&ms[e], ctx->pev[j][e], ctx->pev[j][e + 1]));
      for (int e = 0; e < 3; ++e) ctx->prof_ms[e] += ms[e];
      ctx->prof_steps += 1;
    }
    if (ctx->hflags[0].done) finished = true;
    if (launches >= max_launches) break;
  }
  while (!finished) {
    CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
    const int slot = (int)(launches & 1);
    CK(cudaMemcpyAsync(&ctx->hflags[slot].done, &ctx->ctl->done, sizeof(int),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaEventRecord(ctx->ev_poll[slot], ctx->stream));
    ++launches;
    if (launches >= 2) {
      const int prev = (int)((launches - 2) & 1);
      CK(cudaEventSynchronize(ctx->ev_poll[prev]));
      if (ctx->hflags[prev].done) finished = true;
    }
    if (launches >= max_launches) break;
  }
  ctx->launches += launches * (long long)K * kernels_per_step(ctx);
  CK(cudaMemcpyAsync(&ctx->hflags[0].status, &ctx->ctl->status, sizeof(int),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hflags[0].steps, &ctx->ctl->steps, sizeof(long long),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hflags[0].t, &ctx->ctl->t, sizeof(double), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const double t_dev = ctx->hflags[0].t;
  const long long steps = ctx->hflags[0].steps;
  if (steps & 1) {  // the last completed step wrote ubuf
    CK(cudaMemcpyAsync(u, ctx->ubuf, (size_t)state_count(ctx) * sizeof(double),
                       cudaMemcpyDeviceToDevice, ctx->stream));
  }
  if ((st = join_out(ctx)) != ADER_OK) return st;
  if (steps_out) *steps_out = steps;
  if (t_out) *t_out = t_dev;
  if (!finished && !(max_steps > 0 && steps >= max_steps))
    return fail(ctx, ADER_ERR_TIMEOUT, "time loop stopped after %lld graph launches", launches);
  return status_from_flags(ctx, ctx->hflags[0].status);
}

ader_status ader_solve(ader_ctx* ctx, double* u, double t_end, int64_t max_steps,
                       int64_t* steps_out, double* t_out) {
  return solve_impl(ctx, u, 0.0, t_end, max_steps, steps_out, t_out);
}

ader_status ader_solve_from(ader_ctx* ctx, double* u, double t0, double t_end, int64_t max_steps,
                            int64_t* steps_out, double* t_out) {
  return solve_impl(ctx, u, t0, t_end, max_steps, steps_out, t_out);
}

ader_status ader_solve_host(ader_ctx* ctx, double* u_host, double t_end, int64_t max_steps,
                            int64_t* steps_out, double* t_out) {
  ader_status st = need_bound(ctx);
  if (st != ADER_OK) return st;
  if (!u_host) return fail(ctx, ADER_ERR_ARG, "null pointer");
  const size_t bytes = (size_t)state_count(ctx) * sizeof(double);
  if ((st = fork_in(ctx)) != ADER_OK) return st;
  CK(cudaMemcpyAsync(ctx->hbuf, u_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  if ((st = join_out(ctx)) != ADER_OK) return st;
  ader_status rs = ader_solve(ctx, ctx->hbuf, t_end, max_steps, steps_out, t_out);
  if (rs != ADER_OK && rs != ADER_ERR_NOT_CONVERGED && rs != ADER_ERR_NONPHYSICAL) return rs;
  if ((st = fork_in(ctx)) != ADER_OK) return st;
  CK(cudaMemcpyAsync(u_host, ctx->hbuf, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if ((st = join_out(ctx)) != ADER_OK) return st;
  return rs;
}

// ---- context-resident state (the mesh-level form of the paper's
// get_cell_local_solution(u_prev) / get_dg_solution(u_prev) of Sec. 1.1, 1.2) ----

ader_status ader_set_state(ader_ctx* ctx, const double* u, int64_t count, int on_device) {
  ader_status st = need_bound(ctx);
  if (st != ADER_OK) return st;
  if (!u) return fail(ctx, ADER_ERR_ARG, "null pointer");
  if (count != state_count(ctx))
    return fail(ctx, ADER_ERR_ARG, "count %lld != ader_state_count %lld", (long long)count,
                (long long)state_count(ctx));
  if ((st = fork_in(ctx)) != ADER_OK) return st;
  CK(cudaMemcpyAsync(ctx->sbuf, u, (size_t)count * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  if (!on_device) CK(cudaStreamSynchronize(ctx->stream));  // the host buffer is free on return
  if ((st = join_out(ctx)) != ADER_OK) return st;
  ctx->state_set = true;
  ctx->state_t = 0.0;
  return ADER_OK;
}

ader_status ader_get_state(ader_ctx* ctx, double* u, int64_t count, int on_device) {
  ader_status st = need_bound(ctx);
  if (st != ADER_OK) return st;
  if (!u) return fail(ctx, ADER_ERR_ARG, "null pointer");
  if (!ctx->state_set) return fail(ctx, ADER_ERR_STATE, "no resident state (call ader_set_state)");
  if (count != state_count(ctx))
    return fail(ctx, ADER_ERR_ARG, "count %lld != ader_state_count %lld", (long long)count,
                (long long)state_count(ctx));
  if ((st = fork_in(ctx)) != ADER_OK) return st;
  CK(cudaMemcpyAsync(u, ctx->sbuf, (size_t)count * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  if (!on_device) CK(cudaStreamSynchronize(ctx->stream));
  return join_out(ctx);
}

ader_status ader_get_state_time(ader_ctx* ctx, double* t) {
  if (!ctx || !t) return ADER_ERR_ARG;
  if (!ctx->state_set) return fail(ctx, ADER_ERR_STATE, "no resident state (call ader_set_state)");
  *t = ctx->state_t;
  return ADER_OK;
}

ader_status ader_get_predictor(ader_ctx* ctx, double dt, double* q, int64_t count) {
  ader_status st = need_bound(ctx);
  if (st != ADER_OK) return st;
  if (!ctx->state_set) return fail(ctx, ADER_ERR_STATE, "no resident state (call ader_set_state)");
  if (count != ader_predictor_count(ctx))
    return fail(ctx, ADER_ERR_ARG, "count %lld != ader_predictor_count %lld", (long long)count,
                (long long)ader_predictor_count(ctx));
  return ader_predict(ctx, ctx->sbuf, dt, q);
}

ader_status ader_state_step(ader_ctx* ctx, double dt, double* dt_out) {
  ader_status st = need_bound(ctx);
  if (st != ADER_OK) return st;
  if (!ctx->state_set) return fail(ctx, ADER_ERR_STATE, "no resident state (call ader_set_state)");
  if (std::isnan(dt)) return fail(ctx, ADER_ERR_ARG, "dt is NaN");
  if (!(dt > 0.0) && (st = ader_compute_dt(ctx, ctx->sbuf, ctx->state_t, 0.0, &dt)) != ADER_OK)
    return st;
  if ((st = fork_in(ctx)) != ADER_OK) return st;
  if ((st = reset_ctl(ctx)) != ADER_OK) return st;
  const StepParams sp = make_step(ctx, kDtFixed, 0, dt, 0.0, 0);
  if ((st = enqueue_step(ctx, ctx->sbuf, ctx->ubuf, sp, 0)) != ADER_OK) return st;
  CK(cudaMemcpyAsync(ctx->sbuf, ctx->ubuf, (size_t)state_count(ctx) * sizeof(double),
                     cudaMemcpyDeviceToDevice, ctx->stream));
  if ((st = join_out(ctx)) != ADER_OK) return st;
  ctx->state_t += dt;
  if (dt_out) *dt_out = dt;
  return ADER_OK;
}

ader_status ader_state_solve(ader_ctx* ctx, double t_end, int64_t max_steps, int64_t* steps_out,
                             double* t_out) {
  ader_status st = need_bound(ctx);
  if (st != ADER_OK) return st;
  if (!ctx->state_set) return fail(ctx, ADER_ERR_STATE, "no resident state (call ader_set_state)");
  if (t_end > 0.0 && !(ctx->state_t < t_end))
    return fail(ctx, ADER_ERR_ARG, "the resident state is already at t = %.17g >= t_end",
                ctx->state_t);
  double t = ctx->state_t;
  int64_t steps = 0;
  const ader_status rs = solve_impl(ctx, ctx->sbuf, ctx->state_t, t_end, max_steps, &steps, &t);
  if (rs == ADER_OK || rs == ADER_ERR_NOT_CONVERGED || rs == ADER_ERR_NONPHYSICAL ||
      rs == ADER_ERR_TIMEOUT)
    ctx->state_t = t;
  if (steps_out) *steps_out = steps;
  if (t_out) *t_out = t;
  return rs;
}

// ---- one shard of a periodic global mesh (multi-GPU decomposition) ----

ader_status ader_init_shard(const ader_mesh* global, int64_t first_cell, int64_t n_local,
                            int degree, int scheme, const ader_options* opt, ader_ctx** out) {
  if (!out) return ADER_ERR_ARG;
  *out = nullptr;
  if (!global || global->n_cells <= 0 || !(global->x1 > global->x0)) return ADER_ERR_ARG;
  if (first_cell < 0 || n_local <= 0 || first_cell + n_local > global->n_cells) return ADER_ERR_ARG;
  ader_options o;
  if (opt) {
    o = *opt;
  } else {
    ader_default_options(&o);
  }
  if (o.bc != ADER_BC_PERIODIC || o.limiter != 0) return ADER_ERR_ARG;
  // halo: DG needs the face neighbour's cell only (its predictor is cell-local);
  // WENO-FV needs the neighbour's reconstruction too, whose stencil reaches N
  // cells further: N + 1 cells
  const int H = scheme == ADER_SCHEME_DG ? 1 : degree + 1;
  const int64_t min_local = scheme == ADER_SCHEME_DG ? 1 : degree;
  if (n_local < min_local) return ADER_ERR_ARG;
  const double dx = (global->x1 - global->x0) / (double)global->n_cells;
  ader_mesh m{n_local + 2 * H, global->x0 + dx * (double)(first_cell - H), 0.0};
  m.x1 = m.x0 + dx * (double)m.n_cells;
  ader_ctx* c = nullptr;
  const ader_status st = ader_init(&m, degree, scheme, &o, &c);
  if (st != ADER_OK) return st;
  c->dx = dx;  // the global mesh's spacing, bit for bit
  c->shard_first = first_cell;
  c->shard_local = n_local;
  c->shard_global = global->n_cells;
  c->shard_halo = H;
  *out = c;
  return ADER_OK;
}

ader_status ader_shard_info(const ader_ctx* ctx, ader_shard* out) {
  if (!ctx || !out) return ADER_ERR_ARG;
  if (ctx->shard_first < 0) return ADER_ERR_ARG;
  out->first_cell = ctx->shard_first;
  out->n_local = ctx->shard_local;
  out->n_global = ctx->shard_global;
  out->halo_cells = ctx->shard_halo;
  out->values_per_cell = state_count(ctx) / ctx->mesh.n_cells;
  return ADER_OK;
}

ader_status ader_get_troubled(ader_ctx* ctx, int32_t* flags, int64_t count) {
  ader_status st = need_bound(ctx);
  if (st != ADER_OK) return st;
  if (ctx->dims != 1) return fail(ctx, ADER_ERR_ARG, "the limiter is 1D only");
  if (!ctx->opt.limiter) return fail(ctx, ADER_ERR_ARG, "troubled flags need the limiter");
  if (!flags || count != ctx->mesh.n_cells) return fail(ctx, ADER_ERR_ARG, "flags / count");
  if ((st = fork_in(ctx)) != ADER_OK) return st;
  CK(cudaMemcpyAsync(flags, ctx->lim_flag, (size_t)count * sizeof(int32_t),
                     cudaMemcpyDeviceToDevice, ctx->stream));
  return join_out(ctx);
}

ader_status ader_get_stats(ader_ctx* ctx, ader_stats* out) {
  ader_status st = need_bound(ctx);
  if (st != ADER_OK) return st;
  if (!out) return ADER_ERR_ARG;
  DevCtl h{};
  if ((st = fork_in(ctx)) != ADER_OK) return st;
  CK(cudaMemcpyAsync(&h, ctx->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if ((st = join_out(ctx)) != ADER_OK) return st;
  out->steps = h.steps;
  out->t = h.t;
  out->cells = h.iter_cells;
  out->max_iters = h.iter_max;
  out->mean_iters = h.iter_cells > 0 ? (double)h.iter_sum / (double)h.iter_cells : 0.0;
  out->status = h.status & kStNonPhysical ? ADER_ERR_NONPHYSICAL
                : h.status & kStNotConverged ? ADER_ERR_NOT_CONVERGED
                                             : ADER_OK;
  out->profiled_steps = ctx->prof_steps;
  out->weno_ms = ctx->prof_ms[0];
  out->predict_ms = ctx->prof_ms[1];
  out->face_ms = ctx->prof_ms[2];
  out->kernel_launches = ctx->launches;
  out->troubled_cells = (int64_t)h.troubled;
  return ADER_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// ader_step_noalloc: one step whose scratch is a static device array.
// For callers that cannot allocate device memory and so cannot bind a workspace.
// ---------------------------------------------------------------------------

#include <mutex>

namespace {

constexpr size_t kNoallocBytes = ADER_NOALLOC_SCRATCH_BYTES;
constexpr size_t kNoallocCtlBytes = 256;  // DevCtl, rounded up
static_assert(sizeof(DevCtl) <= kNoallocCtlBytes, "control block does not fit");

// The scratch itself: device memory that exists once per GPU for the life of the
// process.  Host code must not use the symbol as an address (it names a host-side
// stand-in); the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};
bool g_noalloc_degree_ready[kMaxDevices][kMaxDeg + 1] = {};

// Bytes of the static scratch one step of this context needs: the control
// block, the traces (DG: with the volume term) and, for WENO-FV, the
// reconstruction.
size_t noalloc_need(const ader_ctx* ctx, long long cells) {
  const size_t per = (size_t)(ctx->scheme == ADER_SCHEME_DG ? 3 : 2) * ctx->M * ctx->n;
  const size_t trace_bytes = (size_t)cells * per * sizeof(double);
  const size_t wrec_bytes =
      ctx->scheme == ADER_SCHEME_WENO_FV ? (size_t)cells * ctx->n * kM * sizeof(double) : 0;
  return kNoallocCtlBytes + align_up(trace_bytes) + wrec_bytes;
}

// The largest mesh noalloc_need() accepts, from the same expression (bisection).
long long noalloc_max_cells(const ader_ctx* ctx) {
  long long lo = 0, hi = (long long)(kNoallocBytes / sizeof(double)) + 1;
  while (hi - lo > 1) {
    const long long mid = lo + (hi - lo) / 2;
    if (noalloc_need(ctx, mid) <= kNoallocBytes) lo = mid; else hi = mid;
  }
  return lo;
}

// Per-device set-up, with that device current: look up the scratch address and
// raise the predictor's dynamic shared-memory limit for this degree.
ader_status noalloc_setup(ader_ctx* ctx, int N, void** out) {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(ctx, ADER_ERR_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(ctx, ADER_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                  cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
  }
  if (!g_noalloc_degree_ready[dev][N]) {
    CK(dispatch_prepare(N));
    g_noalloc_degree_ready[dev][N] = true;
  }
  *out = g_noalloc_ptr[dev];
  return ADER_OK;
}

}  // namespace

extern "C" ader_status ader_step_noalloc(ader_ctx* ctx, const double* u, double* u_new, double dt,
                                         void* stream) {
  if (!ctx) return ADER_ERR_ARG;
  if (!u || !u_new) return fail(ctx, ADER_ERR_ARG, "null pointer");
  if (u == u_new) return fail(ctx, ADER_ERR_ARG, "u and u_new must not alias");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, ADER_ERR_ARG, "ader_step_noalloc needs dt > 0");
  if (ctx->dims != 1) return fail(ctx, ADER_ERR_ARG, "ader_step_noalloc is 1D only");
  if (ctx->opt.limiter)
    return fail(ctx, ADER_ERR_ARG, "the limiter keeps per-cell data in the bound workspace");
  const size_t trace_bytes = trace_doubles(ctx) * sizeof(double);
  const size_t need = noalloc_need(ctx, ctx->mesh.n_cells);
  if (need > kNoallocBytes) {
    return fail(ctx, ADER_ERR_ARG,
                "mesh of %lld cells needs %zu bytes of scratch; the static scratch holds %zu "
                "bytes (at most %lld cells for this scheme at N = %d)",
                (long long)ctx->mesh.n_cells, need, kNoallocBytes,
                (long long)noalloc_max_cells(ctx), ctx->N);
  }
  void* base = nullptr;
  ader_status st = noalloc_setup(ctx, ctx->N, &base);
  if (st != ADER_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* p = static_cast<char*>(base);
  DevCtl* ctl = reinterpret_cast<DevCtl*>(p);
  double* trace = reinterpret_cast<double*>(p + kNoallocCtlBytes);
  double* wrec = reinterpret_cast<double*>(p + kNoallocCtlBytes + align_up(trace_bytes));
  // the control block (statistics, status) must start at zero; the traces and
  // the reconstruction are written in full before they are read
  CK(cudaMemsetAsync(ctl, 0, sizeof(DevCtl), s));
  StepParams sp = make_step(ctx, kDtFixed, 0, dt, 0.0, 0);
  sp.ctl = ctl;
  const double* nodal = u;
  if (ctx->scheme == ADER_SCHEME_WENO_FV) {
    WenoParams w{};
    w.v = u;
    w.w = wrec;
    w.ncells = ctx->mesh.n_cells;
    w.wo = ctx->basis.weno;
    CK(do_weno(ctx->N, w, s));
    nodal = wrec;
  }
  PredictParams pp = make_predict(ctx, nodal, sp);
  pp.trace = trace;
  CK(do_predict(ctx->N, pp, s));
  // lambda_max of u_new is reduced into the static control block only so that a
  // non-physical result raises the status bit read below; u_new is unchanged by it
  FaceParams f = make_face(ctx, u, u_new, sp, 1);
  f.trace = trace;
  CK(do_face(ctx->N, f, s));
  // the sticky status bits (Picard cap, non-physical state): read back through a
  // host variable on the stack, after the kernels, then the stream is drained
  int flags = 0;
  CK(cudaMemcpyAsync(&flags, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return status_from_flags(ctx, flags);
}

// ---------------------------------------------------------------------------
// autotuning of launch shapes
// ---------------------------------------------------------------------------

extern "C" ader_status ader_get_tuning(const ader_ctx* ctx, ader_tuning* out) {
  if (!ctx || !out) return ADER_ERR_ARG;
  *out = ctx->tune;
  if (out->graph_steps <= 0) out->graph_steps = graph_steps_for(ctx->mesh.n_cells);
  return ADER_OK;
}

extern "C" ader_status ader_set_tuning(ader_ctx* ctx, const ader_tuning* in) {
  if (!ctx || !in) return ADER_ERR_ARG;
  if (!valid_cpb(ctx->N, in->predict_cells_per_block) ||
      (in->face_cells_per_block != 32 && in->face_cells_per_block != 64) || in->graph_steps < 2 ||
      in->graph_steps > ader_ctx::kMaxGraphSteps || (in->graph_steps & 1))
    return fail(ctx, ADER_ERR_ARG, "invalid tuning");
  ctx->tune = *in;
  if (ctx->gexec) {
    cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
  }
  return ADER_OK;
}

extern "C" ader_status ader_autotune(ader_ctx* ctx, const double* u, int reps, ader_tuning* out) {
  ader_status st = need_bound(ctx);
  if (st != ADER_OK) return st;
  if (ctx->dims != 1) return fail(ctx, ADER_ERR_ARG, "ader_autotune tunes the 1D kernels");
  if (!u) return fail(ctx, ADER_ERR_ARG, "null pointer");
  if (reps < 1) reps = 3;
  double dt = 0.0;
  if ((st = ader_compute_dt(ctx, u, 0.0, 0.0, &dt)) != ADER_OK) return st;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto timed = [&](auto&& launch, double* ms_out) -> ader_status {
    ader_status s2 = launch();  // warm-up
    if (s2 != ADER_OK) return s2;
    CK(cudaEventRecord(e0, ctx->stream));
    for (int r = 0; r < reps; ++r)
      if ((s2 = launch()) != ADER_OK) return s2;
    CK(cudaEventRecord(e1, ctx->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    *ms_out = ms / reps;
    return ADER_OK;
  };
  const ader_tuning saved = ctx->tune;
  ader_tuning best = saved;
  if ((st = fork_in(ctx)) != ADER_OK) return st;
  if ((st = reset_ctl(ctx)) != ADER_OK) return st;
  const StepParams sp = make_step(ctx, kDtFixed, 0, dt, 0.0, 0);
  const double* nodal = u;
  if (ctx->scheme == ADER_SCHEME_WENO_FV) {
    WenoParams w{};
    w.v = u;
    w.w = ctx->wrec;
    w.ncells = ctx->mesh.n_cells;
    w.wo = ctx->basis.weno;
    CK(do_weno(ctx->N, w, ctx->stream));
    nodal = ctx->wrec;
  }
  // Tile shapes are timed in interleaved rounds (every shape once per round)
  // and each keeps its fastest round: shapes a percent apart are then told
  // apart reliably, and slow drift (clocks, caches) hits every shape alike.
  constexpr int kRounds = 3;
  // predictor tile shapes
  const int cpbs[3] = {16, 32, 64};
  double pms[3] = {1e300, 1e300, 1e300};
  for (int round = 0; round < kRounds && st == ADER_OK; ++round) {
    for (int i = 0; i < 3 && st == ADER_OK; ++i) {
      if (!valid_cpb(ctx->N, cpbs[i])) continue;
      ctx->tune.predict_cells_per_block = cpbs[i];
      double ms;
      st = timed([&]() -> ader_status {
        PredictParams p = make_predict(ctx, nodal, sp);
        CK(do_predict(ctx->N, p, ctx->stream));
        return ADER_OK;
      }, &ms);
      if (st == ADER_OK && ms < pms[i]) pms[i] = ms;
    }
  }
  double best_ms = 1e300;
  for (int i = 0; i < 3; ++i) {
    if (pms[i] < best_ms) {
      best_ms = pms[i];
      best.predict_cells_per_block = cpbs[i];
      best.predict_ms = pms[i];
    }
  }
  // interface/update tile shapes (the traces of the last predictor run are valid)
  const int cpfs[2] = {32, 64};
  double fms[2] = {1e300, 1e300};
  for (int round = 0; round < kRounds && st == ADER_OK; ++round) {
    for (int i = 0; i < 2 && st == ADER_OK; ++i) {
      ctx->tune.face_cells_per_block = cpfs[i];
      double ms;
      st = timed([&]() -> ader_status {
        FaceParams f = make_face(ctx, u, ctx->ubuf, sp, 1);
        CK(do_face(ctx->N, f, ctx->stream));
        return ADER_OK;
      }, &ms);
      if (st == ADER_OK && ms < fms[i]) fms[i] = ms;
    }
  }
  best_ms = 1e300;
  for (int i = 0; i < 2; ++i) {
    if (fms[i] < best_ms) {
      best_ms = fms[i];
      best.face_cells_per_block = cpfs[i];
      best.face_ms = fms[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != ADER_OK) {
    ctx->tune = saved;
    return st;
  }
  if ((st = join_out(ctx)) != ADER_OK) return st;
  // graph length: solve 64 steps on a workspace copy of u for every candidate
  ctx->tune = best;
  const size_t bytes = (size_t)state_count(ctx) * sizeof(double);
  double best_solve = 1e300;
  const int prof_saved = ctx->opt.profile;
  ctx->opt.profile = 0;
  for (int K : {4, 8, 16, 32, 64}) {
    if (ctx->shard_first >= 0) break;  // a shard has no device-resident time loop
    ctx->tune.graph_steps = K;
    if (ctx->gexec) {
      cudaGraphExecDestroy(ctx->gexec);
      ctx->gexec = nullptr;
    }
    double total = 0.0;
    for (int r = 0; r < 2; ++r) {  // first run captures the graph
      if ((st = fork_in(ctx)) != ADER_OK) break;
      CK(cudaMemcpyAsync(ctx->hbuf, u, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      const auto t0 = std::chrono::steady_clock::now();
      int64_t steps = 0;
      st = ader_solve(ctx, ctx->hbuf, 0.0, 64, &steps, nullptr);
      const double ms =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (st != ADER_OK && st != ADER_ERR_NOT_CONVERGED) break;
      st = ADER_OK;
      if (r == 1) total = ms / 64.0;
    }
    if (st != ADER_OK) break;
    if (total < best_solve) {
      best_solve = total;
      best.graph_steps = K;
      best.solve_ms_per_step = total;
    }
  }
  ctx->opt.profile = prof_saved;
  if (ctx->gexec) {
    cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
  }
  if (st != ADER_OK) {
    ctx->tune = saved;
    return st;
  }
  ctx->tune = best;
  if (out) *out = best;
  return ADER_OK;
}
