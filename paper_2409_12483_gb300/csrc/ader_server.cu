// ader_server.cu -- continuous batching of independent ADER-DG solves on one GPU
// (the serving API of include/ader.h).  Host side: a first-fit sub-allocator over
// the caller's device pool, FIFO admission by slot and memory, per-degree work
// lists of (solve, tile) items, CUDA-graph rounds of ticks, retirement.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <vector>

#include "../../include/ader.h"
#include "ader_dispatch.h"
#include "ader_launch.h"
#include "ader_ops.h"

using namespace ader;

namespace {

constexpr size_t kAl = 256;
size_t al(size_t x) { return (x + kAl - 1) / kAl * kAl; }

// First-fit free list over [0, size) in 256-byte units, with coalescing.
class PoolAlloc {
 public:
  void init(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = al(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = al(bytes);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
 private:
  std::map<size_t, size_t> free_;
};

struct Req {
  uint64_t id = 0;
  int degree = 0;
  int64_t ncells = 0;
  double x0 = 0, x1 = 1, t_end = 0, arrival = 0;
  std::vector<double> u0, result;
  int state = ADER_REQ_QUEUED, status = ADER_OK;
  int64_t steps = 0;
  double t = 0, admitted = 0, finished = 0;
  int slot = -1;
  size_t off = 0, bytes = 0;
};

struct Slot {
  Req* req = nullptr;
  double* u[2] = {nullptr, nullptr};
  double* trace = nullptr;
  long long steps_seen = 0;
};

size_t state_bytes(int degree, int64_t ncells) {
  return (size_t)ncells * (degree + 1) * kM * sizeof(double);
}

size_t request_bytes(int degree, int64_t ncells) {
  return 2 * al(state_bytes(degree, ncells)) + al((size_t)ncells * 9 * (degree + 1) * sizeof(double));
}

}  // namespace

struct ader_server {
  ader_server_opts opt{};
  char* pool = nullptr;
  cudaStream_t user_stream = nullptr;  // the caller's stream (may be the legacy default)
  cudaStream_t stream = nullptr;       // private non-blocking stream: all work and capture
  cudaEvent_t ev_fork = nullptr;
  // one capture branch per degree: the solves of different degrees share no
  // data, so their tick chains run side by side in the round's graph
  cudaStream_t deg_stream[kMaxDeg + 1] = {};
  cudaEvent_t ev_branch = nullptr;
  cudaEvent_t ev_join[kMaxDeg + 1] = {};
  Basis basis[kMaxDeg + 1];
  bool have_basis[kMaxDeg + 1] = {};
  DevCtl* ctl_dev = nullptr;
  SlotDesc* desc_dev = nullptr;
  TileItem* items_dev = nullptr;
  size_t items_cap = 0;
  size_t data_base = 0;
  PoolAlloc alloc;
  std::vector<Slot> slots;
  std::vector<SlotDesc> desc_host;
  DevCtl* ctl_host = nullptr;  // pinned mirror of ctl_dev
  std::vector<Req*> queue;     // sorted by (arrival, id)
  std::map<uint64_t, std::unique_ptr<Req>> reqs;
  uint64_t next_id = 1;
  struct DegList {
    long long pred_off = 0, pred_n = 0, face_off = 0, face_n = 0;
  } lists[kMaxDeg + 1];
  bool dirty = true;
  cudaGraphExec_t gexec = nullptr;
  long long ticks = 0, rounds = 0, launches = 0, cell_updates = 0, graph_launches_per_round = 0;
  char err[512] = {0};
};

namespace {

ader_status sfail(ader_server* s, ader_status st, const char* fmt, ...) {
  if (s) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(s->err, sizeof(s->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

#define SCK(call)                                                                           \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return sfail(srv, ADER_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
  } while (0)

ader_status ensure_basis(ader_server* srv, int N) {
  if (srv->have_basis[N]) return ADER_OK;
  if (build_basis(N, false, &srv->basis[N]) != 0)
    return sfail(srv, ADER_ERR_ARG, "operator construction failed for N = %d", N);
  SCK(dispatch_prepare(N));
  srv->have_basis[N] = true;
  return ADER_OK;
}

PredictParams server_predict_params(const ader_server* srv, int N) {
  PredictParams p{};
  p.out_mode = kOutTrace;
  p.dg = 1;
  p.prec = srv->opt.precision;
  p.sweeps = srv->opt.fp64_sweeps;
  p.max_iter = 4 * (N + 1) + 8;
  p.fixed_iter = 0;
  p.tol = srv->opt.picard_tol;
  p.tol32 = 1e-6f;
  p.gamma = srv->opt.gamma;
  p.gm1 = srv->opt.gamma - 1.0;
  p.gamf = (float)p.gamma;
  p.gm1f = (float)p.gm1;
  p.c1f = (float)(0.5 * (3.0 - p.gamma));
  p.c2f = (float)(0.5 * p.gm1);
  p.tolf = (float)p.tol;
  p.ops = srv->basis[N].d;
  p.opf = srv->basis[N].f;
  return p;
}

FaceParams server_face_params(const ader_server* srv, int N) {
  FaceParams f{};
  f.dg = 1;
  f.want_lambda = 1;
  f.Ns = srv->basis[N].Ns;
  f.gamma = srv->opt.gamma;
  f.gm1 = srv->opt.gamma - 1.0;
  f.ops = srv->basis[N].d;
  return f;
}

ader_status admit(ader_server* srv, Req* r, int slot_id, double now) {
  Slot& sl = srv->slots[slot_id];
  char* base = srv->pool + srv->data_base + r->off;
  const size_t sb = al(state_bytes(r->degree, r->ncells));
  sl.req = r;
  sl.u[0] = reinterpret_cast<double*>(base);
  sl.u[1] = reinterpret_cast<double*>(base + sb);
  sl.trace = reinterpret_cast<double*>(base + 2 * sb);
  sl.steps_seen = 0;
  SCK(cudaMemcpyAsync(sl.u[0], r->u0.data(), state_bytes(r->degree, r->ncells),
                      cudaMemcpyHostToDevice, srv->stream));
  DevCtl* ctl = srv->ctl_dev + slot_id;
  SCK(cudaMemsetAsync(ctl, 0, sizeof(DevCtl), srv->stream));
  const Basis& b = srv->basis[r->degree];
  CflParams cp{};
  cp.u = sl.u[0];
  cp.ncells = r->ncells;
  cp.vars = kM;
  cp.dg = 1;
  cp.slot = 0;
  cp.Ns = b.Ns;
  cp.gamma = srv->opt.gamma;
  cp.gm1 = srv->opt.gamma - 1.0;
  cp.ctl = ctl;
  cp.ops = b.d;
  SCK(do_cfl(r->degree, cp, srv->stream));
  srv->launches += 1;
  const double dx = (r->x1 - r->x0) / (double)r->ncells;
  SlotDesc d{};
  d.u[0] = sl.u[0];
  d.u[1] = sl.u[1];
  d.trace = sl.trace;
  d.ncells = r->ncells;
  d.par0 = 0;  // rounds start at even ticks, so the first step of every solve has parity 0
  d.degree = r->degree;
  d.sp.mode = kDtSolve;
  d.sp.par = 0;
  d.sp.t_end = r->t_end;
  d.sp.max_steps = 0;
  d.sp.cfl_factor = srv->opt.cfl * dx / (double)(2 * r->degree + 1);
  d.sp.inv_dx = 1.0 / dx;
  d.sp.ctl = ctl;
  srv->desc_host[slot_id] = d;
  r->u0.clear();
  r->u0.shrink_to_fit();
  r->slot = slot_id;
  r->state = ADER_REQ_RUNNING;
  r->admitted = now;
  srv->dirty = true;
  return ADER_OK;
}

ader_status rebuild(ader_server* srv) {
  std::vector<TileItem> items;
  for (int N = 0; N <= kMaxDeg; ++N) {
    auto& L = srv->lists[N];
    L.pred_off = (long long)items.size();
    for (size_t s = 0; s < srv->slots.size(); ++s) {
      const Req* r = srv->slots[s].req;
      if (!r || r->degree != N) continue;
      const long long T = server_pred_cells(N);
      for (long long t = 0; t < (r->ncells + T - 1) / T; ++t) items.push_back({(int)s, (int)t});
    }
    L.pred_n = (long long)items.size() - L.pred_off;
    L.face_off = (long long)items.size();
    for (size_t s = 0; s < srv->slots.size(); ++s) {
      const Req* r = srv->slots[s].req;
      if (!r || r->degree != N) continue;
      const long long T = kServerFaceCells;
      for (long long t = 0; t < (r->ncells + T - 1) / T; ++t) items.push_back({(int)s, (int)t});
    }
    L.face_n = (long long)items.size() - L.face_off;
  }
  if (items.size() > srv->items_cap)
    return sfail(srv, ADER_ERR_NOMEM, "work list of %zu tiles exceeds its capacity %zu",
                 items.size(), srv->items_cap);
  if (!items.empty())
    SCK(cudaMemcpyAsync(srv->items_dev, items.data(), items.size() * sizeof(TileItem),
                        cudaMemcpyHostToDevice, srv->stream));
  SCK(cudaMemcpyAsync(srv->desc_dev, srv->desc_host.data(), srv->desc_host.size() * sizeof(SlotDesc),
                      cudaMemcpyHostToDevice, srv->stream));
  srv->graph_launches_per_round = 0;
  if (items.empty()) {
    if (srv->gexec) cudaGraphExecDestroy(srv->gexec);
    srv->gexec = nullptr;
    srv->dirty = false;
    return ADER_OK;
  }
  // one round: ticks_per_round ticks; each tick = the batched predictor, then the
  // batched update, of every degree present.  Each degree's chain of ticks is
  // captured on its own stream (a branch of the graph), so a tick takes the time
  // of the slowest degree rather than the sum over degrees.
  cudaGraph_t g;
  SCK(cudaStreamBeginCapture(srv->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t ce = cudaEventRecord(srv->ev_branch, srv->stream);
  long long per_round = 0;
  for (int N = 0; N <= kMaxDeg; ++N) {
    const auto& L = srv->lists[N];
    if (!L.pred_n) continue;
    cudaStream_t bs = srv->deg_stream[N];
    // fork and join even after an error, so that the capture ends with every
    // branch joined
    cudaError_t fe = cudaStreamWaitEvent(bs, srv->ev_branch, 0);
    if (fe != cudaSuccess) {
      if (ce == cudaSuccess) ce = fe;
      continue;  // this stream did not join the capture
    }
    for (int j = 0; j < srv->opt.ticks_per_round && ce == cudaSuccess; ++j) {
      MultiArgs mp{srv->desc_dev, srv->items_dev + L.pred_off, L.pred_n, j & 1};
      const int gp = (int)std::min<long long>(L.pred_n, 152LL * 4);
      ce = do_predict_multi(N, server_predict_params(srv, N), mp, gp, bs);
      ++per_round;
      if (ce != cudaSuccess) break;
      MultiArgs mf{srv->desc_dev, srv->items_dev + L.face_off, L.face_n, j & 1};
      const int gf = (int)std::min<long long>(L.face_n, 152LL * 8);
      ce = do_face_multi(N, server_face_params(srv, N), mf, gf, bs);
      ++per_round;
    }
    cudaError_t je = cudaEventRecord(srv->ev_join[N], bs);
    if (je == cudaSuccess) je = cudaStreamWaitEvent(srv->stream, srv->ev_join[N], 0);
    if (ce == cudaSuccess) ce = je;
  }
  cudaError_t ee = cudaStreamEndCapture(srv->stream, &g);
  if (ce != cudaSuccess || ee != cudaSuccess) {
    if (ee == cudaSuccess) cudaGraphDestroy(g);
    if (srv->gexec) cudaGraphExecDestroy(srv->gexec);
    srv->gexec = nullptr;
    if (ce != cudaSuccess)
      return sfail(srv, ADER_ERR_CUDA, "batched launch failed during capture: %s",
                   cudaGetErrorString(ce));
    return sfail(srv, ADER_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ee));
  }
  // Most rounds change only the work lists' lengths and offsets (kernel
  // parameters and grid sizes) of the same degrees: update the executable graph
  // in place, and instantiate afresh only when the graph's shape changed.
  if (srv->gexec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(srv->gexec, g, &info) != cudaSuccess) {
      (void)cudaGetLastError();  // the failed update leaves no error behind
      cudaGraphExecDestroy(srv->gexec);
      srv->gexec = nullptr;
    }
  }
  ee = srv->gexec ? cudaSuccess : cudaGraphInstantiate(&srv->gexec, g, 0);
  cudaGraphDestroy(g);
  if (ee != cudaSuccess)
    return sfail(srv, ADER_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ee));
  srv->graph_launches_per_round = per_round;
  srv->dirty = false;
  return ADER_OK;
}

// destroys the server's graph, pinned mirror, streams and events (any subset
// that exists)
void release_cuda(ader_server* s) {
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  s->gexec = nullptr;
  if (s->ctl_host) cudaFreeHost(s->ctl_host);
  s->ctl_host = nullptr;
  for (int N = 0; N <= kMaxDeg; ++N) {
    if (s->deg_stream[N]) cudaStreamDestroy(s->deg_stream[N]);
    if (s->ev_join[N]) cudaEventDestroy(s->ev_join[N]);
    s->deg_stream[N] = nullptr;
    s->ev_join[N] = nullptr;
  }
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_branch) cudaEventDestroy(s->ev_branch);
  s->stream = nullptr;
  s->ev_fork = s->ev_branch = nullptr;
}

}  // namespace

extern "C" {

ader_status ader_server_default_options(ader_server_opts* o) {
  if (!o) return ADER_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  o->max_slots = 256;
  o->ticks_per_round = 16;
  o->precision = ADER_PREC_FP64;
  o->fp64_sweeps = 1;
  o->gamma = 1.4;
  o->cfl = 0.4;
  o->picard_tol = 1e-13;
  return ADER_OK;
}

size_t ader_server_request_bytes(int degree, int64_t n_cells) {
  if (degree < 0 || degree > kMaxDeg || n_cells <= 0) return 0;
  return request_bytes(degree, n_cells);
}

ader_status ader_server_create(const ader_server_opts* opt, ader_server** out) {
  if (!opt || !out) return ADER_ERR_ARG;
  *out = nullptr;
  if (!opt->pool_dev || opt->max_slots < 1 || opt->max_slots > 65536 || opt->ticks_per_round < 2 ||
      (opt->ticks_per_round & 1) || opt->ticks_per_round > 4096 || !(opt->gamma > 1.0) ||
      !(opt->cfl > 0.0) ||
      (opt->precision != ADER_PREC_FP64 && opt->precision != ADER_PREC_FP32_PREDICTOR &&
       opt->precision != ADER_PREC_FF_PREDICTOR && opt->precision != ADER_PREC_FP32_FF_SWEEPS &&
       opt->precision != ADER_PREC_FP32_INCREMENT) ||
      ((opt->precision == ADER_PREC_FP32_PREDICTOR || opt->precision == ADER_PREC_FP32_FF_SWEEPS) &&
       opt->fp64_sweeps < 1) ||
      reinterpret_cast<uintptr_t>(opt->pool_dev) % kAl)
    return ADER_ERR_ARG;
  std::unique_ptr<ader_server> s(new (std::nothrow) ader_server());
  if (!s) return ADER_ERR_NOMEM;
  s->opt = *opt;
  if (!(s->opt.picard_tol > 0.0)) s->opt.picard_tol = 1e-13;
  s->pool = static_cast<char*>(opt->pool_dev);
  s->user_stream = static_cast<cudaStream_t>(opt->stream);
  // the server's CUDA objects are released by release_cuda on every exit path
  struct Guard {
    ader_server* s;
    ~Guard() {
      if (s) release_cuda(s);
    }
  } guard{s.get()};
  bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&s->ev_branch, cudaEventDisableTiming) == cudaSuccess;
  for (int N = 0; ok && N <= kMaxDeg; ++N)
    ok = cudaStreamCreateWithFlags(&s->deg_stream[N], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->ev_join[N], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) return ADER_ERR_CUDA;
  const size_t ctl_bytes = al((size_t)opt->max_slots * sizeof(DevCtl));
  const size_t desc_bytes = al((size_t)opt->max_slots * sizeof(SlotDesc));
  // at most 1/16 + 1/32 tiles per cell and >= 120 pool bytes per cell
  s->items_cap = std::max<size_t>(4096, opt->pool_bytes / 1024);
  const size_t item_bytes = al(s->items_cap * sizeof(TileItem));
  if (opt->pool_bytes < ctl_bytes + desc_bytes + item_bytes + kAl) return ADER_ERR_NOMEM;
  s->ctl_dev = reinterpret_cast<DevCtl*>(s->pool);
  s->desc_dev = reinterpret_cast<SlotDesc*>(s->pool + ctl_bytes);
  s->items_dev = reinterpret_cast<TileItem*>(s->pool + ctl_bytes + desc_bytes);
  s->data_base = ctl_bytes + desc_bytes + item_bytes;
  s->alloc.init(opt->pool_bytes - s->data_base);
  s->slots.assign(opt->max_slots, Slot{});
  s->desc_host.assign(opt->max_slots, SlotDesc{});
  if (cudaMallocHost(&s->ctl_host, (size_t)opt->max_slots * sizeof(DevCtl)) != cudaSuccess) {
    s->ctl_host = nullptr;
    return ADER_ERR_CUDA;
  }
  std::memset(s->ctl_host, 0, (size_t)opt->max_slots * sizeof(DevCtl));
  guard.s = nullptr;
  *out = s.release();
  return ADER_OK;
}

void ader_server_destroy(ader_server* s) {
  if (!s) return;
  release_cuda(s);
  delete s;
}

const char* ader_server_last_error(const ader_server* s) { return s ? s->err : "null server"; }

ader_status ader_server_submit(ader_server* srv, const ader_request* rq, uint64_t* id_out) {
  if (!srv || !rq || !rq->u0_host) return ADER_ERR_ARG;
  if (rq->degree < 0 || rq->degree > kMaxDeg || rq->n_cells <= 0 || !(rq->x1 > rq->x0) ||
      !(rq->t_end > 0.0) || !std::isfinite(rq->t_end) || std::isnan(rq->arrival))
    return sfail(srv, ADER_ERR_ARG, "invalid request");
  if (rq->n_cells > (int64_t)1 << 30) return sfail(srv, ADER_ERR_ARG, "mesh too large");
  const size_t need = request_bytes(rq->degree, rq->n_cells);
  if (need > srv->opt.pool_bytes - srv->data_base)
    return sfail(srv, ADER_ERR_NOMEM, "request needs %zu bytes; the pool's data region is %zu",
                 need, srv->opt.pool_bytes - srv->data_base);
  ader_status st = ensure_basis(srv, rq->degree);
  if (st != ADER_OK) return st;
  auto r = std::make_unique<Req>();
  r->id = srv->next_id++;
  r->degree = rq->degree;
  r->ncells = rq->n_cells;
  r->x0 = rq->x0;
  r->x1 = rq->x1;
  r->t_end = rq->t_end;
  r->arrival = rq->arrival;
  r->bytes = need;
  const size_t cnt = (size_t)rq->n_cells * (rq->degree + 1) * kM;
  r->u0.assign(rq->u0_host, rq->u0_host + cnt);
  Req* raw = r.get();
  auto pos = std::upper_bound(srv->queue.begin(), srv->queue.end(), raw, [](Req* a, Req* b) {
    return a->arrival < b->arrival || (a->arrival == b->arrival && a->id < b->id);
  });
  srv->queue.insert(pos, raw);
  if (id_out) *id_out = raw->id;
  srv->reqs.emplace(raw->id, std::move(r));
  return ADER_OK;
}

ader_status ader_server_progress(ader_server* srv, double now, int* running, int* queued) {
  if (!srv) return ADER_ERR_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  auto clock = [&]() {
    return now + std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  };
  ader_status st;
  // order after the caller's pending work on its stream (e.g. pool initialisation)
  SCK(cudaEventRecord(srv->ev_fork, srv->user_stream));
  SCK(cudaStreamWaitEvent(srv->stream, srv->ev_fork, 0));
  // admission: FIFO by arrival, while a slot and pool memory are free
  while (!srv->queue.empty() && srv->queue.front()->arrival <= clock()) {
    Req* r = srv->queue.front();
    int slot = -1;
    for (size_t i = 0; i < srv->slots.size(); ++i)
      if (!srv->slots[i].req) {
        slot = (int)i;
        break;
      }
    if (slot < 0) break;
    size_t off;
    if (!srv->alloc.alloc(r->bytes, &off)) break;  // wait for memory (keeps FIFO order)
    r->off = off;
    srv->queue.erase(srv->queue.begin());
    if ((st = admit(srv, r, slot, clock())) != ADER_OK) return st;
  }
  if (srv->dirty && (st = rebuild(srv)) != ADER_OK) return st;
  int nrun = 0;
  for (auto& sl : srv->slots) nrun += sl.req != nullptr;
  if (nrun > 0 && srv->gexec) {
    SCK(cudaGraphLaunch(srv->gexec, srv->stream));
    srv->ticks += srv->opt.ticks_per_round;
    srv->rounds += 1;
    srv->launches += srv->graph_launches_per_round;
    SCK(cudaMemcpyAsync(srv->ctl_host, srv->ctl_dev, srv->slots.size() * sizeof(DevCtl),
                        cudaMemcpyDeviceToHost, srv->stream));
    SCK(cudaStreamSynchronize(srv->stream));
    // retire finished solves
    std::vector<Req*> retired;
    for (size_t i = 0; i < srv->slots.size(); ++i) {
      Slot& sl = srv->slots[i];
      if (!sl.req) continue;
      const DevCtl& c = srv->ctl_host[i];
      srv->cell_updates += (c.steps - sl.steps_seen) * sl.req->ncells;
      sl.steps_seen = c.steps;
      if (!(c.done || (c.status & kStNonPhysical))) continue;
      Req* r = sl.req;
      r->steps = c.steps;
      r->t = c.t;
      r->status = (c.status & kStNonPhysical)    ? ADER_ERR_NONPHYSICAL
                  : (c.status & kStNotConverged) ? ADER_ERR_NOT_CONVERGED
                                                 : ADER_OK;
      r->result.resize((size_t)r->ncells * (r->degree + 1) * kM);
      SCK(cudaMemcpyAsync(r->result.data(), sl.u[c.steps & 1], state_bytes(r->degree, r->ncells),
                          cudaMemcpyDeviceToHost, srv->stream));
      retired.push_back(r);
      srv->alloc.release(r->off, r->bytes);
      sl = Slot{};
      srv->desc_host[i] = SlotDesc{};
      srv->dirty = true;
    }
    if (!retired.empty()) {
      SCK(cudaStreamSynchronize(srv->stream));
      const double tf = clock();
      for (Req* r : retired) {
        r->state = (r->status == ADER_ERR_NONPHYSICAL) ? ADER_REQ_FAILED : ADER_REQ_DONE;
        r->finished = tf;
        r->slot = -1;
      }
    }
  }
  if (running) {
    *running = 0;
    for (auto& sl : srv->slots) *running += sl.req != nullptr;
  }
  if (queued) *queued = (int)srv->queue.size();
  return ADER_OK;
}

ader_status ader_server_poll(ader_server* srv, uint64_t id, ader_result* out, double* u_host) {
  if (!srv || !out) return ADER_ERR_ARG;
  auto it = srv->reqs.find(id);
  if (it == srv->reqs.end()) return sfail(srv, ADER_ERR_ARG, "unknown request id %llu",
                                          (unsigned long long)id);
  const Req& r = *it->second;
  out->state = r.state;
  out->status = r.status;
  out->steps = r.steps;
  out->t = r.t;
  out->arrival = r.arrival;
  out->admitted = r.admitted;
  out->finished = r.finished;
  out->n_cells = r.ncells;
  out->degree = r.degree;
  if (u_host && (r.state == ADER_REQ_DONE || r.state == ADER_REQ_FAILED) && !r.result.empty())
    std::memcpy(u_host, r.result.data(), r.result.size() * sizeof(double));
  return ADER_OK;
}

ader_status ader_server_release(ader_server* srv, uint64_t id) {
  if (!srv) return ADER_ERR_ARG;
  auto it = srv->reqs.find(id);
  if (it == srv->reqs.end()) return ADER_ERR_ARG;
  if (it->second->state != ADER_REQ_DONE && it->second->state != ADER_REQ_FAILED)
    return sfail(srv, ADER_ERR_STATE, "request %llu is not finished", (unsigned long long)id);
  srv->reqs.erase(it);
  return ADER_OK;
}

ader_status ader_server_totals(const ader_server* srv, int64_t* cu, int64_t* ticks, int64_t* rounds,
                               int64_t* launches) {
  if (!srv) return ADER_ERR_ARG;
  if (cu) *cu = srv->cell_updates;
  if (ticks) *ticks = srv->ticks;
  if (rounds) *rounds = srv->rounds;
  if (launches) *launches = srv->launches;
  return ADER_OK;
}

}  // extern "C"
