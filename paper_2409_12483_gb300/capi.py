"""Thin ctypes binding of include/ader.h (argument marshalling only).

Every step of the method runs in libader_gb300.so; this module converts torch
tensors to device pointers, passes torch's current CUDA stream, and raises on a
non-OK status.  There is no CPU fallback: if the library or a GPU is missing the
calls fail loudly.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libader_gb300.so")

ADER_OK = 0
ADER_ERR_ARG = 1
ADER_ERR_NOMEM = 2
ADER_ERR_CUDA = 3
ADER_ERR_NOT_CONVERGED = 4
ADER_ERR_NONPHYSICAL = 5
ADER_ERR_TIMEOUT = 6
ADER_ERR_STATE = 7

SCHEMES = {"dg": 0, "fv": 1, "weno": 1}
PRECISIONS = {"fp64": 0, "fp32": 1, "ff": 2, "fp32ff": 3, "incr": 4}
SYSTEMS = {"euler": 0, "reacting": 1, "tracer": 2}
BOUNDARIES = {"periodic": 0, "outflow": 1}
CFL_MODES = {"subcell": 0, "nodal": 1}  # where lambda_max is taken (ader_options.cfl_mode)
SYSTEM_VARS = {0: 3, 1: 5, 2: 4}


class AderError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[{status}] {msg}")
        self.status = status


class Mesh(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("x0", C.c_double), ("x1", C.c_double)]


class Mesh2D(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("x0", C.c_double), ("x1", C.c_double),
                ("y0", C.c_double), ("y1", C.c_double)]


class Mesh3D(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64), ("x0", C.c_double),
                ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double), ("z0", C.c_double),
                ("z1", C.c_double)]


class Options(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("picard_tol", C.c_double),
                ("picard_max_iter", C.c_int), ("picard_fixed_iter", C.c_int),
                ("precision", C.c_int), ("fp64_sweeps", C.c_int), ("fp32_tol", C.c_double),
                ("profile", C.c_int), ("system", C.c_int), ("omega", C.c_double),
                ("bc", C.c_int), ("limiter", C.c_int), ("nad_delta0", C.c_double),
                ("nad_eps", C.c_double), ("cfl_mode", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("t", C.c_double), ("cells", C.c_int64),
                ("max_iters", C.c_int), ("mean_iters", C.c_double), ("status", C.c_int),
                ("profiled_steps", C.c_int64), ("weno_ms", C.c_double), ("predict_ms", C.c_double),
                ("face_ms", C.c_double), ("kernel_launches", C.c_int64),
                ("troubled_cells", C.c_int64)]


class ShardInfo(C.Structure):
    _fields_ = [("first_cell", C.c_int64), ("n_local", C.c_int64), ("n_global", C.c_int64),
                ("halo_cells", C.c_int64), ("values_per_cell", C.c_int64)]


class Tuning(C.Structure):
    _fields_ = [("predict_cells_per_block", C.c_int), ("face_cells_per_block", C.c_int),
                ("graph_steps", C.c_int), ("predict_ms", C.c_double), ("face_ms", C.c_double),
                ("solve_ms_per_step", C.c_double)]


class ServerOpts(C.Structure):
    _fields_ = [("pool_dev", C.c_void_p), ("pool_bytes", C.c_size_t), ("max_slots", C.c_int),
                ("ticks_per_round", C.c_int), ("precision", C.c_int), ("fp64_sweeps", C.c_int),
                ("gamma", C.c_double), ("cfl", C.c_double), ("picard_tol", C.c_double),
                ("stream", C.c_void_p)]


class Request(C.Structure):
    _fields_ = [("degree", C.c_int), ("n_cells", C.c_int64), ("x0", C.c_double),
                ("x1", C.c_double), ("t_end", C.c_double), ("arrival", C.c_double),
                ("u0_host", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("state", C.c_int), ("status", C.c_int), ("steps", C.c_int64), ("t", C.c_double),
                ("arrival", C.c_double), ("admitted", C.c_double), ("finished", C.c_double),
                ("n_cells", C.c_int64), ("degree", C.c_int)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3

_lib = None
_lock = threading.Lock()


def load(build_if_missing: bool = True):
    """Load libader_gb300.so (building it in-tree first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2409_12483_gb300.build")
        L = C.CDLL(LIB_PATH)
        V, P, D, I64, SZ = C.c_void_p, C.POINTER, C.c_double, C.c_int64, C.c_size_t
        sig = {
            "ader_default_options": ([P(Options)], C.c_int),
            "ader_init": ([P(Mesh), C.c_int, C.c_int, P(Options), P(V)], C.c_int),
            "ader_destroy": ([V], None),
            "ader_last_error": ([V], C.c_char_p),
            "ader_status_string": ([C.c_int], C.c_char_p),
            "ader_state_count": ([V], I64),
            "ader_predictor_count": ([V], I64),
            "ader_workspace_bytes": ([V], SZ),
            "ader_node_coords": ([V, V, I64], C.c_int),
            "ader_get_table": ([V, C.c_char_p, V, I64], C.c_int),
            "ader_bind": ([V, V, SZ, V], C.c_int),
            "ader_compute_dt": ([V, V, D, D, P(D)], C.c_int),
            "ader_predict": ([V, V, D, V], C.c_int),
            "ader_correct": ([V, V, V, D, V], C.c_int),
            "ader_step": ([V, V, V, D], C.c_int),
            "ader_weno_reconstruct": ([V, V, V], C.c_int),
            "ader_solve": ([V, V, D, I64, P(I64), P(D)], C.c_int),
            "ader_solve_host": ([V, V, D, I64, P(I64), P(D)], C.c_int),
            "ader_solve_from": ([V, V, D, D, I64, P(I64), P(D)], C.c_int),
            "ader_get_stats": ([V, P(Stats)], C.c_int),
            "ader_init_2d": ([V, C.c_int, V, V], C.c_int),
            "ader_init_3d": ([V, C.c_int, V, V], C.c_int),
            "ader_get_troubled": ([V, V, I64], C.c_int),
            "ader_step_noalloc": ([V, V, V, D, V], C.c_int),
            "ader_set_state": ([V, V, I64, C.c_int], C.c_int),
            "ader_get_state": ([V, V, I64, C.c_int], C.c_int),
            "ader_get_state_time": ([V, P(D)], C.c_int),
            "ader_get_predictor": ([V, D, V, I64], C.c_int),
            "ader_state_step": ([V, D, P(D)], C.c_int),
            "ader_state_solve": ([V, D, I64, P(I64), P(D)], C.c_int),
            "ader_init_shard": ([P(Mesh), I64, I64, C.c_int, C.c_int, P(Options), P(V)], C.c_int),
            "ader_shard_info": ([V, P(ShardInfo)], C.c_int),
            "ader_autotune": ([V, V, C.c_int, P(Tuning)], C.c_int),
            "ader_get_tuning": ([V, P(Tuning)], C.c_int),
            "ader_set_tuning": ([V, P(Tuning)], C.c_int),
            "ader_server_default_options": ([P(ServerOpts)], C.c_int),
            "ader_server_create": ([P(ServerOpts), P(V)], C.c_int),
            "ader_server_destroy": ([V], None),
            "ader_server_last_error": ([V], C.c_char_p),
            "ader_server_request_bytes": ([C.c_int, I64], SZ),
            "ader_server_submit": ([V, P(Request), P(C.c_uint64)], C.c_int),
            "ader_server_progress": ([V, D, P(C.c_int), P(C.c_int)], C.c_int),
            "ader_server_poll": ([V, C.c_uint64, P(Result), V], C.c_int),
            "ader_server_release": ([V, C.c_uint64], C.c_int),
            "ader_server_totals": ([V, P(I64), P(I64), P(I64), P(I64)], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return _lib


def exported_symbols():
    """Names the header declares (for the ABI test)."""
    return ["ader_default_options", "ader_init", "ader_destroy", "ader_last_error",
            "ader_status_string", "ader_state_count", "ader_predictor_count",
            "ader_workspace_bytes", "ader_node_coords", "ader_get_table", "ader_bind",
            "ader_compute_dt", "ader_predict", "ader_correct", "ader_step",
            "ader_weno_reconstruct", "ader_solve", "ader_solve_host", "ader_solve_from",
            "ader_get_stats", "ader_get_troubled", "ader_init_2d", "ader_init_3d",
            "ader_step_noalloc", "ader_set_state", "ader_get_state", "ader_get_state_time",
            "ader_get_predictor", "ader_state_step", "ader_state_solve", "ader_init_shard",
            "ader_shard_info", "ader_autotune", "ader_get_tuning", "ader_set_tuning",
            "ader_server_default_options", "ader_server_create",
            "ader_server_destroy", "ader_server_last_error", "ader_server_request_bytes",
            "ader_server_submit", "ader_server_progress", "ader_server_poll",
            "ader_server_release", "ader_server_totals"]


def default_options(**kw) -> Options:
    o = Options()
    load().ader_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "system" and isinstance(v, str):
            v = SYSTEMS[v]
        if k == "bc" and isinstance(v, str):
            v = BOUNDARIES[v]
        if k == "limiter" and isinstance(v, bool):
            v = int(v)
        if k == "cfl_mode" and isinstance(v, str):
            v = CFL_MODES[v]
        setattr(o, k, v)
    return o


def _torch():
    import torch
    return torch


def _ptr(t, dtype=None, numel=None, name="tensor"):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


class Context:
    """An ader_ctx bound to a torch-allocated workspace and torch's current stream."""

    def __init__(self, n_cells: int, degree: int, scheme: str = "dg", x0: float = 0.0,
                 x1: float = 1.0, device=None, **options):
        torch = _torch()
        L = load()
        self._L = L
        self.n_cells = int(n_cells)
        self.degree = int(degree)
        self.scheme = scheme
        self.n = self.degree + 1
        mesh = Mesh(self.n_cells, float(x0), float(x1))
        self.options = default_options(**options)
        ctx = C.c_void_p()
        rc = self._create(L, mesh, ctx)
        if rc != ADER_OK:
            raise AderError(rc, f"ader_init failed ({L.ader_status_string(rc).decode()})")
        self._ctx = ctx
        self._bind_workspace(device)
        self.vars = SYSTEM_VARS[self.options.system] if scheme == "dg" else 3

    def _create(self, L, mesh, ctx):
        return L.ader_init(C.byref(mesh), self.degree, SCHEMES[self.scheme], C.byref(self.options),
                           C.byref(ctx))

    def _bind_workspace(self, device):
        torch = _torch()
        L, ctx = self._L, self._ctx
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        nbytes = int(L.ader_workspace_bytes(ctx))
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        stream = torch.cuda.current_stream(self.device).cuda_stream
        self._check(L.ader_bind(ctx, C.c_void_p(aligned), nbytes, C.c_void_p(stream)))
        self.state_count = int(L.ader_state_count(ctx))
        self.predictor_count = int(L.ader_predictor_count(ctx))
        self.workspace_bytes = nbytes

    # -- helpers --
    def _check(self, rc: int, ok=(ADER_OK,)):
        if rc not in ok:
            msg = self._L.ader_last_error(self._ctx).decode()
            raise AderError(rc, msg or self._L.ader_status_string(rc).decode())
        return rc

    def close(self):
        if getattr(self, "_ctx", None):
            self._L.ader_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def state_shape(self):
        return (self.n_cells, self.n, self.vars) if self.scheme == "dg" else (self.n_cells, 3)

    # -- host-side queries --
    def node_coords(self):
        import numpy as np
        per = self.n if self.scheme == "dg" else 1
        x = np.zeros(self.n_cells * per)
        self._check(self._L.ader_node_coords(self._ctx, x.ctypes.data_as(C.c_void_p), x.size))
        return x.reshape(self.n_cells, per) if per > 1 else x

    def table(self, name: str):
        import numpy as np
        n = self.n
        H = (n + 1) // 2
        size = {"xi": n, "w": n, "psi0": n, "psi1": n, "P": (2 * self.degree + 1) * n,
                "ksa": H * H, "ksb": H * H, "wamono": 3 * n * n,
                "R": n * (2 * self.degree + 1)}.get(name, n * n)
        out = np.zeros(size)
        self._check(self._L.ader_get_table(self._ctx, name.encode(), out.ctypes.data_as(C.c_void_p),
                                           size))
        if name in ("xi", "w", "psi0", "psi1"):
            return out
        if name == "R":
            return out.reshape(n, -1)
        return out.reshape(-1, H if name in ("ksa", "ksb") else n)

    # -- hot path (same names as the C ABI) --
    def ader_compute_dt(self, u, t: float = 0.0, t_end: float = 0.0) -> float:
        dt = C.c_double(0.0)
        self._check(self._L.ader_compute_dt(self._ctx, _ptr(u, numel=self.state_count, name="u"),
                                            t, t_end, C.byref(dt)))
        return dt.value

    def ader_predict(self, u, dt: float, q):
        return self._check(self._L.ader_predict(self._ctx, _ptr(u, numel=self.state_count, name="u"),
                                                float(dt),
                                                _ptr(q, numel=self.predictor_count, name="q")))

    def ader_correct(self, u, q, dt: float, u_new):
        return self._check(self._L.ader_correct(
            self._ctx, _ptr(u, numel=self.state_count, name="u"),
            _ptr(q, numel=self.predictor_count, name="q"), float(dt),
            _ptr(u_new, numel=self.state_count, name="u_new")))

    def ader_step(self, u, u_new, dt: float = 0.0):
        return self._check(self._L.ader_step(self._ctx, _ptr(u, numel=self.state_count, name="u"),
                                             _ptr(u_new, numel=self.state_count, name="u_new"),
                                             float(dt)))

    def ader_weno_reconstruct(self, v, w):
        return self._check(self._L.ader_weno_reconstruct(
            self._ctx, _ptr(v, numel=self.n_cells * 3, name="v"),
            _ptr(w, numel=self.n_cells * self.n * 3, name="w")))

    def ader_solve(self, u, t_end: float = 0.0, max_steps: int = 0, allow=()):
        steps = C.c_int64(0)
        t = C.c_double(0.0)
        rc = self._L.ader_solve(self._ctx, _ptr(u, numel=self.state_count, name="u"),
                                float(t_end), int(max_steps), C.byref(steps), C.byref(t))
        self._check(rc, ok=(ADER_OK, *allow))
        return steps.value, t.value, rc

    def ader_solve_from(self, u, t0: float, t_end: float = 0.0, max_steps: int = 0, allow=()):
        steps = C.c_int64(0)
        t = C.c_double(0.0)
        rc = self._L.ader_solve_from(self._ctx, _ptr(u, numel=self.state_count, name="u"),
                                     float(t0), float(t_end), int(max_steps), C.byref(steps),
                                     C.byref(t))
        self._check(rc, ok=(ADER_OK, *allow))
        return steps.value, t.value, rc

    def ader_solve_host(self, u_host, t_end: float = 0.0, max_steps: int = 0, allow=()):
        """u_host: a C-contiguous float64 numpy array or CPU torch tensor (pinned is faster)."""
        import numpy as np
        torch = _torch()
        if isinstance(u_host, torch.Tensor):
            if u_host.is_cuda or u_host.dtype != torch.float64 or not u_host.is_contiguous():
                raise ValueError("u_host: expected a contiguous CPU float64 tensor")
            ptr, numel = u_host.data_ptr(), u_host.numel()
        else:
            if u_host.dtype != np.float64 or not u_host.flags.c_contiguous:
                raise ValueError("u_host: expected a C-contiguous float64 array")
            ptr, numel = u_host.ctypes.data, u_host.size
        if numel != self.state_count:
            raise ValueError(f"u_host: expected {self.state_count} elements")
        steps = C.c_int64(0)
        t = C.c_double(0.0)
        rc = self._L.ader_solve_host(self._ctx, C.c_void_p(ptr), float(t_end), int(max_steps),
                                     C.byref(steps), C.byref(t))
        self._check(rc, ok=(ADER_OK, *allow))
        return steps.value, t.value, rc

    def ader_autotune(self, u, reps: int = 3) -> dict:
        t = Tuning()
        self._check(self._L.ader_autotune(self._ctx, _ptr(u, numel=self.state_count, name="u"),
                                          int(reps), C.byref(t)))
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    def ader_get_tuning(self) -> dict:
        t = Tuning()
        self._check(self._L.ader_get_tuning(self._ctx, C.byref(t)))
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    def ader_set_tuning(self, **kw):
        t = Tuning()
        self._check(self._L.ader_get_tuning(self._ctx, C.byref(t)))
        for k, v in kw.items():
            setattr(t, k, v)
        self._check(self._L.ader_set_tuning(self._ctx, C.byref(t)))

    def ader_get_troubled(self, flags=None):
        """troubled-cell flags (int32 per cell, on the device) of the last limited step"""
        torch = _torch()
        if flags is None:
            flags = torch.empty(self.n_cells, dtype=torch.int32, device=self.device)
        self._check(self._L.ader_get_troubled(self._ctx, C.c_void_p(flags.data_ptr()), flags.numel()))
        return flags

    # -- context-resident state --
    def ader_set_state(self, u):
        """u: a CUDA tensor (copied on the device) or a host array / CPU tensor."""
        torch = _torch()
        if isinstance(u, torch.Tensor) and u.is_cuda:
            return self._check(self._L.ader_set_state(
                self._ctx, _ptr(u, numel=self.state_count, name="u"), self.state_count, 1))
        import numpy as np
        a = np.ascontiguousarray(np.asarray(u.cpu() if isinstance(u, torch.Tensor) else u,
                                            dtype=np.float64).ravel())
        if a.size != self.state_count:
            raise ValueError(f"state has {a.size} values, expected {self.state_count}")
        return self._check(self._L.ader_set_state(self._ctx, a.ctypes.data_as(C.c_void_p),
                                                  a.size, 0))

    def ader_get_state(self, out=None, on_device: bool = True):
        """The resident state: into `out` (a CUDA tensor, or a host numpy array),
        else a new CUDA tensor (on_device) or numpy array."""
        torch = _torch()
        import numpy as np
        if out is None:
            out = (torch.empty(self.state_count, dtype=torch.float64, device=self.device)
                   if on_device else np.empty(self.state_count))
        if isinstance(out, torch.Tensor):
            self._check(self._L.ader_get_state(
                self._ctx, _ptr(out, numel=self.state_count, name="out"), self.state_count, 1))
        else:
            if out.dtype != np.float64 or out.size != self.state_count or not out.flags.c_contiguous:
                raise ValueError("out must be a contiguous float64 array of state_count values")
            self._check(self._L.ader_get_state(self._ctx, out.ctypes.data_as(C.c_void_p),
                                               self.state_count, 0))
        return out

    def ader_get_state_time(self) -> float:
        t = C.c_double(0.0)
        self._check(self._L.ader_get_state_time(self._ctx, C.byref(t)))
        return t.value

    def ader_get_predictor(self, dt: float = 0.0, q=None):
        torch = _torch()
        if q is None:
            q = torch.empty(self.predictor_count, dtype=torch.float64, device=self.device)
        self._check(self._L.ader_get_predictor(self._ctx, float(dt),
                                               _ptr(q, numel=self.predictor_count, name="q"),
                                               self.predictor_count))
        return q

    def ader_state_step(self, dt: float = 0.0) -> float:
        used = C.c_double(0.0)
        self._check(self._L.ader_state_step(self._ctx, float(dt), C.byref(used)))
        return used.value

    def ader_state_solve(self, t_end: float = 0.0, max_steps: int = 0, allow=()):
        steps, t = C.c_int64(0), C.c_double(0.0)
        rc = self._check(self._L.ader_state_solve(self._ctx, float(t_end), int(max_steps),
                                                  C.byref(steps), C.byref(t)),
                         ok=(ADER_OK,) + tuple(allow))
        return steps.value, t.value, rc

    def ader_get_stats(self) -> dict:
        s = Stats()
        self._check(self._L.ader_get_stats(self._ctx, C.byref(s)))
        return {"steps": s.steps, "t": s.t, "cells": s.cells, "max_iters": s.max_iters,
                "mean_iters": s.mean_iters, "status": s.status,
                "profiled_steps": s.profiled_steps, "weno_ms": s.weno_ms,
                "predict_ms": s.predict_ms, "face_ms": s.face_ms,
                "kernel_launches": s.kernel_launches, "troubled_cells": s.troubled_cells}


class Context2D(Context):
    """An ader_ctx of the 2D Euler equations on a periodic nx x ny Cartesian mesh
    (ader_init_2d); state [iy][ix][k1][k2][4] with r = (rho, m_x, m_y, E).
    ader_step / ader_solve / ader_solve_host / ader_compute_dt / ader_get_stats
    work as for 1D contexts."""

    def __init__(self, nx: int, ny: int, degree: int, x0: float = 0.0, x1: float = 1.0,
                 y0: float = 0.0, y1: float = 1.0, device=None, **options):
        L = load()
        self._L = L
        self.nx, self.ny = int(nx), int(ny)
        self.n_cells = self.nx * self.ny
        self.degree = int(degree)
        self.scheme = "dg"
        self.n = self.degree + 1
        self.bounds = (float(x0), float(x1), float(y0), float(y1))
        mesh = Mesh2D(self.nx, self.ny, *self.bounds)
        self.options = default_options(**options)
        ctx = C.c_void_p()
        rc = L.ader_init_2d(C.byref(mesh), self.degree, C.byref(self.options), C.byref(ctx))
        if rc != ADER_OK:
            raise AderError(rc, f"ader_init_2d failed ({L.ader_status_string(rc).decode()})")
        self._ctx = ctx
        self._bind_workspace(device)
        self.vars = 4

    def state_shape(self):
        return (self.ny, self.nx, self.n, self.n, 4)

    def node_coords(self):
        """(X, Y), each [ny][nx][n][n]: the GL nodes of every cell (k1 along x, k2 along y)."""
        import numpy as np
        xi = self.table("xi")
        x0, x1, y0, y1 = self.bounds
        dx, dy = (x1 - x0) / self.nx, (y1 - y0) / self.ny
        X = x0 + dx * (np.arange(self.nx)[None, :, None, None] + xi[None, None, :, None])
        Y = y0 + dy * (np.arange(self.ny)[:, None, None, None] + xi[None, None, None, :])
        shape = (self.ny, self.nx, self.n, self.n)
        return np.broadcast_to(X, shape).copy(), np.broadcast_to(Y, shape).copy()


class Context3D(Context):
    """An ader_ctx of the 3D Euler equations on a periodic nx x ny x nz Cartesian
    mesh (ader_init_3d, degrees 0..7); state [iz][iy][ix][k1][k2][k3][5] with
    r = (rho, m_x, m_y, m_z, E)."""

    def __init__(self, nx: int, ny: int, nz: int, degree: int, box=(1.0, 1.0, 1.0), device=None,
                 **options):
        L = load()
        self._L = L
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.n_cells = self.nx * self.ny * self.nz
        self.degree = int(degree)
        self.scheme = "dg"
        self.n = self.degree + 1
        self.box = tuple(float(b) for b in box)
        mesh = Mesh3D(self.nx, self.ny, self.nz, 0.0, self.box[0], 0.0, self.box[1], 0.0,
                      self.box[2])
        self.options = default_options(**options)
        ctx = C.c_void_p()
        rc = L.ader_init_3d(C.byref(mesh), self.degree, C.byref(self.options), C.byref(ctx))
        if rc != ADER_OK:
            raise AderError(rc, f"ader_init_3d failed ({L.ader_status_string(rc).decode()})")
        self._ctx = ctx
        self._bind_workspace(device)
        self.vars = 5

    def state_shape(self):
        return (self.nz, self.ny, self.nx, self.n, self.n, self.n, 5)

    def node_coords(self):
        """(X, Y, Z), each [nz][ny][nx][n][n][n]."""
        import numpy as np
        xi = self.table("xi")
        n = self.n
        shape = (self.nz, self.ny, self.nx, n, n, n)
        X = self.box[0] / self.nx * (np.arange(self.nx)[None, None, :, None, None, None]
                                     + xi[None, None, None, :, None, None])
        Y = self.box[1] / self.ny * (np.arange(self.ny)[None, :, None, None, None, None]
                                     + xi[None, None, None, None, :, None])
        Z = self.box[2] / self.nz * (np.arange(self.nz)[:, None, None, None, None, None]
                                     + xi[None, None, None, None, None, :])
        return tuple(np.broadcast_to(A, shape).copy() for A in (X, Y, Z))


class ShardContext(Context):
    """One shard of a periodic global 1D mesh (ader_init_shard): the cells
    [first_cell, first_cell + n_local) plus `halo` copies of the neighbours'
    cells on each side, as one state array of n_local + 2 halo cells."""

    def __init__(self, n_global: int, first_cell: int, n_local: int, degree: int,
                 scheme: str = "dg", x0: float = 0.0, x1: float = 1.0, device=None, **options):
        self._shard_args = (int(n_global), int(first_cell), int(n_local))
        self._gx = (float(x0), float(x1))
        super().__init__(n_local, degree, scheme, x0, x1, device, **options)
        info = ShardInfo()
        self._check(self._L.ader_shard_info(self._ctx, C.byref(info)))
        self.first_cell, self.n_local = info.first_cell, info.n_local
        self.n_global, self.halo = info.n_global, info.halo_cells
        self.values_per_cell = info.values_per_cell
        self.n_cells = self.n_local + 2 * self.halo

    def _create(self, L, mesh, ctx):
        n_global, first, n_local = self._shard_args
        return L.ader_init_shard(C.byref(Mesh(n_global, *self._gx)), first, n_local, self.degree,
                                 SCHEMES[self.scheme], C.byref(self.options), C.byref(ctx))


class NoAllocStep:
    """ader_step_noalloc for callers that cannot allocate device memory.

    Holds only an ader_ctx from ader_init (host memory); no workspace is bound.
    Each call runs one time step with its scratch in the library's static device
    array (ADER_NOALLOC_SCRATCH_BYTES per GPU); the caller passes the input and
    output states.  Calls whose work overlaps on the GPU race on that array.
    """

    def __init__(self, n_cells: int, degree: int, scheme: str = "dg", x0: float = 0.0,
                 x1: float = 1.0, **options):
        L = load()
        self._L = L
        self.n_cells, self.degree, self.scheme = int(n_cells), int(degree), scheme
        self.options = default_options(**options)
        ctx = C.c_void_p()
        rc = L.ader_init(C.byref(Mesh(self.n_cells, float(x0), float(x1))), self.degree,
                         SCHEMES[scheme], C.byref(self.options), C.byref(ctx))
        if rc != ADER_OK:
            raise AderError(rc, f"ader_init failed ({L.ader_status_string(rc).decode()})")
        self._ctx = ctx
        self.state_count = int(L.ader_state_count(ctx))

    def step(self, u, u_new, dt: float, stream=None, allow=()):
        """One step; synchronises the stream and returns the status (statuses in
        `allow`, e.g. ADER_ERR_NOT_CONVERGED, are returned instead of raised)."""
        torch = _torch()
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        rc = self._L.ader_step_noalloc(self._ctx, _ptr(u, numel=self.state_count, name="u"),
                                       _ptr(u_new, numel=self.state_count, name="u_new"),
                                       float(dt), C.c_void_p(s))
        if rc != ADER_OK and rc not in allow:
            raise AderError(rc, self._L.ader_last_error(self._ctx).decode())
        return rc

    def close(self):
        if getattr(self, "_ctx", None):
            self._L.ader_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server of independent ADER-DG solves (ader_server_*).

    torch allocates the device pool; the server sub-allocates it, admits requests
    by memory and slots, and advances every resident solve each tick."""

    def __init__(self, pool_bytes: int = 1 << 30, max_slots: int = 256, ticks_per_round: int = 16,
                 precision: str = "fp64", fp64_sweeps: int = 1, device=None, cfl: float = 0.4,
                 gamma: float = 1.4):
        torch = _torch()
        L = load()
        self._L = L
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self._pool = torch.empty(int(pool_bytes) + 256, dtype=torch.uint8, device=self.device)
        aligned = (self._pool.data_ptr() + 255) // 256 * 256
        o = ServerOpts()
        L.ader_server_default_options(C.byref(o))
        o.pool_dev = aligned
        o.pool_bytes = int(pool_bytes)
        o.max_slots = int(max_slots)
        o.ticks_per_round = int(ticks_per_round)
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.fp64_sweeps = int(fp64_sweeps)
        o.cfl = float(cfl)
        o.gamma = float(gamma)
        o.stream = torch.cuda.current_stream(self.device).cuda_stream
        srv = C.c_void_p()
        rc = L.ader_server_create(C.byref(o), C.byref(srv))
        if rc != ADER_OK:
            raise AderError(rc, f"ader_server_create failed ({L.ader_status_string(rc).decode()})")
        self._srv = srv
        self.opts = o

    def _check(self, rc, ok=(ADER_OK,)):
        if rc not in ok:
            raise AderError(rc, self._L.ader_server_last_error(self._srv).decode())
        return rc

    @staticmethod
    def request_bytes(degree: int, n_cells: int) -> int:
        return int(load().ader_server_request_bytes(int(degree), int(n_cells)))

    def submit(self, degree: int, u0, t_end: float, arrival: float = 0.0, x0: float = 0.0,
               x1: float = 1.0) -> int:
        import numpy as np
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        n_cells = u0.size // ((degree + 1) * 3)
        if n_cells * (degree + 1) * 3 != u0.size:
            raise ValueError("u0 size does not match the degree")
        rq = Request(int(degree), int(n_cells), float(x0), float(x1), float(t_end), float(arrival),
                     u0.ctypes.data)
        rid = C.c_uint64(0)
        self._check(self._L.ader_server_submit(self._srv, C.byref(rq), C.byref(rid)))
        return rid.value

    def progress(self, now: float):
        run, que = C.c_int(0), C.c_int(0)
        self._check(self._L.ader_server_progress(self._srv, float(now), C.byref(run), C.byref(que)))
        return run.value, que.value

    def poll(self, rid: int, want_state: bool = False):
        import numpy as np
        r = Result()
        self._check(self._L.ader_server_poll(self._srv, int(rid), C.byref(r), None))
        out = {"state": r.state, "status": r.status, "steps": r.steps, "t": r.t,
               "arrival": r.arrival, "admitted": r.admitted, "finished": r.finished,
               "n_cells": r.n_cells, "degree": r.degree}
        if want_state and r.state in (REQ_DONE, REQ_FAILED):
            u = np.zeros(r.n_cells * (r.degree + 1) * 3)
            self._check(self._L.ader_server_poll(self._srv, int(rid), C.byref(r),
                                                 u.ctypes.data_as(C.c_void_p)))
            out["u"] = u
        return out

    def release(self, rid: int):
        self._check(self._L.ader_server_release(self._srv, int(rid)))

    def totals(self):
        a, b, c, d = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self._L.ader_server_totals(self._srv, C.byref(a), C.byref(b), C.byref(c),
                                               C.byref(d)))
        return {"cell_updates": a.value, "ticks": b.value, "rounds": c.value,
                "kernel_launches": d.value}

    def close(self):
        if getattr(self, "_srv", None):
            self._L.ader_server_destroy(self._srv)
            self._srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
