"""Plain FP64 CPU oracle of the 1D ADER-DG / ADER-WENO schemes (arXiv 2409.12483).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package; the product package ``paper_2409_12483_gb300`` never does, and this
package never imports the product package.  The arithmetic lives in
``ader_oracle.c`` (plain C, FP64, long double for the basis); this module only
marshals numpy arrays through ctypes and adds the error norms of Sec. 2.1
(eq. epsilons), which are plain numpy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ader_oracle.c")
_SRC_RS = os.path.join(_HERE, "ader_oracle_src.c")
_SRC_LIM = os.path.join(_HERE, "ader_oracle_lim.c")
_SRC_2D = os.path.join(_HERE, "ader_oracle_2d.c")
_SRC_3D = os.path.join(_HERE, "ader_oracle_3d.c")
_SRC_NC = os.path.join(_HERE, "ader_oracle_nc.c")
_HDR = os.path.join(_HERE, "ader_oracle.h")
_LIB_PATH = os.path.join(_HERE, "libader_oracle.so")

M = 3
MRS = 5  # reacting system: rho, m, E, rho c1, rho c2
M2 = 4   # 2D Euler: rho, m_x, m_y, E
M3 = 5   # 3D Euler: rho, m_x, m_y, m_z, E
MNC = 4  # Euler + non-conservative passive tracer: rho, m, E, phi
MAXN = 10
MAXNS = 19

OB_OK = 0
OB_ERR_ARG = 1
OB_ERR_NOT_CONVERGED = 4
OB_ERR_NONPHYSICAL = 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no fast-math)."""
    newest = max(os.path.getmtime(f) for f in (_SRC, _SRC_RS, _SRC_LIM, _SRC_2D, _SRC_3D, _SRC_NC, _HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, _SRC_RS, _SRC_LIM, _SRC_2D,
           _SRC_3D, _SRC_NC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Basis(C.Structure):
    _fields_ = [
        ("N", C.c_int), ("n", C.c_int), ("Ns", C.c_int),
        ("xi", C.c_double * MAXN), ("w", C.c_double * MAXN),
        ("psi0", C.c_double * MAXN), ("psi1", C.c_double * MAXN),
        ("dphi", (C.c_double * MAXN) * MAXN),
        ("lam", (C.c_double * MAXN) * MAXN),
        ("xi_m", (C.c_double * MAXN) * MAXN),
        ("ups", (C.c_double * MAXN) * MAXN),
        ("kap", (C.c_double * MAXN) * MAXN),
        ("kt", (C.c_double * MAXN) * MAXN),
        ("dt_m", (C.c_double * MAXN) * MAXN),
        ("P", (C.c_double * MAXN) * MAXNS),
    ]


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("tol", C.c_double),
                ("max_iter", C.c_int), ("fixed_iter", C.c_int), ("cfl_mode", C.c_int)]


class Weno(C.Structure):
    _fields_ = [
        ("N", C.c_int), ("n", C.c_int), ("shift", C.c_int * 3),
        ("lin", C.c_double * 3), ("eps", C.c_double), ("r", C.c_int),
        ("ainv", ((C.c_double * MAXN) * MAXN) * 3),
        ("sig", (C.c_double * MAXN) * MAXN),
        ("dal", ((C.c_double * MAXN) * MAXN) * MAXN),
        ("wq", C.c_double * MAXN),
    ]


class LimParams(C.Structure):
    _fields_ = [("bc", C.c_int), ("limiter", C.c_int), ("delta0", C.c_double), ("eps", C.c_double)]


class RSParams(C.Structure):
    _fields_ = [("gamma", C.c_double), ("omega", C.c_double), ("cfl", C.c_double),
                ("tol", C.c_double), ("max_iter", C.c_int), ("fixed_iter", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("cells", C.c_int64), ("max_iters", C.c_int), ("min_iters", C.c_int),
                ("mean_iters", C.c_double), ("status", C.c_int)]


_lib = None
_lock = threading.Lock()
_DP = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_IP = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            P = C.POINTER
            L.ob_basis_build.argtypes = [C.c_int, P(Basis)]
            L.ob_basis_eval.argtypes = [P(Basis), C.c_double, _DP]
            L.ob_basis_eval.restype = None
            L.ob_euler_flux.argtypes = [C.c_double, _DP, _DP]
            L.ob_euler_flux.restype = None
            L.ob_wave_speed.argtypes = [C.c_double, _DP]
            L.ob_wave_speed.restype = C.c_double
            L.ob_rusanov.argtypes = [C.c_double, _DP, _DP, _DP]
            L.ob_rusanov.restype = None
            for name in ("ob_predict_cell", "ob_predict_cell_nested"):
                f = getattr(L, name)
                f.argtypes = [P(Basis), P(Params), C.c_double, _DP, _DP, P(C.c_int)]
            L.ob_dg_lambda_max.argtypes = [P(Basis), C.c_double, C.c_int64, _DP]
            L.ob_dg_lambda_max.restype = C.c_double
            L.ob_dg_lambda_max_nodal.argtypes = [P(Basis), C.c_double, C.c_int64, _DP]
            L.ob_dg_lambda_max_nodal.restype = C.c_double
            L.ob_fv_lambda_max.argtypes = [C.c_double, C.c_int64, _DP]
            L.ob_fv_lambda_max.restype = C.c_double
            L.ob_dg_dt.argtypes = [P(Basis), P(Params), C.c_double, C.c_int64, _DP]
            L.ob_dg_dt.restype = C.c_double
            L.ob_fv_dt.argtypes = [P(Params), C.c_double, C.c_int64, _DP]
            L.ob_fv_dt.restype = C.c_double
            L.ob_dg_correct.argtypes = [P(Basis), P(Params), C.c_int64, C.c_double, C.c_double,
                                        _DP, _DP, _DP]
            L.ob_dg_step.argtypes = [P(Basis), P(Params), C.c_int64, C.c_double, C.c_double,
                                     _DP, _DP, C.c_void_p, P(Stats)]
            L.ob_dg_step_cells.argtypes = [P(Basis), P(Params), C.c_int64, C.c_double, C.c_double,
                                           _DP, _IP, C.c_int64, _DP]
            L.ob_weno_build.argtypes = [C.c_int, P(Basis), P(Weno)]
            L.ob_weno_sigma.argtypes = [P(Weno), _DP]
            L.ob_weno_sigma.restype = C.c_double
            L.ob_weno_reconstruct.argtypes = [P(Weno), C.c_int64, _DP, _DP]
            L.ob_weno_cell.argtypes = [P(Weno), C.c_int64, _DP, C.c_int64, _DP, C.c_void_p]
            L.ob_fv_step.argtypes = [P(Basis), P(Weno), P(Params), C.c_int64, C.c_double,
                                     C.c_double, _DP, _DP, P(Stats)]
            L.ob_fv_step_cells.argtypes = [P(Basis), P(Weno), P(Params), C.c_int64, C.c_double,
                                           C.c_double, _DP, _IP, C.c_int64, _DP]
            L.ob_solve.argtypes = [C.c_int, P(Basis), C.c_void_p, P(Params), C.c_int64,
                                   C.c_double, _DP, C.c_double, C.c_int64, P(C.c_int64),
                                   P(C.c_double)]
            L.ob_r_matrix.argtypes = [P(Basis), _DP]
            L.ob2_flux.argtypes = [C.c_double, _DP, _DP, _DP]
            L.ob2_flux.restype = None
            L.ob2_rusanov.argtypes = [C.c_double, C.c_int, _DP, _DP, _DP]
            L.ob2_rusanov.restype = None
            L.ob2_predict_cell.argtypes = [P(Basis), P(Params), C.c_double, C.c_double, _DP, _DP,
                                           P(C.c_int)]
            L.ob2_dg_step.argtypes = [P(Basis), P(Params), C.c_int64, C.c_int64, C.c_double,
                                      C.c_double, C.c_double, _DP, _DP, P(Stats)]
            L.ob2_dg_step_cells.argtypes = [P(Basis), P(Params), C.c_int64, C.c_int64, C.c_double,
                                            C.c_double, C.c_double, _DP, _IP, C.c_int64, _DP]
            L.ob3_dg_step_cells.argtypes = [P(Basis), P(Params), C.c_int64, C.c_int64, C.c_int64,
                                            C.c_double, C.c_double, C.c_double, C.c_double, _DP, _IP,
                                            C.c_int64, _DP]
            L.ob2_dt.argtypes = [P(Basis), P(Params), C.c_int64, C.c_int64, C.c_double, C.c_double,
                                 _DP]
            L.ob2_dt.restype = C.c_double
            L.ob2_solve.argtypes = [P(Basis), P(Params), C.c_int64, C.c_int64, C.c_double,
                                    C.c_double, _DP, C.c_double, C.c_int64, P(C.c_int64),
                                    P(C.c_double)]
            L.ob3_flux.argtypes = [C.c_double, _DP, _DP]
            L.ob3_flux.restype = None
            L.ob3_rusanov.argtypes = [C.c_double, C.c_int, _DP, _DP, _DP]
            L.ob3_rusanov.restype = None
            L.ob3_predict_cell.argtypes = [P(Basis), P(Params), C.c_double, C.c_double,
                                           C.c_double, _DP, _DP, P(C.c_int)]
            L.ob3_dg_step.argtypes = [P(Basis), P(Params), C.c_int64, C.c_int64, C.c_int64,
                                      C.c_double, C.c_double, C.c_double, C.c_double, _DP, _DP,
                                      P(Stats)]
            L.ob3_dt.argtypes = [P(Basis), P(Params), C.c_int64, C.c_int64, C.c_int64, C.c_double,
                                 C.c_double, C.c_double, _DP]
            L.ob3_dt.restype = C.c_double
            L.ob3_solve.argtypes = [P(Basis), P(Params), C.c_int64, C.c_int64, C.c_int64,
                                    C.c_double, C.c_double, C.c_double, _DP, C.c_double,
                                    C.c_int64, P(C.c_int64), P(C.c_double)]
            L.ob_nc_flux.argtypes = [C.c_double, _DP, _DP]
            L.ob_nc_flux.restype = None
            L.ob_nc_face.argtypes = [C.c_double, _DP, _DP, _DP, P(C.c_double)]
            L.ob_nc_face.restype = None
            L.ob_nc_predict_cell.argtypes = [P(Basis), P(Params), C.c_double, _DP, _DP, P(C.c_int)]
            L.ob_nc_step.argtypes = [P(Basis), P(Params), C.c_int64, C.c_double, C.c_double, _DP,
                                     _DP, P(Stats)]
            L.ob_nc_solve.argtypes = [P(Basis), P(Params), C.c_int64, C.c_double, _DP, C.c_double,
                                      C.c_int64, P(C.c_int64), P(C.c_double)]
            L.ob_lim_weno2.argtypes = [_DP, _DP, _DP, _DP, _DP]
            L.ob_lim_weno2.restype = None
            L.ob_dgl_step.argtypes = [P(Basis), P(Params), P(LimParams), C.c_int64, C.c_double,
                                      C.c_double, _DP, _DP, C.c_void_p, P(Stats)]
            L.ob_dgl_solve.argtypes = [P(Basis), P(Params), P(LimParams), C.c_int64, C.c_double, _DP,
                                       C.c_double, C.c_int64, P(C.c_int64), P(C.c_double),
                                       P(C.c_int64)]
            L.ob_rs_flux.argtypes = [C.c_double, _DP, _DP]
            L.ob_rs_flux.restype = None
            L.ob_rs_source.argtypes = [C.c_double, _DP, _DP]
            L.ob_rs_source.restype = None
            L.ob_rs_rusanov.argtypes = [C.c_double, _DP, _DP, _DP]
            L.ob_rs_rusanov.restype = None
            L.ob_rs_predict_cell.argtypes = [P(Basis), P(RSParams), C.c_double, C.c_double, _DP,
                                             _DP, P(C.c_int), P(C.c_int)]
            L.ob_rs_predict_cell_direct.argtypes = [P(Basis), P(RSParams), C.c_double, C.c_double,
                                                    _DP, _DP, P(C.c_int)]
            L.ob_rs_dg_dt.argtypes = [P(Basis), P(RSParams), C.c_double, C.c_int64, _DP]
            L.ob_rs_dg_dt.restype = C.c_double
            L.ob_rs_dg_step.argtypes = [P(Basis), P(RSParams), C.c_int64, C.c_double, C.c_double,
                                        _DP, _DP, C.c_void_p, P(Stats)]
            L.ob_rs_dg_step_cells.argtypes = [P(Basis), P(RSParams), C.c_int64, C.c_double,
                                              C.c_double, _DP, _IP, C.c_int64, _DP]
            L.ob_rs_solve.argtypes = [P(Basis), P(RSParams), C.c_int64, C.c_double, _DP, C.c_double,
                                      C.c_int64, C.c_double, P(C.c_int64), P(C.c_double)]
            _lib = L
    return _lib


def _arr(x, n=None):
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a if n is None else a.reshape(n)


class Oracle:
    """One degree N: basis, operators and (for even N >= 2) WENO tables."""

    def __init__(self, N: int, gamma: float = 1.4, cfl: float = 0.4, tol: float = 1e-13,
                 max_iter: int | None = None, fixed_iter: int = 0):
        L = lib()
        self.N = N
        self.n = N + 1
        self.basis = Basis()
        rc = L.ob_basis_build(N, C.byref(self.basis))
        if rc != OB_OK:
            raise ValueError(f"oracle basis build failed for N={N}")
        self.params = Params(gamma, cfl, tol, max_iter if max_iter else 4 * self.n + 8, fixed_iter)
        self.weno = None
        if N >= 2 and N % 2 == 0:
            self.weno = Weno()
            if L.ob_weno_build(N, C.byref(self.basis), C.byref(self.weno)) != OB_OK:
                raise ValueError("oracle WENO build failed")

    # -- operator tables as numpy (views copied) --
    def table(self, name: str) -> np.ndarray:
        n, b = self.n, self.basis
        if name in ("xi", "w", "psi0", "psi1"):
            return np.array(getattr(b, name)[:n])
        if name == "P":
            return np.array([[b.P[j][k] for k in range(n)] for j in range(b.Ns)])
        m = getattr(b, name)
        return np.array([[m[i][j] for j in range(n)] for i in range(n)])

    def phi(self, x: float) -> np.ndarray:
        out = np.zeros(self.n)
        lib().ob_basis_eval(C.byref(self.basis), float(x), out)
        return out

    def set(self, **kw):
        for k, v in kw.items():
            setattr(self.params, k, v)
        return self

    # -- predictor --
    def predict_cell(self, u_cell, lam: float, nested: bool = False):
        u = _arr(u_cell, self.n * M)
        q = np.zeros(self.n * self.n * M)
        it = C.c_int(0)
        f = lib().ob_predict_cell_nested if nested else lib().ob_predict_cell
        rc = f(C.byref(self.basis), C.byref(self.params), lam, u, q, C.byref(it))
        return q.reshape(self.n, self.n, M), it.value, rc

    def predict(self, u, lam: float):
        u = _arr(u).reshape(-1, self.n, M)
        out = np.zeros((u.shape[0], self.n, self.n, M))
        iters = np.zeros(u.shape[0], dtype=np.int32)
        for i in range(u.shape[0]):
            out[i], iters[i], _ = self.predict_cell(u[i], lam)
        return out, iters

    # -- CFL --
    def dg_lambda_max(self, u, nodal: bool = False):
        u = _arr(u)
        f = lib().ob_dg_lambda_max_nodal if nodal else lib().ob_dg_lambda_max
        return f(C.byref(self.basis), self.params.gamma, u.size // (self.n * M), u)

    def dg_dt(self, u, dx):
        u = _arr(u)
        return lib().ob_dg_dt(C.byref(self.basis), C.byref(self.params), dx,
                              u.size // (self.n * M), u)

    def fv_dt(self, v, dx):
        v = _arr(v)
        return lib().ob_fv_dt(C.byref(self.params), dx, v.size // M, v)

    # -- DG --
    def dg_correct(self, u, q, dx, dt):
        u = _arr(u)
        q = _arr(q)
        out = np.zeros_like(u)
        nc = u.size // (self.n * M)
        rc = lib().ob_dg_correct(C.byref(self.basis), C.byref(self.params), nc, dx, dt, u, q, out)
        if rc != OB_OK:
            raise RuntimeError(f"ob_dg_correct rc={rc}")
        return out

    def dg_step(self, u, dx, dt, want_q: bool = False):
        u = _arr(u)
        nc = u.size // (self.n * M)
        out = np.zeros_like(u)
        q = np.zeros(nc * self.n * self.n * M) if want_q else None
        st = Stats()
        rc = lib().ob_dg_step(C.byref(self.basis), C.byref(self.params), nc, dx, dt, u, out,
                              q.ctypes.data if want_q else None, C.byref(st))
        return out, q, st, rc

    def dg_step_cells(self, u, dx, dt, cells):
        u = _arr(u)
        nc = u.size // (self.n * M)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros(cells.size * self.n * M)
        rc = lib().ob_dg_step_cells(C.byref(self.basis), C.byref(self.params), nc, dx, dt, u,
                                    cells, cells.size, out)
        return out.reshape(cells.size, self.n, M), rc

    # -- WENO / FV --
    def weno_reconstruct(self, v):
        v = _arr(v)
        nc = v.size // M
        out = np.zeros(nc * self.n * M)
        lib().ob_weno_reconstruct(C.byref(self.weno), nc, v, out)
        return out.reshape(nc, self.n, M)

    def weno_sigma(self, c):
        return lib().ob_weno_sigma(C.byref(self.weno), _arr(c, self.n))

    def weno_cell(self, v, i):
        v = _arr(v)
        out = np.zeros(self.n * M)
        om = np.zeros(3 * M)
        lib().ob_weno_cell(C.byref(self.weno), v.size // M, v, int(i), out, om.ctypes.data)
        return out.reshape(self.n, M), om.reshape(3, M)

    def fv_step(self, v, dx, dt):
        v = _arr(v)
        out = np.zeros_like(v)
        st = Stats()
        rc = lib().ob_fv_step(C.byref(self.basis), C.byref(self.weno), C.byref(self.params),
                              v.size // M, dx, dt, v, out, C.byref(st))
        return out, st, rc

    def fv_step_cells(self, v, dx, dt, cells):
        v = _arr(v)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros(cells.size * M)
        rc = lib().ob_fv_step_cells(C.byref(self.basis), C.byref(self.weno), C.byref(self.params),
                                    v.size // M, dx, dt, v, cells, cells.size, out)
        return out.reshape(cells.size, M), rc

    # -- time loop --
    def solve(self, scheme: str, u, dx, t_end: float = 0.0, max_steps: int = 0):
        u = np.array(u, dtype=np.float64, copy=True).ravel()
        nc = u.size // (self.n * M) if scheme == "dg" else u.size // M
        steps = C.c_int64(0)
        t = C.c_double(0.0)
        wp = C.cast(C.pointer(self.weno), C.c_void_p) if (scheme == "fv") else None
        rc = lib().ob_solve(0 if scheme == "dg" else 1, C.byref(self.basis), wp,
                            C.byref(self.params), nc, dx, u, t_end, max_steps, C.byref(steps),
                            C.byref(t))
        return u, steps.value, t.value, rc

    # -- boundaries and the a posteriori subcell limiter (ader_oracle_lim.c) --
    def r_matrix(self):
        R = np.zeros(self.n * self.basis.Ns)
        if lib().ob_r_matrix(C.byref(self.basis), R) != OB_OK:
            raise RuntimeError("ob_r_matrix failed")
        return R.reshape(self.n, self.basis.Ns)

    @staticmethod
    def lim_params(bc: str = "periodic", limiter: bool | int = True, delta0: float = 1e-4,
                   eps: float = 1e-3):
        """limiter: False / 0 off, True / 1 detect and recompute troubled cells, 2 every
        cell recomputed by the subcell ADER-WENO2 scheme"""
        return LimParams(1 if bc == "outflow" else 0, int(limiter), delta0, eps)

    def weno2(self, vm, v0, vp):
        """degree-1 WENO nodal values [2][3] on a subcell with averages v0 and
        neighbours vm, vp (the reconstruction of the subcell ADER-WENO2 scheme)"""
        w = np.zeros(2 * M)
        xi = Oracle(1).table("xi")
        lib().ob_lim_weno2(_arr(vm, M), _arr(v0, M), _arr(vp, M), _arr(xi, 2), w)
        return w.reshape(2, M)

    def dgl_step(self, u, dx, dt, bc: str = "periodic", limiter: bool = True,
                 delta0: float = 1e-4, eps: float = 1e-3):
        u = _arr(u)
        nc = u.size // (self.n * M)
        out = np.zeros_like(u)
        tr = np.zeros(nc, dtype=np.int32)
        st = Stats()
        lp = self.lim_params(bc, limiter, delta0, eps)
        rc = lib().ob_dgl_step(C.byref(self.basis), C.byref(self.params), C.byref(lp), nc, dx, dt,
                               u, out, tr.ctypes.data, C.byref(st))
        return out, tr, rc

    def dgl_solve(self, u, dx, t_end: float = 0.0, max_steps: int = 0, bc: str = "periodic",
                  limiter: bool = True):
        u = np.array(u, dtype=np.float64, copy=True).ravel()
        nc = u.size // (self.n * M)
        steps, t, ttot = C.c_int64(0), C.c_double(0.0), C.c_int64(0)
        lp = self.lim_params(bc, limiter)
        rc = lib().ob_dgl_solve(C.byref(self.basis), C.byref(self.params), C.byref(lp), nc, dx, u,
                                t_end, max_steps, C.byref(steps), C.byref(t), C.byref(ttot))
        return u, steps.value, t.value, rc, ttot.value

    # -- node coordinates of the DG representation (Sec. 1, eq. dg_repr) --
    def node_x(self, ncells: int, x0: float = 0.0, x1: float = 1.0) -> np.ndarray:
        dx = (x1 - x0) / ncells
        xi = self.table("xi")
        return x0 + dx * (np.arange(ncells)[:, None] + xi[None, :])


class ReactingOracle:
    """ADER-DG for the 1D two-component reacting flow (Sec. 2, eq. pdes_2_comps in
    1D): state [cell][k][5] = (rho, m, E, rho c1, rho c2), source
    (0, 0, 0, rho c2, -omega^2 rho c1); nested Picard predictor
    (eq. lst_dg_predictor_nested_picards) and the corrector's source term."""

    def __init__(self, N: int, omega: float = 1.0, gamma: float = 1.4, cfl: float = 0.4,
                 tol: float = 1e-13, max_iter: int | None = None, fixed_iter: int = 0):
        self.N, self.n = N, N + 1
        self.base = Oracle(N, gamma=gamma, cfl=cfl, tol=tol)
        self.basis = self.base.basis
        self.params = RSParams(gamma, omega, cfl, tol,
                               max_iter if max_iter else 4 * self.n + 8, fixed_iter)

    def table(self, name):
        return self.base.table(name)

    def set(self, **kw):
        for k, v in kw.items():
            setattr(self.params, k, v)
        return self

    def node_x(self, ncells, x0=0.0, x1=1.0):
        return self.base.node_x(ncells, x0, x1)

    def flux(self, U):
        F = np.zeros(MRS)
        lib().ob_rs_flux(self.params.gamma, _arr(U, MRS), F)
        return F

    def source(self, U):
        S = np.zeros(MRS)
        lib().ob_rs_source(self.params.omega, _arr(U, MRS), S)
        return S

    def rusanov(self, a, b):
        G = np.zeros(MRS)
        lib().ob_rs_rusanov(self.params.gamma, _arr(a, MRS), _arr(b, MRS), G)
        return G

    def predict_cell(self, u_cell, lam: float, dt: float, direct: bool = False):
        u = _arr(u_cell, self.n * MRS)
        q = np.zeros(self.n * self.n * MRS)
        it, inner = C.c_int(0), C.c_int(0)
        if direct:
            rc = lib().ob_rs_predict_cell_direct(C.byref(self.basis), C.byref(self.params), lam,
                                                 dt, u, q, C.byref(it))
        else:
            rc = lib().ob_rs_predict_cell(C.byref(self.basis), C.byref(self.params), lam, dt, u,
                                          q, C.byref(it), C.byref(inner))
        return q.reshape(self.n, self.n, MRS), it.value, inner.value, rc

    def predict(self, u, lam: float, dt: float):
        u = _arr(u).reshape(-1, self.n, MRS)
        out = np.zeros((u.shape[0], self.n, self.n, MRS))
        iters = np.zeros(u.shape[0], dtype=np.int32)
        for i in range(u.shape[0]):
            out[i], iters[i], _, _ = self.predict_cell(u[i], lam, dt)
        return out, iters

    def dg_dt(self, u, dx):
        u = _arr(u)
        return lib().ob_rs_dg_dt(C.byref(self.basis), C.byref(self.params), dx,
                                 u.size // (self.n * MRS), u)

    def dg_step(self, u, dx, dt, want_q: bool = False):
        u = _arr(u)
        nc = u.size // (self.n * MRS)
        out = np.zeros_like(u)
        q = np.zeros(nc * self.n * self.n * MRS) if want_q else None
        st = Stats()
        rc = lib().ob_rs_dg_step(C.byref(self.basis), C.byref(self.params), nc, dx, dt, u, out,
                                 q.ctypes.data if want_q else None, C.byref(st))
        return out, q, st, rc

    def dg_step_cells(self, u, dx, dt, cells):
        u = _arr(u)
        nc = u.size // (self.n * MRS)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros(cells.size * self.n * MRS)
        rc = lib().ob_rs_dg_step_cells(C.byref(self.basis), C.byref(self.params), nc, dx, dt, u,
                                       cells, cells.size, out)
        return out.reshape(cells.size, self.n, MRS), rc

    def solve(self, u, dx, t_end: float = 0.0, max_steps: int = 0, dt_fixed: float = 0.0):
        u = np.array(u, dtype=np.float64, copy=True).ravel()
        nc = u.size // (self.n * MRS)
        steps, t = C.c_int64(0), C.c_double(0.0)
        rc = lib().ob_rs_solve(C.byref(self.basis), C.byref(self.params), nc, dx, u, t_end,
                               max_steps, dt_fixed, C.byref(steps), C.byref(t))
        return u, steps.value, t.value, rc


def ode_errors(orc: "ReactingOracle", dt: float, nodes, locals_, t_end: float, omega: float = 1.0,
               npts: int = 25):
    """Errors of the ODE initial-value problem of Sec. 2.1 (eq. harm_osc, eq.
    epsilons_q): u1 = cos(omega t), u2 = -omega sin(omega t) against the species
    components (rho c1, rho c2) of a one-cell uniform solve.

    nodes: [K, 2] species values u^n at t_n = n dt, n = 1..K (the solution at
    time nodes); locals_: [K, n, 2] predictor time coefficients q_{l0} of step n
    (any xi node: the state is uniform).  Returns ((eps_L1, eps_L2, eps_Linf) at
    time nodes, (L1, L2, Linf) of the local solution over [0, t_end]), the
    integrals by the npts-point GL rule per step and vector norms summed over
    both components."""
    nodes = np.asarray(nodes)
    K = nodes.shape[0]
    t = dt * np.arange(1, K + 1)
    ex = np.stack([np.cos(omega * t), -omega * np.sin(omega * t)], 1)
    e = np.abs(nodes - ex).sum(1)
    glob = (float(dt * e.sum()), float(np.sqrt(dt * (e ** 2).sum())), float(e.max()))
    gx, gw = np.polynomial.legendre.leggauss(npts)
    gx, gw = 0.5 * (gx + 1.0), 0.5 * gw
    phi = np.stack([orc.base.phi(x) for x in gx])  # [npts, n]
    l1 = l2 = linf = 0.0
    for k in range(K):
        ts = dt * (k + gx)
        exk = np.stack([np.cos(omega * ts), -omega * np.sin(omega * ts)], 1)
        ek = np.abs(phi @ np.asarray(locals_[k]) - exk).sum(1)
        l1 += dt * float(gw @ ek)
        l2 += dt * float(gw @ ek ** 2)
        linf = max(linf, float(ek.max()))
    return glob, (l1, float(np.sqrt(l2)), linf)


# ---------------------------------------------------------------------------
# error norms of Sec. 2.1 (eq. epsilons) in 1D: 25-point Gauss-Legendre rule per cell
# ---------------------------------------------------------------------------

def dg_density_errors(orc: Oracle, u, rho_exact, x0: float = 0.0, x1: float = 1.0, npts: int = 25):
    """L1 and Linf errors of the density of a DG solution u[cell][k][r].

    rho_exact: callable x -> exact density (vectorised).  The L1 integral and
    the Linf maximum use the same npts Gauss-Legendre points in each cell.
    """
    u = np.asarray(u, dtype=np.float64).reshape(-1, orc.n, M)
    nc = u.shape[0]
    dx = (x1 - x0) / nc
    gx, gw = np.polynomial.legendre.leggauss(npts)
    gx = 0.5 * (gx + 1.0)
    gw = 0.5 * gw
    phi = np.stack([orc.phi(x) for x in gx])  # [npts, n]
    rho_h = u[:, :, 0] @ phi.T  # [nc, npts]
    xs = x0 + dx * (np.arange(nc)[:, None] + gx[None, :])
    err = np.abs(rho_h - rho_exact(xs))
    return float(dx * (err @ gw).sum()), float(err.max())


def fv_density_errors(v, rho_avg_exact, x0: float = 0.0, x1: float = 1.0):
    """L1 and Linf errors of FV cell averages against exact cell averages."""
    v = np.asarray(v, dtype=np.float64).reshape(-1, M)
    nc = v.shape[0]
    dx = (x1 - x0) / nc
    edges = x0 + dx * np.arange(nc + 1)
    err = np.abs(v[:, 0] - rho_avg_exact(edges[:-1], edges[1:]))
    return float(dx * err.sum()), float(err.max())


def order(e1: float, e2: float, h1: float, h2: float) -> float:
    """Empirical convergence order p = ln(e1/e2)/ln(h1/h2)."""
    return float(np.log(e1 / e2) / np.log(h1 / h2))


# ---------------------------------------------------------------------------
# 2D Euler on a periodic Cartesian mesh (ader_oracle_2d.c)
# ---------------------------------------------------------------------------

class Oracle2D:
    """ADER-DG for the 2D Euler equations on [x0, x1] x [y0, y1], periodic: state
    u[iy][ix][k1][k2][r] (k1 the xi node, k2 the eta node, r = rho, m_x, m_y, E),
    the tensor-product predictor of Sec. 1.1 and the corrector of Sec. 1.2."""

    def __init__(self, N: int, gamma: float = 1.4, cfl: float = 0.4, tol: float = 1e-13,
                 max_iter: int | None = None, fixed_iter: int = 0):
        self.base = Oracle(N, gamma=gamma, cfl=cfl, tol=tol, max_iter=max_iter,
                           fixed_iter=fixed_iter)
        self.N, self.n = N, N + 1
        self.basis, self.params = self.base.basis, self.base.params

    def table(self, name):
        return self.base.table(name)

    def set(self, **kw):
        self.base.set(**kw)
        return self

    def node_xy(self, nx: int, ny: int, x0=0.0, x1=1.0, y0=0.0, y1=1.0):
        """(X, Y) of shape [ny][nx][n][n] (k1 along x, k2 along y)."""
        xi = self.table("xi")
        dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
        X = x0 + dx * (np.arange(nx)[None, :, None, None] + xi[None, None, :, None])
        Y = y0 + dy * (np.arange(ny)[:, None, None, None] + xi[None, None, None, :])
        return np.broadcast_to(X, (ny, nx, self.n, self.n)), np.broadcast_to(Y, (ny, nx, self.n, self.n))

    def flux(self, U):
        F, G = np.zeros(M2), np.zeros(M2)
        lib().ob2_flux(self.params.gamma, _arr(U, M2), F, G)
        return F, G

    def rusanov(self, direction: int, a, b):
        H = np.zeros(M2)
        lib().ob2_rusanov(self.params.gamma, direction, _arr(a, M2), _arr(b, M2), H)
        return H

    def predict_cell(self, u_cell, lx: float, ly: float):
        q = np.zeros(self.n ** 3 * M2)
        it = C.c_int(0)
        rc = lib().ob2_predict_cell(C.byref(self.basis), C.byref(self.params), lx, ly,
                                    _arr(u_cell, self.n * self.n * M2), q, C.byref(it))
        return q.reshape(self.n, self.n, self.n, M2), it.value, rc

    def step(self, u, nx: int, ny: int, dx: float, dy: float, dt: float):
        u = _arr(u).ravel()
        out = np.zeros_like(u)
        st = Stats()
        rc = lib().ob2_dg_step(C.byref(self.basis), C.byref(self.params), nx, ny, dx, dy, dt, u,
                               out, C.byref(st))
        return out, rc, st.mean_iters

    def step_cells(self, u, nx: int, ny: int, dx: float, dy: float, dt: float, cells):
        """u^{n+1} of the listed cells only: [count][n][n][4]"""
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros(cells.size * self.n * self.n * M2)
        rc = lib().ob2_dg_step_cells(C.byref(self.basis), C.byref(self.params), nx, ny, dx, dy, dt,
                                     _arr(u).ravel(), cells, cells.size, out)
        return out.reshape(cells.size, self.n, self.n, M2), rc

    def dt(self, u, nx: int, ny: int, dx: float, dy: float) -> float:
        return lib().ob2_dt(C.byref(self.basis), C.byref(self.params), nx, ny, dx, dy,
                            _arr(u).ravel())

    def solve(self, u, nx: int, ny: int, dx: float, dy: float, t_end: float = 0.0,
              max_steps: int = 0):
        u = np.array(u, dtype=np.float64, copy=True).ravel()
        steps, t = C.c_int64(0), C.c_double(0.0)
        rc = lib().ob2_solve(C.byref(self.basis), C.byref(self.params), nx, ny, dx, dy, u, t_end,
                             max_steps, C.byref(steps), C.byref(t))
        return u, steps.value, t.value, rc


def dg2_density_errors(orc: Oracle2D, u, nx: int, ny: int, rho_exact, x0=0.0, x1=1.0, y0=0.0,
                       y1=1.0, npts: int = 25):
    """L1, L2 and Linf errors of the density of a 2D DG solution (eq. epsilons):
    the npts x npts Gauss-Legendre rule per cell for the integrals, Linf over the
    same points."""
    u = np.asarray(u, dtype=np.float64).reshape(ny, nx, orc.n, orc.n, M2)
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    gx, gw = np.polynomial.legendre.leggauss(npts)
    gx, gw = 0.5 * (gx + 1.0), 0.5 * gw
    phi = np.stack([orc.base.phi(x) for x in gx])  # [npts, n]
    rho_h = np.einsum("ak,bl,yxkl->yxab", phi, phi, u[..., 0])
    X = x0 + dx * (np.arange(nx)[None, :, None, None] + gx[None, None, :, None])
    Y = y0 + dy * (np.arange(ny)[:, None, None, None] + gx[None, None, None, :])
    err = np.abs(rho_h - rho_exact(X, Y))
    wts = dx * dy * np.outer(gw, gw)
    l1 = float((err * wts).sum())
    l2 = float(np.sqrt((err ** 2 * wts).sum()))
    return l1, l2, float(err.max())


# ---------------------------------------------------------------------------
# 3D Euler on a periodic Cartesian mesh (ader_oracle_3d.c)
# ---------------------------------------------------------------------------

class Oracle3D:
    """ADER-DG for the 3D Euler equations on a periodic box: state
    u[iz][iy][ix][k1][k2][k3][r] (r = rho, m_x, m_y, m_z, E), the tensor-product
    predictor of Sec. 1.1 and the corrector of Sec. 1.2."""

    def __init__(self, N: int, gamma: float = 1.4, cfl: float = 0.4, tol: float = 1e-13,
                 max_iter: int | None = None, fixed_iter: int = 0):
        self.base = Oracle(N, gamma=gamma, cfl=cfl, tol=tol, max_iter=max_iter,
                           fixed_iter=fixed_iter)
        self.N, self.n = N, N + 1
        self.basis, self.params = self.base.basis, self.base.params

    def table(self, name):
        return self.base.table(name)

    def node_xyz(self, nx: int, ny: int, nz: int, box=(1.0, 1.0, 1.0)):
        """(X, Y, Z), each [nz][ny][nx][n][n][n] (k1 along x, k2 along y, k3 along z)."""
        xi, n = self.table("xi"), self.n
        shape = (nz, ny, nx, n, n, n)
        X = box[0] / nx * (np.arange(nx)[None, None, :, None, None, None]
                           + xi[None, None, None, :, None, None])
        Y = box[1] / ny * (np.arange(ny)[None, :, None, None, None, None]
                           + xi[None, None, None, None, :, None])
        Z = box[2] / nz * (np.arange(nz)[:, None, None, None, None, None]
                           + xi[None, None, None, None, None, :])
        return tuple(np.broadcast_to(A, shape).copy() for A in (X, Y, Z))

    def flux(self, U):
        F = np.zeros(3 * M3)
        lib().ob3_flux(self.params.gamma, _arr(U, M3), F)
        return F.reshape(3, M3)

    def rusanov(self, direction: int, a, b):
        H = np.zeros(M3)
        lib().ob3_rusanov(self.params.gamma, direction, _arr(a, M3), _arr(b, M3), H)
        return H

    def predict_cell(self, u_cell, lx: float, ly: float, lz: float):
        q = np.zeros(self.n ** 4 * M3)
        it = C.c_int(0)
        rc = lib().ob3_predict_cell(C.byref(self.basis), C.byref(self.params), lx, ly, lz,
                                    _arr(u_cell, self.n ** 3 * M3), q, C.byref(it))
        return q.reshape(self.n, self.n, self.n, self.n, M3), it.value, rc

    def step(self, u, dims, h, dt: float):
        u = _arr(u).ravel()
        out = np.zeros_like(u)
        st = Stats()
        rc = lib().ob3_dg_step(C.byref(self.basis), C.byref(self.params), *dims, *h, dt, u, out,
                               C.byref(st))
        return out, rc, st.mean_iters

    def step_cells(self, u, dims, h, dt: float, cells):
        """u^{n+1} of the listed cells only: [count][n][n][n][5]"""
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros(cells.size * self.n ** 3 * M3)
        rc = lib().ob3_dg_step_cells(C.byref(self.basis), C.byref(self.params), *dims, *h, dt,
                                     _arr(u).ravel(), cells, cells.size, out)
        return out.reshape(cells.size, self.n, self.n, self.n, M3), rc

    def dt(self, u, dims, h) -> float:
        return lib().ob3_dt(C.byref(self.basis), C.byref(self.params), *dims, *h, _arr(u).ravel())

    def solve(self, u, dims, h, t_end: float = 0.0, max_steps: int = 0):
        u = np.array(u, dtype=np.float64, copy=True).ravel()
        steps, t = C.c_int64(0), C.c_double(0.0)
        rc = lib().ob3_solve(C.byref(self.basis), C.byref(self.params), *dims, *h, u, t_end,
                             max_steps, C.byref(steps), C.byref(t))
        return u, steps.value, t.value, rc


def dg3_density_errors(orc: Oracle3D, u, dims, rho_exact, npts: int = 10):
    """L1, L2 and Linf density errors of a 3D DG solution on the unit box (eq.
    epsilons) with an npts^3 Gauss-Legendre rule per cell."""
    nx, ny, nz = dims
    n = orc.n
    u = np.asarray(u, dtype=np.float64).reshape(nz, ny, nx, n, n, n, M3)
    gx, gw = np.polynomial.legendre.leggauss(npts)
    gx, gw = 0.5 * (gx + 1.0), 0.5 * gw
    phi = np.stack([orc.base.phi(x) for x in gx])
    rho_h = np.einsum("ak,bl,cm,zyxklm->zyxabc", phi, phi, phi, u[..., 0])
    X = (np.arange(nx)[None, None, :, None, None, None] + gx[None, None, None, :, None, None]) / nx
    Y = (np.arange(ny)[None, :, None, None, None, None] + gx[None, None, None, None, :, None]) / ny
    Z = (np.arange(nz)[:, None, None, None, None, None] + gx[None, None, None, None, None, :]) / nz
    err = np.abs(rho_h - rho_exact(X, Y, Z))
    wts = np.einsum("a,b,c->abc", gw, gw, gw) / (nx * ny * nz)
    return float((err * wts).sum()), float(np.sqrt((err ** 2 * wts).sum())), float(err.max())


# ---------------------------------------------------------------------------
# non-conservative product: Euler + passive tracer (ader_oracle_nc.c)
# ---------------------------------------------------------------------------

class NCOracle:
    """ADER-DG for the 1D Euler equations with a passive tracer in non-conservative
    form (U = rho, m, E, phi; B(U) dU/dx = (0, 0, 0, u dphi/dx)), periodic; state
    u[cell][k][4]."""

    def __init__(self, N: int, gamma: float = 1.4, cfl: float = 0.4, tol: float = 1e-13,
                 max_iter: int | None = None, fixed_iter: int = 0):
        self.base = Oracle(N, gamma=gamma, cfl=cfl, tol=tol, max_iter=max_iter,
                           fixed_iter=fixed_iter)
        self.N, self.n = N, N + 1
        self.basis, self.params = self.base.basis, self.base.params

    def table(self, name):
        return self.base.table(name)

    def node_x(self, ncells, x0=0.0, x1=1.0):
        return self.base.node_x(ncells, x0, x1)

    def flux(self, U):
        F = np.zeros(MNC)
        lib().ob_nc_flux(self.params.gamma, _arr(U, MNC), F)
        return F

    def face(self, a, b):
        G, bt = np.zeros(MNC), C.c_double(0.0)
        lib().ob_nc_face(self.params.gamma, _arr(a, MNC), _arr(b, MNC), G, C.byref(bt))
        return G, bt.value

    def predict_cell(self, u_cell, lam: float):
        q = np.zeros(self.n * self.n * MNC)
        it = C.c_int(0)
        rc = lib().ob_nc_predict_cell(C.byref(self.basis), C.byref(self.params), lam,
                                      _arr(u_cell, self.n * MNC), q, C.byref(it))
        return q.reshape(self.n, self.n, MNC), it.value, rc

    def step(self, u, dx: float, dt: float):
        u = _arr(u).ravel()
        out = np.zeros_like(u)
        st = Stats()
        nc = u.size // (self.n * MNC)
        rc = lib().ob_nc_step(C.byref(self.basis), C.byref(self.params), nc, dx, dt, u, out,
                              C.byref(st))
        return out, rc, st.mean_iters

    def dt(self, u, dx: float) -> float:
        u = _arr(u).reshape(-1, self.n, MNC)
        return self.base.dg_dt(np.ascontiguousarray(u[..., :3]), dx)

    def solve(self, u, dx: float, t_end: float = 0.0, max_steps: int = 0):
        u = np.array(u, dtype=np.float64, copy=True).ravel()
        nc = u.size // (self.n * MNC)
        steps, t = C.c_int64(0), C.c_double(0.0)
        rc = lib().ob_nc_solve(C.byref(self.basis), C.byref(self.params), nc, dx, u, t_end,
                               max_steps, C.byref(steps), C.byref(t))
        return u, steps.value, t.value, rc
