"""ctypes wrapper of the plain FP64 SuperSCS reference (superscs_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA implementation; problems are passed in as plain numpy arrays.

Paper: Sopasakis, Menounou, Patrinos, "SuperSCS: fast and accurate large-scale
conic optimization" (arXiv 1903.06477).  Each wrapped routine cites the
section it follows in the C source.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "superscs_oracle.c")
_LIB = os.path.join(_HERE, "libsuperscs_oracle.so")

SOLVED, INFEASIBLE, UNBOUNDED, MAX_ITERS, NUMERICAL = 1, -1, -2, -3, -5
DIR_AA, DIR_RB, DIR_NONE, DIR_AA_QR = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "superscs_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("m", C.c_int32),
        ("Ap", C.POINTER(C.c_int64)), ("Ai", C.POINTER(C.c_int32)), ("Ax", C.POINTER(C.c_double)),
        ("b", C.POINTER(C.c_double)), ("c", C.POINTER(C.c_double)),
        ("f", C.c_int32), ("l", C.c_int32),
        ("nq", C.c_int32), ("q", C.POINTER(C.c_int32)),
        ("ns", C.c_int32), ("s", C.POINTER(C.c_int32)),
        ("ep", C.c_int32), ("ed", C.c_int32),
    ]


class _Settings(C.Structure):
    _fields_ = [
        ("direction", C.c_int32), ("mem", C.c_int32),
        ("eps", C.c_double), ("c0", C.c_double), ("c1", C.c_double), ("q", C.c_double),
        ("sigma", C.c_double), ("lam", C.c_double), ("thetabar", C.c_double),
        ("max_iters", C.c_int32), ("ls_max", C.c_int32), ("cg_max", C.c_int32),
        ("check_every", C.c_int32),
        ("cg_rtol", C.c_double), ("aa_reg", C.c_double),
        ("warm_u", C.POINTER(C.c_double)),
        ("cg_adapt", C.c_double),
    ]


class _Info(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("iters", C.c_int32), ("k0", C.c_int32), ("k1", C.c_int32),
        ("k2", C.c_int32), ("backtracks", C.c_int32), ("cg_iters", C.c_int64),
        ("pr", C.c_double), ("dr", C.c_double), ("gap", C.c_double), ("ic", C.c_double),
        ("uc", C.c_double), ("pobj", C.c_double), ("dobj", C.c_double), ("nRu", C.c_double),
    ]


class _Trace(C.Structure):
    _fields_ = [
        ("cap", C.c_int32), ("len", C.c_int32),
        ("nRu", C.POINTER(C.c_double)), ("step", C.POINTER(C.c_int32)),
        ("alpha", C.POINTER(C.c_double)), ("u_dist", C.POINTER(C.c_double)),
        ("ustar", C.POINTER(C.c_double)),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int32)
        L.orc_proj_soc.argtypes = [dp, C.c_int32]
        L.orc_jacobi_eig.argtypes = [C.c_int32, dp, dp, dp]
        L.orc_proj_psd.argtypes = [dp, C.c_int32]
        L.orc_proj_exp.argtypes = [dp]
        L.orc_proj_exp_dual.argtypes = [dp]
        L.orc_in_exp.argtypes = [dp, C.c_double]
        L.orc_in_exp_dual.argtypes = [dp, C.c_double]
        L.orc_svec_to_mat.argtypes = [C.c_int32, dp, dp]
        L.orc_mat_to_svec.argtypes = [C.c_int32, dp, dp]
        for name in ("orc_proj_dual_cone", "orc_proj_primal_cone"):
            getattr(L, name).argtypes = [C.POINTER(_Problem), dp]
        L.orc_proj_C.argtypes = [C.POINTER(_Problem), dp, dp]
        L.orc_setup.argtypes = [C.POINTER(_Problem), C.POINTER(_Settings)]
        L.orc_setup.restype = C.c_void_p
        L.orc_finish.argtypes = [C.c_void_p]
        L.orc_linsys.argtypes = [C.c_void_p, dp, dp, C.c_int32, ip]
        L.orc_apply_T.argtypes = [C.c_void_p, dp, dp, dp]
        L.orc_termination.argtypes = [C.c_void_p, dp, dp, dp, C.c_double, C.POINTER(_Info)]
        L.orc_solve.argtypes = [C.c_void_p, dp, dp, dp, dp, C.POINTER(_Info), C.POINTER(_Trace)]
        L.orc_dir_new.argtypes = [C.c_int32, C.c_int64, C.c_int32, C.c_double, C.c_double]
        L.orc_dir_new.restype = C.c_void_p
        L.orc_dir_free.argtypes = [C.c_void_p]
        L.orc_dir_compute.argtypes = [C.c_void_p, dp, dp, dp, C.c_int32, dp]
        L.orc_dir_count.argtypes = [C.c_void_p]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


DEFAULTS = dict(direction=DIR_AA, mem=10, eps=1e-5, c0=0.99, c1=0.99, q=0.99, sigma=1e-2, lam=1.0,
                thetabar=0.1, max_iters=2000, ls_max=20, cg_max=1000, check_every=1,
                cg_rtol=1e-12, aa_reg=1e-10, cg_adapt=0.0)


@dataclass
class Info:
    status: int
    iters: int
    k0: int
    k1: int
    k2: int
    backtracks: int
    cg_iters: int
    pr: float
    dr: float
    gap: float
    ic: float
    uc: float
    pobj: float
    dobj: float
    nRu: float


def _info(ci: _Info) -> Info:
    return Info(*(getattr(ci, f) for f, _ in _Info._fields_))


class Oracle:
    """One problem set up in the oracle.  ``prob`` is a dict with keys
    A (scipy CSR, m x n), b, c, f, l, q (list), s (list)."""

    def __init__(self, prob: dict, **settings):
        L = lib()
        A = prob["A"]
        self.n, self.m = A.shape[1], A.shape[0]
        self.N = self.n + self.m + 1
        self._keep = dict(
            Ap=np.ascontiguousarray(A.indptr, dtype=np.int64),
            Ai=np.ascontiguousarray(A.indices, dtype=np.int32),
            Ax=np.ascontiguousarray(A.data, dtype=np.float64),
            b=np.ascontiguousarray(prob["b"], dtype=np.float64),
            c=np.ascontiguousarray(prob["c"], dtype=np.float64),
            q=np.ascontiguousarray(prob.get("q", []) or [0], dtype=np.int32),
            s=np.ascontiguousarray(prob.get("s", []) or [0], dtype=np.int32),
        )
        k = self._keep
        self.P = _Problem(
            self.n, self.m,
            k["Ap"].ctypes.data_as(C.POINTER(C.c_int64)), _ip(k["Ai"]), _dp(k["Ax"]),
            _dp(k["b"]), _dp(k["c"]),
            int(prob.get("f", 0)), int(prob.get("l", 0)),
            len(prob.get("q", [])), _ip(k["q"]), len(prob.get("s", [])), _ip(k["s"]),
            int(prob.get("ep", 0)), int(prob.get("ed", 0)),
        )
        st = dict(DEFAULTS)
        warm = settings.pop("warm_u", None)
        st.update(settings)
        self.settings = st
        self.S = _Settings(**{f: st[f] for f, _ in _Settings._fields_ if f != "warm_u"})
        if warm is not None:
            self._warm = np.ascontiguousarray(warm, dtype=np.float64)
            self.S.warm_u = _dp(self._warm)
        self.W = L.orc_setup(C.byref(self.P), C.byref(self.S))
        if not self.W:
            raise ValueError("oracle setup rejected the problem")

    def close(self):
        if getattr(self, "W", None):
            lib().orc_finish(self.W)
            self.W = None

    def __del__(self):
        self.close()

    # --- single operators -------------------------------------------------
    def linsys(self, r, slot=0):
        r = np.ascontiguousarray(r, dtype=np.float64)
        out = np.empty(self.N)
        it = C.c_int32(0)
        lib().orc_linsys(self.W, _dp(r), _dp(out), slot, C.byref(it))
        return out

    def apply_T(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        Tu, Ru = np.empty(self.N), np.empty(self.N)
        lib().orc_apply_T(self.W, _dp(u), _dp(Tu), _dp(Ru))
        return Tu, Ru

    def proj_C(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.empty(self.N)
        lib().orc_proj_C(C.byref(self.P), _dp(v), _dp(out))
        return out

    def proj_dual_cone(self, v):
        out = np.array(v, dtype=np.float64, copy=True)
        lib().orc_proj_dual_cone(C.byref(self.P), _dp(out))
        return out

    def proj_primal_cone(self, v):
        out = np.array(v, dtype=np.float64, copy=True)
        lib().orc_proj_primal_cone(C.byref(self.P), _dp(out))
        return out

    def termination(self, u, ut, ub, eps):
        ci = _Info()
        st = lib().orc_termination(self.W, _dp(np.ascontiguousarray(u)), _dp(np.ascontiguousarray(ut)),
                                   _dp(np.ascontiguousarray(ub)), eps, C.byref(ci))
        return st, _info(ci)

    # --- Algorithm 1 --------------------------------------------------------
    def solve(self, trace_cap=0, ustar=None):
        x, y, s = np.empty(self.n), np.empty(self.m), np.empty(self.m)
        u = np.empty(self.N)
        ci = _Info()
        tr = None
        trace = None
        if trace_cap > 0:
            tr = dict(nRu=np.zeros(trace_cap), step=np.zeros(trace_cap, np.int32),
                      alpha=np.zeros(trace_cap), u_dist=np.zeros(trace_cap))
            us = None if ustar is None else np.ascontiguousarray(ustar, dtype=np.float64)
            tr["_ustar"] = us
            trace = _Trace(trace_cap, 0, _dp(tr["nRu"]), _ip(tr["step"]), _dp(tr["alpha"]),
                           _dp(tr["u_dist"]), _dp(us) if us is not None else None)
        lib().orc_solve(self.W, _dp(x), _dp(y), _dp(s), _dp(u), C.byref(ci),
                        C.byref(trace) if trace is not None else None)
        out = dict(x=x, y=y, s=s, u=u, info=_info(ci))
        if tr is not None:
            k = trace.len
            out["trace"] = {key: val[:k] for key, val in tr.items() if not key.startswith("_")}
        return out


# --- standalone cone routines (Sec. 2) ---------------------------------------
def proj_soc(z):
    z = np.array(z, dtype=np.float64, copy=True)
    lib().orc_proj_soc(_dp(z), len(z))
    return z


def proj_exp(v):
    """Pi on the exponential cone of Sec. 2, cone (v), order (x1, x2, x3)."""
    v = np.array(v, dtype=np.float64, copy=True)
    lib().orc_proj_exp(_dp(v))
    return v


def proj_exp_dual(v):
    v = np.array(v, dtype=np.float64, copy=True)
    lib().orc_proj_exp_dual(_dp(v))
    return v


def in_exp(v, tol=0.0):
    return bool(lib().orc_in_exp(_dp(np.ascontiguousarray(v, dtype=np.float64)), tol))


def in_exp_dual(v, tol=0.0):
    return bool(lib().orc_in_exp_dual(_dp(np.ascontiguousarray(v, dtype=np.float64)), tol))


def proj_psd(v, d):
    v = np.array(v, dtype=np.float64, copy=True)
    lib().orc_proj_psd(_dp(v), d)
    return v


def jacobi_eig(X):
    X = np.ascontiguousarray(X, dtype=np.float64)
    d = X.shape[0]
    lam, V = np.empty(d), np.empty((d, d))
    lib().orc_jacobi_eig(d, _dp(X), _dp(lam), _dp(V))
    return lam, V


def svec_to_mat(v, d):
    v = np.ascontiguousarray(v, dtype=np.float64)
    X = np.empty((d, d))
    lib().orc_svec_to_mat(d, _dp(v), _dp(X))
    return X


def mat_to_svec(X):
    X = np.ascontiguousarray(X, dtype=np.float64)
    d = X.shape[0]
    v = np.empty(d * (d + 1) // 2)
    lib().orc_mat_to_svec(d, _dp(X), _dp(v))
    return v


class Direction:
    """Stateful RB (Algorithm 2) or AA (Sec. 4.4.2) direction for pins."""

    def __init__(self, kind, N, mem, thetabar=0.1, aa_reg=1e-10):
        self.N = N
        self.D = lib().orc_dir_new(kind, N, mem, thetabar, aa_reg)

    def __call__(self, Ru, z=None, xi=None):
        have = z is not None
        Ru = np.ascontiguousarray(Ru, dtype=np.float64)
        zz = np.ascontiguousarray(z if have else np.zeros(self.N), dtype=np.float64)
        xx = np.ascontiguousarray(xi if have else np.zeros(self.N), dtype=np.float64)
        d = np.empty(self.N)
        lib().orc_dir_compute(self.D, _dp(Ru), _dp(zz), _dp(xx), int(have), _dp(d))
        return d

    @property
    def count(self):
        return lib().orc_dir_count(self.D)

    def __del__(self):
        if getattr(self, "D", None):
            lib().orc_dir_free(self.D)
            self.D = None
