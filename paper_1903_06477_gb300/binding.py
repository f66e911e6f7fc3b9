"""Thin ctypes binding of libsuperscs.so (include/superscs.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Loading fails loudly if the library has not been built; there
is no CPU fallback.  Vectors may be numpy arrays (host) or CUDA torch tensors
(device); the library copies with unified addressing either way.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsuperscs.so")

SCS_OK, SCS_EINVAL, SCS_ENOMEM, SCS_ECUDA, SCS_ETIMEOUT = 0, -1, -2, -3, -4
SOLVED, INFEASIBLE, UNBOUNDED, MAX_ITERS, TIME_LIMIT, NUMERICAL = 1, -1, -2, -3, -4, -5
DIR_AA, DIR_RB, DIR_NONE, DIR_AA_QR = 0, 1, 2, 3
FP64, MIXED = 0, 1
TEAM_AUTO, TEAM_BLOCK, TEAM_GRID = 0, 1, 2


class Cone(C.Structure):
    _fields_ = [("f", C.c_int32), ("l", C.c_int32), ("nq", C.c_int32), ("q", C.POINTER(C.c_int32)),
                ("ns", C.c_int32), ("s", C.POINTER(C.c_int32)), ("ep", C.c_int32), ("ed", C.c_int32)]


class Data(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("Ap", C.POINTER(C.c_int64)), ("Ai", C.POINTER(C.c_int32)),
                ("Ax", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double)), ("c", C.POINTER(C.c_double))]


class Settings(C.Structure):
    _fields_ = [
        ("direction", C.c_int32), ("mem", C.c_int32), ("eps", C.c_double),
        ("c0", C.c_double), ("c1", C.c_double), ("q", C.c_double), ("sigma", C.c_double),
        ("lam", C.c_double), ("thetabar", C.c_double),
        ("max_iters", C.c_int32), ("ls_max", C.c_int32), ("cg_max", C.c_int32), ("check_every", C.c_int32),
        ("cg_rtol", C.c_double), ("time_limit_s", C.c_double),
        ("precision", C.c_int32), ("warm", C.c_int32), ("warm_u", C.c_void_p), ("verbose", C.c_int32),
        ("aa_reg", C.c_double), ("team", C.c_int32), ("threads", C.c_int32),
        ("mixed_cg_rtol", C.c_double), ("mixed_stall", C.c_int32), ("mixed_max_iters", C.c_int32),
        ("mixed_switch", C.c_double), ("cg_adapt", C.c_double), ("spmv_path", C.c_int32),
        ("warm_fallback", C.c_int32), ("mixed_resume", C.c_int32), ("mixed_refine", C.c_int32),
        ("linsys_direct", C.c_int32), ("mixed_stall_after_tau", C.c_int32), ("psd_recheck_tol", C.c_double),
    ]


class Info(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("iters", C.c_int32), ("k0", C.c_int32), ("k1", C.c_int32), ("k2", C.c_int32),
        ("backtracks", C.c_int32), ("cg_iters", C.c_int64),
        ("pr", C.c_double), ("dr", C.c_double), ("gap", C.c_double), ("ic", C.c_double), ("uc", C.c_double),
        ("pobj", C.c_double), ("dobj", C.c_double), ("setup_s", C.c_double), ("solve_s", C.c_double),
        ("err_vs_fp64", C.c_double), ("iters_fp32", C.c_int32), ("device_error", C.c_int32),
        ("kernel_s", C.c_double * 2), ("mat_passes", C.c_int64 * 2), ("cg_iters_fp32", C.c_int64),
        ("psd_resid_fp32", C.c_double), ("threads_per_block", C.c_int32), ("warm_fallback_taken", C.c_int32),
        ("kkt_fp32", C.c_double), ("mat_passes_ir", C.c_int64), ("cg_iters_ir", C.c_int64),
        ("ir_sweeps", C.c_int64), ("batch_device_s", C.c_double), ("team", C.c_int32),
        ("part_s", (C.c_double * 5) * 2), ("psd_redo_fp32", C.c_int64),
    ]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        for k in ("kernel_s", "mat_passes"):
            d[k] = list(d[k])
        d["part_s"] = [list(r) for r in d["part_s"]]
        return d


class SCSError(RuntimeError):
    pass


_lib = None

# (name, restype, argtypes) of every exported entry point of include/superscs.h and superscs_mlp.h
_SIGS = [
    ("scs_default_settings", C.c_int, [C.POINTER(Settings)]),
    ("scs_setup", C.c_int, [C.POINTER(Data), C.POINTER(Cone), C.POINTER(Settings), C.c_void_p, C.POINTER(C.c_void_p)]),
    ("scs_solve", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Info)]),
    ("scs_update_bc", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("scs_get_u", C.c_int, [C.c_void_p, C.c_void_p]),
    ("scs_set_warm", C.c_int, [C.c_void_p, C.c_void_p]),
    ("scs_linsys", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    ("scs_project_cone", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("scs_project_cone_prec", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("scs_apply_T", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("scs_profile", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]),
    ("scs_spmv", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("scs_cb_layout_check", C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                      C.c_int32, C.c_int32, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    ("scs_tile_layout_check", C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                        C.c_int32, C.c_int32, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p,
                                        C.c_void_p]),
    ("scs_residuals", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("scs_residuals_noalloc", C.c_int, [C.c_int32, C.c_int32] + [C.c_void_p] * 10),
    ("scs_finish", None, [C.c_void_p]),
    ("scs_last_error", C.c_char_p, [C.c_void_p]),
    ("scs_batch_setup", C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.POINTER(Settings), C.c_void_p,
                                  C.POINTER(C.c_void_p)]),
    ("scs_batch_solve", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Info)]),
    ("scs_batch_finish", None, [C.c_void_p]),
    ("scs_batch_setup_shared", C.c_int, [C.c_int32, C.POINTER(Data), C.POINTER(Cone), C.c_void_p, C.c_void_p,
                                         C.POINTER(Settings), C.c_void_p, C.POINTER(C.c_void_p)]),
    ("scs_batch_set_warm", C.c_int, [C.c_void_p, C.c_void_p]),
    ("scs_solve_batch", C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.POINTER(Settings), C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Info)]),
    ("scs_mlp_create", C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.c_void_p,
                                 C.POINTER(C.c_void_p)]),
    ("scs_mlp_fit_normalization", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    ("scs_mlp_train_step", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float,
                                     C.POINTER(C.c_float)]),
    ("scs_mlp_forward", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    ("scs_mlp_gradients", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                    C.POINTER(C.c_float)]),
    ("scs_mlp_num_params", C.c_int64, [C.c_void_p]),
    ("scs_mlp_get_params", C.c_int, [C.c_void_p, C.c_void_p]),
    ("scs_mlp_set_params", C.c_int, [C.c_void_p, C.c_void_p]),
    ("scs_mlp_destroy", None, [C.c_void_p]),
    ("scs_mlp_set_gemm", C.c_int, [C.c_void_p, C.c_int32]),
    ("scs_mlp_gemm_nt", C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                                  C.c_int32, C.c_void_p, C.c_int32, C.c_void_p]),
    ("scs_mlp_read", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                               C.POINTER(C.c_int32)]),
]


def lib():
    """Load libsuperscs.so; raise if it is missing (build it with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise SCSError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error(work=None) -> str:
    msg = lib().scs_last_error(work)
    return msg.decode() if msg else ""


def _check(rc, work=None):
    if rc != SCS_OK:
        raise SCSError(f"superscs error {rc}: {last_error(work)}")


def default_settings(**kw) -> Settings:
    s = Settings()
    _check(lib().scs_default_settings(C.byref(s)))
    for k, v in kw.items():
        if k == "lambda":
            k = "lam"
        if not hasattr(s, k):
            raise KeyError(k)
        setattr(s, k, v)
    return s


def _ptr(a):
    """Address of a numpy array or a torch tensor (host or CUDA)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


class _Keep:
    """Holds the numpy buffers behind a Data/Cone pair."""

    def __init__(self, prob):
        A = prob["A"]
        self.m, self.n = A.shape
        self.Ap = np.ascontiguousarray(A.indptr, dtype=np.int64)
        self.Ai = np.ascontiguousarray(A.indices, dtype=np.int32)
        self.Ax = np.ascontiguousarray(A.data, dtype=np.float64)
        self.b = np.ascontiguousarray(prob["b"], dtype=np.float64)
        self.c = np.ascontiguousarray(prob["c"], dtype=np.float64)
        self.q = np.ascontiguousarray(list(prob.get("q", [])) or [0], dtype=np.int32)
        self.s = np.ascontiguousarray(list(prob.get("s", [])) or [0], dtype=np.int32)
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
        self.data = Data(self.m, self.n, self.Ap.ctypes.data_as(C.POINTER(C.c_int64)), ip(self.Ai), dp(self.Ax),
                         dp(self.b), dp(self.c))
        self.cone = Cone(int(prob.get("f", 0)), int(prob.get("l", 0)), len(prob.get("q", [])), ip(self.q),
                         len(prob.get("s", [])), ip(self.s), int(prob.get("ep", 0)), int(prob.get("ed", 0)))


class Work:
    """One problem set up on the device (scs_setup ... scs_finish)."""

    def __init__(self, prob, settings: Settings | None = None, stream=None, **kw):
        L = lib()
        self._keep = _Keep(prob)
        self.n, self.m = self._keep.n, self._keep.m
        self.N = self.n + self.m + 1
        self.settings = settings if settings is not None else default_settings(**kw)
        self._warm = None
        h = C.c_void_p()
        st = C.c_void_p(stream) if isinstance(stream, int) else (C.c_void_p(stream.cuda_stream) if stream is not None else None)
        _check(L.scs_setup(C.byref(self._keep.data), C.byref(self._keep.cone), C.byref(self.settings), st,
                           C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().scs_finish(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_warm(self, u):
        """Warm start from an HSDE iterate u (N values, numpy or CUDA); None for a cold start."""
        if u is None:
            _check(lib().scs_set_warm(self.h, None), self.h)
            return
        u = u if hasattr(u, "data_ptr") else np.ascontiguousarray(u, dtype=np.float64)
        _check(lib().scs_set_warm(self.h, _ptr(u)), self.h)

    def solve(self, x=None, y=None, s=None):
        """Returns (x, y, s, info dict); outputs may be preallocated host or device buffers."""
        x = np.empty(self.n) if x is None else x
        y = np.empty(self.m) if y is None else y
        s = np.empty(self.m) if s is None else s
        info = Info()
        _check(lib().scs_solve(self.h, _ptr(x), _ptr(y), _ptr(s), C.byref(info)), self.h)
        return x, y, s, info.as_dict()

    def update_bc(self, b=None, c=None):
        bb = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
        cc = None if c is None else np.ascontiguousarray(c, dtype=np.float64)
        _check(lib().scs_update_bc(self.h, _ptr(bb), _ptr(cc)), self.h)

    def get_u(self):
        u = np.empty(self.N)
        _check(lib().scs_get_u(self.h, _ptr(u)), self.h)
        return u

    def linsys(self, r, slot=0):
        r = np.ascontiguousarray(r, dtype=np.float64)
        out = np.empty(self.N)
        _check(lib().scs_linsys(self.h, _ptr(r), _ptr(out), slot), self.h)
        return out

    def project_cone(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.empty(self.N)
        _check(lib().scs_project_cone(self.h, _ptr(v), _ptr(out)), self.h)
        return out

    def project_cone_prec(self, v, precision):
        """Pi_C(v) as the given precision's phase computes it; returns (out, [max eigen-residual, blocks redone])."""
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.empty(self.N)
        stats = np.zeros(2)
        _check(lib().scs_project_cone_prec(self.h, precision, _ptr(v), _ptr(out), _ptr(stats)), self.h)
        return out, stats

    def residuals(self, x, y, s, out=None):
        """(pr, dr, gap) of Sec. 4.3 for a candidate; arrays host or CUDA."""
        conv = lambda a: a if hasattr(a, "data_ptr") else np.ascontiguousarray(a, dtype=np.float64)
        x, y, s = conv(x), conv(y), conv(s)
        o = np.empty(3) if out is None else out
        _check(lib().scs_residuals(self.h, _ptr(x), _ptr(y), _ptr(s), _ptr(o)), self.h)
        return o

    def profile(self, precision=FP64, reps=20):
        """ns per A pass, A^T pass, barrier, reduction, CG iteration (device timer)."""
        ns = np.zeros(5)
        _check(lib().scs_profile(self.h, precision, reps, _ptr(ns)), self.h)
        return dict(zip(("A", "AT", "barrier", "reduce", "cg_iter"), ns.tolist()))

    def spmv(self, v, op=0, precision=FP64, v2=None):
        """op 0: A v; op 1: A^T v; op 2: (A^T v, A^T v2) in one fused pass --
        the work's own matrix copy in the given bulk precision, widened to FP64."""
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.empty(self.m if op == 0 else self.n)
        if op == 2:
            v2 = np.ascontiguousarray(v2, dtype=np.float64)
            out2 = np.empty(self.n)
            _check(lib().scs_spmv(self.h, precision, op, _ptr(v), _ptr(v2), _ptr(out), _ptr(out2)), self.h)
            return out, out2
        _check(lib().scs_spmv(self.h, precision, op, _ptr(v), None, _ptr(out), None), self.h)
        return out

    def apply_T(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        Tu, Ru = np.empty(self.N), np.empty(self.N)
        _check(lib().scs_apply_T(self.h, _ptr(u), _ptr(Tu), _ptr(Ru)), self.h)
        return Tu, Ru


def cb_layout_check(A, x, ctas=152, compute_warps=15, elem_bytes=4, vectors=1, smem_bytes=209536):
    """Host-only check of the column-blocked layout of the CSR matrix A (see
    scs_cb_layout_check): returns (y = A x replayed through the layout,
    stats dict)."""
    A = A.tocsr()
    Ap = np.ascontiguousarray(A.indptr, dtype=np.int64)
    Ai = np.ascontiguousarray(A.indices, dtype=np.int32)
    Ax = np.ascontiguousarray(A.data, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.shape[0])
    st = np.zeros(8, dtype=np.int64)
    _check(lib().scs_cb_layout_check(A.shape[0], A.shape[1], _ptr(Ap), _ptr(Ai), _ptr(Ax), ctas, compute_warps,
                                     elem_bytes, vectors, smem_bytes, _ptr(x), _ptr(y), _ptr(st)))
    keys = ("violations", "column_blocks", "block_width", "lanes", "entries", "smem_bytes", "stages", "meta_words")
    return y, dict(zip(keys, st.tolist()))


def tile_layout_check(A, x, ctas=152, compute_warps=15, elem_bytes=4, vectors=1, smem_bytes=209536):
    """Host-only check of the two-dimensional tiled layout of the CSR matrix A
    (see scs_tile_layout_check): returns (y = A x replayed through the tiles
    and the partial-sum pass, stats dict)."""
    A = A.tocsr()
    Ap = np.ascontiguousarray(A.indptr, dtype=np.int64)
    Ai = np.ascontiguousarray(A.indices, dtype=np.int32)
    Ax = np.ascontiguousarray(A.data, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.shape[0])
    st = np.zeros(8, dtype=np.int64)
    _check(lib().scs_tile_layout_check(A.shape[0], A.shape[1], _ptr(Ap), _ptr(Ai), _ptr(Ax), ctas, compute_warps,
                                       elem_bytes, vectors, smem_bytes, _ptr(x), _ptr(y), _ptr(st)))
    keys = ("violations", "column_blocks", "row_blocks", "lanes", "entries", "smem_bytes", "chunks", "meta_words")
    return y, dict(zip(keys, st.tolist()))


class Batch:
    """B independent problems solved by one persistent launch.  With
    ``shared=(prob0, bs, cs)`` the instances share prob0's A and cones and
    differ in b = bs[i], c = cs[i] (scs_batch_setup_shared)."""

    def __init__(self, probs=None, settings: Settings | None = None, stream=None, shared=None, **kw):
        L = lib()
        self.settings = settings if settings is not None else default_settings(**kw)
        h = C.c_void_p()
        st = C.c_void_p(stream) if isinstance(stream, int) else (C.c_void_p(stream.cuda_stream) if stream is not None else None)
        if shared is not None:
            prob0, bs, cs = shared
            k0 = _Keep(prob0)
            self.B = len(bs)
            self._bs = [np.ascontiguousarray(b, dtype=np.float64) for b in bs]
            self._cs = [np.ascontiguousarray(c, dtype=np.float64) for c in cs]
            self.keeps = [k0] * self.B
            bp = (C.c_void_p * self.B)(*[b.ctypes.data for b in self._bs])
            cp = (C.c_void_p * self.B)(*[c.ctypes.data for c in self._cs])
            _check(L.scs_batch_setup_shared(self.B, C.byref(k0.data), C.byref(k0.cone), bp, cp,
                                            C.byref(self.settings), st, C.byref(h)))
        else:
            self.keeps = [_Keep(p) for p in probs]
            self.B = len(probs)
            self._dp = (C.POINTER(Data) * self.B)(*[C.pointer(k.data) for k in self.keeps])
            self._cp = (C.POINTER(Cone) * self.B)(*[C.pointer(k.cone) for k in self.keeps])
            _check(L.scs_batch_setup(self.B, self._dp, self._cp, C.byref(self.settings), st, C.byref(h)))
        self.h = h

    def set_warm(self, us):
        """us: list of N-vectors (numpy or CUDA tensors) or None for cold starts."""
        if us is None:
            _check(lib().scs_batch_set_warm(self.h, None))
            return
        self._warm = [u if hasattr(u, "data_ptr") else np.ascontiguousarray(u, dtype=np.float64) for u in us]
        arr = (C.c_void_p * self.B)(*[_ptr(u).value for u in self._warm])
        _check(lib().scs_batch_set_warm(self.h, arr))

    def solve(self):
        xs = [np.empty(k.n) for k in self.keeps]
        ys = [np.empty(k.m) for k in self.keeps]
        ss = [np.empty(k.m) for k in self.keeps]
        arr = lambda lst: (C.c_void_p * self.B)(*[a.ctypes.data for a in lst])
        infos = (Info * self.B)()
        _check(lib().scs_batch_solve(self.h, arr(xs), arr(ys), arr(ss), infos))
        return xs, ys, ss, [infos[i].as_dict() for i in range(self.B)]

    def close(self):
        if getattr(self, "h", None):
            lib().scs_batch_finish(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


GEMM_MMA, GEMM_TCGEN05 = 0, 1
# buffers of scs_mlp_read (include/superscs_mlp.h)
MLP_BUFFERS = ("params", "grad", "adam_m", "adam_v", "in_mean", "in_std", "out_mean", "out_std", "xn", "h1", "h2",
               "y", "dy", "dy16", "dh2", "dh2_16", "dh1", "dh1_16", "w1", "w2", "w3", "w2t", "w3t")


def gemm_nt(A, B, impl=GEMM_MMA, stream=None):
    """C = A @ B.T (FP32) from CUDA bf16 tensors A (M x K) and B (N x K) whose
    row strides are multiples of 8 (scs_mlp_gemm_nt); returns a new CUDA
    float32 tensor."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    out = torch.empty(M, N, dtype=torch.float32, device=A.device)
    st = None if stream is None else C.c_void_p(stream.cuda_stream)
    _check(lib().scs_mlp_gemm_nt(impl, M, N, K, C.c_void_p(A.data_ptr()), A.stride(0), C.c_void_p(B.data_ptr()),
                                 B.stride(0), C.c_void_p(out.data_ptr()), N, st))
    return out


class MLP:
    """The learned warm-start network (include/superscs_mlp.h).  Batches are
    CUDA torch tensors (float32, row-major)."""

    def __init__(self, d_in, d_hidden, d_out, max_batch, seed=0, stream=None, gemm=None):
        h = C.c_void_p()
        st = None if stream is None else C.c_void_p(stream.cuda_stream)
        _check(lib().scs_mlp_create(d_in, d_hidden, d_out, max_batch, seed, st, C.byref(h)))
        self.h = h
        self.dims = (d_in, d_hidden, d_out)
        if gemm is not None:
            _check(lib().scs_mlp_set_gemm(self.h, gemm))

    @property
    def num_params(self):
        return lib().scs_mlp_num_params(self.h)

    def fit_normalization(self, X, Y):
        _check(lib().scs_mlp_fit_normalization(self.h, _ptr(X), _ptr(Y), X.shape[0]))

    def train_step(self, X, Y, lr):
        loss = C.c_float()
        _check(lib().scs_mlp_train_step(self.h, _ptr(X), _ptr(Y), X.shape[0], lr, C.byref(loss)))
        return loss.value

    def forward(self, X, out):
        _check(lib().scs_mlp_forward(self.h, _ptr(X), X.shape[0], _ptr(out)))
        return out

    def gradients(self, X, Y, grad_out=None):
        loss = C.c_float()
        _check(lib().scs_mlp_gradients(self.h, _ptr(X), _ptr(Y), X.shape[0], _ptr(grad_out), C.byref(loss)))
        return loss.value

    def get_params(self):
        p = np.empty(self.num_params, dtype=np.float32)
        _check(lib().scs_mlp_get_params(self.h, _ptr(p)))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().scs_mlp_set_params(self.h, _ptr(p)))

    def read(self, name):
        """An internal buffer (scs_mlp_read) as a host float32 array of its
        shape; BF16 buffers are widened exactly (their bits shifted into the
        high half of an FP32 word)."""
        what = MLP_BUFFERS.index(name)
        r, c, eb = C.c_int64(), C.c_int64(), C.c_int32()
        _check(lib().scs_mlp_read(self.h, what, None, C.byref(r), C.byref(c), C.byref(eb)))
        if eb.value == 4:
            out = np.empty((r.value, c.value), dtype=np.float32)
            _check(lib().scs_mlp_read(self.h, what, _ptr(out), None, None, None))
            return out
        raw = np.empty((r.value, c.value), dtype=np.uint16)
        _check(lib().scs_mlp_read(self.h, what, _ptr(raw), None, None, None))
        return (raw.astype(np.uint32) << 16).view(np.float32)

    def close(self):
        if getattr(self, "h", None):
            lib().scs_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
