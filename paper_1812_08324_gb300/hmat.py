"""Thin ctypes binding of the C ABI in ``include/levy_hmat.h``.

Argument marshalling only: problem/option dictionaries become the C structs,
torch CUDA tensors become device pointers, the current torch stream becomes
the cudaStream_t.  Every numerical step runs in the CUDA library; if the
library is missing this module raises instead of computing anything on the CPU.
"""
from __future__ import annotations

import ctypes as C
import math
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "liblevyhm.so")

HM_OK = 0
HM_ERR_NOT_CONVERGED = -5
HM_NU_GAUSS, HM_NU_STABLE = 0, 1
HM_FP64, HM_MIXED_FP32, HM_MIXED_BF16 = 0, 1, 2
HM_SOLVE_AUTO, HM_SOLVE_SUBST, HM_SOLVE_HINV = 0, 1, 2
PRECISIONS = {"fp64": HM_FP64, "fp32": HM_MIXED_FP32, "mixed_fp32": HM_MIXED_FP32, "bf16": HM_MIXED_BF16,
              "mixed_bf16": HM_MIXED_BF16}
SOLVES = {"auto": HM_SOLVE_AUTO, "subst": HM_SOLVE_SUBST, "hinv": HM_SOLVE_HINV}
HM_CN_IDENTITY, HM_CN_LITERAL = 0, 1
CN_FORMS = {"identity": HM_CN_IDENTITY, "literal": HM_CN_LITERAL}
HM_DOMAIN_BOX, HM_DOMAIN_L = 0, 1

EXPORTED = [
    "hm_error_string", "hm_last_error", "hm_plan_info", "hm_plan_blocks", "hm_build",
    "hm_matvec", "hm_to_dense", "hm_entries", "hm_factor", "hm_solve", "cn_step", "cn_solve",
    "hm_sync", "hm_stats", "hm_free", "hm_factors_free", "hm_plan_factor", "hm_launch_count",
    "hm_matvec_noalloc", "hm_factor_batch", "cn_solve_batch", "hm_batch_graphed",
    "hm_batch_create", "hm_batch_step", "hm_batch_free", "hm_factor_shifted", "hm_shifted_solve",
]


class Problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 2), ("lo", C.c_double * 2), ("hi", C.c_double * 2),
                ("a", C.c_double), ("b", C.c_double * 2), ("c", C.c_double), ("kernel", C.c_int),
                ("s", C.c_double), ("eps", C.c_double), ("lam", C.c_double), ("trunc", C.c_double),
                ("LW", C.c_double), ("r", C.c_double), ("domain", C.c_int), ("s_slope", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("leaf", C.c_int), ("eta", C.c_double), ("aca_tol", C.c_double),
                ("max_rank", C.c_int), ("lu_tol", C.c_double), ("lu_max_rank", C.c_int),
                ("precision", C.c_int), ("refine_tol", C.c_double), ("refine_max", C.c_int),
                ("solve", C.c_int), ("solve_block", C.c_int), ("hinv_tol", C.c_double),
                ("cn_form", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("clusters", C.c_int), ("leaves", C.c_int), ("depth", C.c_int),
                ("dense_blocks", C.c_int), ("lowrank_blocks", C.c_int),
                ("dense_entries", C.c_int64), ("lowrank_entries", C.c_int64),
                ("h_bytes", C.c_int64), ("lu_bytes", C.c_int64), ("max_rank_seen", C.c_int),
                ("rank_capped_blocks", C.c_int), ("lu_max_rank_seen", C.c_int),
                ("lu_rank_capped", C.c_int), ("last_refine_iters", C.c_int),
                ("last_refine_resid", C.c_double), ("device_bytes", C.c_int64),
                ("factor_fma", C.c_double), ("factor_ms", C.c_double), ("solve_mode", C.c_int),
                ("hinv_max_rank", C.c_int), ("hinv_capped", C.c_int), ("hinv_ms", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class FactorPlan(C.Structure):
    _fields_ = [("fact_ops", C.c_int64), ("fact_waves", C.c_int), ("solve_ops", C.c_int64),
                ("solve_waves", C.c_int), ("bad_spans", C.c_int64), ("arena_bytes", C.c_int64),
                ("kf", C.c_int), ("gemm_fma", C.c_double * 3)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["gemm_fma"] = list(self.gemm_fma)
        return d


class HMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None


def load() -> C.CDLL:
    """Load the CUDA library (build it first with ``paper_1812_08324_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run paper_1812_08324_gb300.build)")
    lib = C.CDLL(LIB_PATH)
    vp, d, i, i64 = C.c_void_p, C.c_double, C.c_int, C.c_int64
    P, O, S = C.POINTER(Problem), C.POINTER(Opts), C.POINTER(Stats)
    sig = {
        "hm_error_string": (C.c_char_p, [i]),
        "hm_last_error": (C.c_char_p, []),
        "hm_plan_info": (i, [P, O, S]),
        "hm_plan_blocks": (i, [P, O, C.POINTER(i), vp, vp, vp, vp, vp, vp]),
        "hm_build": (i, [P, O, vp, C.POINTER(vp)]),
        "hm_matvec": (i, [vp, d, d, vp, d, vp, vp, vp, vp]),
        "hm_to_dense": (i, [vp, vp, vp]),
        "hm_entries": (i, [vp, i64, vp, vp, vp, vp]),
        "hm_factor": (i, [vp, d, vp, C.POINTER(vp)]),
        "hm_solve": (i, [vp, vp, vp, vp]),
        "cn_step": (i, [vp, vp, d, vp, vp, vp, vp, vp]),
        "cn_solve": (i, [vp, vp, d, i, i, vp, vp, vp]),
        "hm_sync": (i, [vp, vp]),
        "hm_stats": (i, [vp, vp, S]),
        "hm_free": (None, [vp]),
        "hm_factors_free": (None, [vp]),
        "hm_plan_factor": (i, [P, O, d, C.POINTER(FactorPlan)]),
        "hm_launch_count": (i64, []),
        "hm_matvec_noalloc": (i, [vp, d, d, vp, d, vp, vp, vp, vp]),
        "hm_factor_batch": (i, [C.POINTER(vp), C.POINTER(d), i, vp, C.POINTER(vp)]),
        "cn_solve_batch": (i, [C.POINTER(vp), C.POINTER(vp), i, d, i, C.POINTER(vp), vp]),
        "hm_batch_graphed": (i, []),
        "hm_batch_create": (i, [C.POINTER(vp), C.POINTER(vp), C.POINTER(d), i, C.POINTER(vp)]),
        "hm_batch_step": (i, [vp, C.POINTER(vp), i, vp]),
        "hm_batch_free": (None, [vp]),
        "hm_factor_shifted": (i, [vp, d, d, vp, C.POINTER(vp)]),
        "hm_shifted_solve": (i, [vp, vp, vp, vp, d, i, vp, C.POINTER(i), C.POINTER(d)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != HM_OK:
        lib = load()
        raise HMError(status, f"{lib.hm_error_string(status).decode()}: {lib.hm_last_error().decode()}")


def make_problem(p: dict) -> Problem:
    s = Problem()
    s.dim = int(p["dim"])
    n = list(p["n"]) + [1]
    s.n[0], s.n[1] = int(n[0]), int(n[1])
    lo = list(p["lo"]) + [0.0]
    hi = list(p["hi"]) + [0.0]
    s.lo[0], s.lo[1] = float(lo[0]), float(lo[1])
    s.hi[0], s.hi[1] = float(hi[0]), float(hi[1])
    s.a = float(p.get("a", 0.0))
    b = list(p.get("b", [0.0, 0.0])) + [0.0]
    s.b[0], s.b[1] = float(b[0]), float(b[1])
    s.c = float(p.get("c", 0.0))
    s.kernel = HM_NU_GAUSS if p["kernel"] == "gauss" else HM_NU_STABLE
    s.s = float(p.get("s", 0.0))
    s.eps = float(p.get("eps", 0.0))
    s.lam = float(p.get("lam", 0.0))
    s.trunc = float(p.get("trunc", math.inf))
    s.LW = float(p["LW"])
    s.r = float(p.get("r", 0.2))
    domain = p.get("domain", "box")
    s.domain = domain if isinstance(domain, int) else {"box": HM_DOMAIN_BOX, "L": HM_DOMAIN_L}[domain]
    s.s_slope = float(p.get("s_slope", 0.0))
    return s


def make_opts(o: dict) -> Opts:
    s = Opts()
    s.leaf = int(o.get("leaf", 64))
    s.eta = float(o.get("eta", 1.0))
    s.aca_tol = float(o.get("aca_tol", 1e-10))
    s.max_rank = int(o.get("max_rank", 64))
    s.lu_tol = float(o.get("lu_tol", 1e-10))
    s.lu_max_rank = int(o.get("lu_max_rank", 64))
    prec = o.get("precision", "fp64")
    s.precision = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    s.refine_tol = float(o.get("refine_tol", 1e-13))
    s.refine_max = int(o.get("refine_max", 4))
    solve = o.get("solve", "auto")
    s.solve = SOLVES[solve] if isinstance(solve, str) else int(solve)
    s.solve_block = int(o.get("solve_block", 0))
    s.hinv_tol = float(o.get("hinv_tol", 0.0))
    form = o.get("cn_form", "identity")
    s.cn_form = CN_FORMS[form] if isinstance(form, str) else int(form)
    return s


def plan_info(problem: dict, opts: dict) -> dict:
    """Cluster/block-tree statistics from the host planner (no GPU needed)."""
    lib = load()
    st = Stats()
    _check(lib.hm_plan_info(C.byref(make_problem(problem)), C.byref(make_opts(opts)), C.byref(st)))
    return st.as_dict()


def plan_factor(problem: dict, opts: dict, theta: float = -5e-4) -> dict:
    """Dry-run H-LU / solve schedules on the host (fake addresses): op and wave
    counts, memory, and the operand-span check."""
    lib = load()
    fp = FactorPlan()
    _check(lib.hm_plan_factor(C.byref(make_problem(problem)), C.byref(make_opts(opts)), theta,
                              C.byref(fp)))
    return fp.as_dict()


def plan_blocks(problem: dict, opts: dict):
    """Leaf blocks of the block tree: (row0, m, col0, ncols, type, perm) numpy arrays."""
    import numpy as np
    lib = load()
    info = plan_info(problem, opts)
    cnt = info["dense_blocks"] + info["lowrank_blocks"]
    arrs = [np.zeros(cnt, dtype=np.int32) for _ in range(5)]
    perm = np.zeros(info["n"], dtype=np.int32)
    c = C.c_int(cnt)
    _check(lib.hm_plan_blocks(C.byref(make_problem(problem)), C.byref(make_opts(opts)), C.byref(c),
                              *[a.ctypes.data for a in arrs], perm.ctypes.data))
    return (*arrs, perm)


def launch_count() -> int:
    """Kernel launches issued by the library in this process."""
    return int(load().hm_launch_count())


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int | None:
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return int(t.data_ptr())


class HMatrix:
    """Device-resident H-matrix of the discrete generator G (owned by the library)."""

    def __init__(self, problem: dict, opts: dict, stream=None):
        lib = load()
        self.problem = dict(problem)
        self.opts = dict(opts)
        self._h = C.c_void_p()
        self._p = make_problem(problem)
        self._o = make_opts(opts)
        _check(lib.hm_build(C.byref(self._p), C.byref(self._o), _stream(stream), C.byref(self._h)))
        self.n = int(self.stats()["n"])

    @property
    def handle(self):
        return self._h

    def matvec(self, x, alpha=0.0, beta=1.0, gamma=0.0, w1=None, w2=None, out=None, stream=None):
        """out = alpha x + beta G x + gamma (w1 + w2)."""
        import torch
        if out is None:
            out = torch.empty_like(x)
        _check(load().hm_matvec(self._h, alpha, beta, _ptr(x), gamma, _ptr(w1), _ptr(w2), _ptr(out),
                                _stream(stream)))
        return out

    def to_dense(self, stream=None):
        import torch
        out = torch.zeros(self.n, self.n, dtype=torch.float64, device="cuda")
        _check(load().hm_to_dense(self._h, _ptr(out), _stream(stream)))
        return out

    def entries(self, rows, cols, stream=None):
        import torch
        rows = rows.to(device="cuda", dtype=torch.int32).contiguous()
        cols = cols.to(device="cuda", dtype=torch.int32).contiguous()
        out = torch.empty(rows.numel(), dtype=torch.float64, device="cuda")
        _check(load().hm_entries(self._h, rows.numel(), rows.data_ptr(), cols.data_ptr(), _ptr(out),
                                 _stream(stream)))
        return out

    def sync(self, stream=None):
        _check(load().hm_sync(self._h, _stream(stream)))

    def stats(self, factors=None) -> dict:
        st = Stats()
        _check(load().hm_stats(self._h, factors._f if factors is not None else None, C.byref(st)))
        return st.as_dict()

    def factor(self, theta: float, stream=None) -> "Factors":
        return Factors(self, theta, stream)

    def factor_shifted(self, alpha: float, theta: float, stream=None) -> "Factors":
        """H-LU factors of alpha I + theta G (alpha = 0, theta = 1: G itself)."""
        f = C.c_void_p()
        _check(load().hm_factor_shifted(self._h, float(alpha), float(theta), _stream(stream), C.byref(f)))
        F = Factors(self, theta, _handle=f.value)
        F.alpha = float(alpha)
        return F

    def free(self):
        if self._h:
            load().hm_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Factors:
    """H-LU factors of alpha I + theta G (owned by the library); alpha = 1
    unless made by HMatrix.factor_shifted."""

    def __init__(self, H: HMatrix, theta: float, stream=None, _handle=None):
        self.H = H
        self.theta = theta
        self.alpha = 1.0
        self._f = C.c_void_p()
        if _handle is not None:
            self._f = C.c_void_p(_handle)
            return
        _check(load().hm_factor(H.handle, theta, _stream(stream), C.byref(self._f)))

    def solve(self, b, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(b)
        _check(load().hm_solve(self._f, _ptr(b), _ptr(out), _stream(stream)))
        return out

    def free(self):
        if self._f:
            load().hm_factors_free(self._f)
            self._f = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def cn_step(H: HMatrix, F: Factors, dt: float, u, f_n=None, f_np1=None, out=None, stream=None):
    """One Crank-Nicolson step; returns u^{n+1}."""
    import torch
    if out is None:
        out = torch.empty_like(u)
    _check(load().cn_step(H.handle, F._f, dt, _ptr(u), _ptr(f_n), _ptr(f_np1), _ptr(out),
                          _stream(stream)))
    return out


def cn_solve(H: HMatrix, F: Factors, dt: float, steps: int, u, f=None, step0: int = 0, stream=None):
    """Advance u in place by `steps` CN steps; f is (steps+1) x N forcing or None."""
    _check(load().cn_solve(H.handle, F._f, dt, int(steps), int(step0), _ptr(u), _ptr(f),
                           _stream(stream)))
    return u


def shifted_solve(H: HMatrix, F: Factors, b, tol: float = 1e-12, maxit: int = 50, out=None, stream=None,
                  check: bool = True):
    """x with (alpha I + theta G) x = b by H-LU-preconditioned Richardson
    iteration; returns (x, iterations, relative residual).  With check=False a
    missed tolerance is reported only through the residual."""
    import torch
    if out is None:
        out = torch.empty_like(b)
    it = C.c_int(0)
    res = C.c_double(0.0)
    st = load().hm_shifted_solve(H.handle, F._f, _ptr(b), _ptr(out), float(tol), int(maxit), _stream(stream),
                                 C.byref(it), C.byref(res))
    if check or st != HM_ERR_NOT_CONVERGED:
        _check(st)
    return out, it.value, res.value


def factor_batch(Hs, thetas, stream=None):
    """H-LU factors of I + theta_i G_i for many matrices in one persistent launch;
    returns one Factors per matrix (each equal to H.factor(theta) bit for bit)."""
    n = len(Hs)
    hs = (C.c_void_p * n)(*[H.handle.value for H in Hs])
    th = (C.c_double * n)(*[float(t) for t in thetas])
    out = (C.c_void_p * n)()
    _check(load().hm_factor_batch(hs, th, n, _stream(stream), out))
    return [Factors(H, t, _handle=out[i]) for i, (H, t) in enumerate(zip(Hs, thetas))]


def cn_solve_batch(Hs, Fs, dt: float, steps: int, us, stream=None):
    """Advance every us[i] in place by `steps` CN steps (no forcing), all
    problems per step in one batched H-matvec and one merged solve launch."""
    n = len(Hs)
    hs = (C.c_void_p * n)(*[H.handle.value for H in Hs])
    fs = (C.c_void_p * n)(*[F._f.value for F in Fs])
    ps = (C.c_void_p * n)(*[_ptr(u) for u in us])
    _check(load().cn_solve_batch(hs, fs, n, float(dt), int(steps), ps, _stream(stream)))
    return us


def batch_graphed() -> bool:
    return bool(load().hm_batch_graphed())


class Batch:
    """Problems stepped together: merged solve schedule and batched H-matvec,
    one CUDA graph per step (hm_batch_create).  Keeps references to its
    matrices and factors; free() before freeing them."""

    def __init__(self, Hs, Fs, dts):
        n = len(Hs)
        self.Hs, self.Fs = list(Hs), list(Fs)
        hs = (C.c_void_p * n)(*[H.handle.value for H in Hs])
        fs = (C.c_void_p * n)(*[F._f.value for F in Fs])
        ds = (C.c_double * n)(*[float(x) for x in dts])
        self._b = C.c_void_p()
        _check(load().hm_batch_create(hs, fs, ds, n, C.byref(self._b)))

    def step(self, us, steps: int, stream=None):
        n = len(self.Hs)
        ps = (C.c_void_p * n)(*[_ptr(u) for u in us])
        _check(load().hm_batch_step(self._b, ps, int(steps), _stream(stream)))
        return us

    def free(self):
        if self._b:
            load().hm_batch_free(self._b)
            self._b = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
