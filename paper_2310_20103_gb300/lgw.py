"""ctypes binding of the lgw C ABI (include/lgw.h).

Argument marshalling only: every function below forwards pointers and sizes
to the entry point of the same name in ``liblgw.so``; all arithmetic of the
hot path runs in the library's CUDA kernels.  Arrays may be torch tensors
(CUDA or CPU) or numpy arrays; they must be C-contiguous with the dtype the
C ABI expects (float64 or int32).  Importing this module fails loudly when
the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblgw.so")

LGW_OK = 0
STATUS_NAMES = {0: "LGW_OK", 1: "LGW_ERR_ARG", 2: "LGW_ERR_SHAPE", 3: "LGW_ERR_CUDA",
                4: "LGW_ERR_OOM", 5: "LGW_ERR_NOT_SPD", 6: "LGW_ERR_NO_CONVERGENCE",
                7: "LGW_ERR_TIMEOUT", 8: "LGW_ERR_UNSUPPORTED"}
PRECISION = {"fp64": 0, "bf16": 1, "fp8": 3, "fp8_deq": 4}
REORTH = {"none": 0, "cgs2": 1, "cgs1k": 2, "dcgs": 3}
REORTH_ARITH = {"auto": 0, "fp64": 1, "split": 2, "split32": 3}
QP_MODE = {"graphical": 0, "linearised": 1}


class LgwError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class lgw_system_desc(ctypes.Structure):
    _fields_ = [("n_v", ctypes.c_int32), ("n_c", ctypes.c_int32), ("n_aux", ctypes.c_int32),
                ("eps", ctypes.c_void_p), ("L", ctypes.c_void_p),
                ("kernel_factor", ctypes.c_double), ("flags", ctypes.c_int32)]


SYS_NO_FP64, SYS_NO_BF16, SYS_FP8 = 1, 2, 4


class lgw_poly(ctypes.Structure):
    _fields_ = [("g", ctypes.c_int32), ("x_lo", ctypes.c_double), ("x_hi", ctypes.c_double)]


class lgw_problem(ctypes.Structure):
    _fields_ = [("n_t", ctypes.c_int32), ("targets", ctypes.c_void_p),
                ("n_m", ctypes.c_int32), ("m_idx", ctypes.c_void_p),
                ("M", ctypes.c_void_p), ("V", ctypes.c_void_p),
                ("n_freq", ctypes.c_int32), ("omega", ctypes.c_void_p),
                ("delta", ctypes.c_double), ("static_shift", ctypes.c_void_p)]


class lgw_options(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("reorth", ctypes.c_int32), ("b_sub", ctypes.c_int32),
                ("breakdown_tol", ctypes.c_double), ("qp_max_iter", ctypes.c_int32),
                ("qp_tol", ctypes.c_double), ("use_graph", ctypes.c_int32),
                ("reorth_arith", ctypes.c_int32), ("qp_mode", ctypes.c_int32),
                ("ckpt_every", ctypes.c_int32)]


class lgw_report(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "ms_total", "ms_start", "ms_gemm1", "ms_gemm2", "ms_dots", "ms_update", "ms_pass2",
        "ms_normalize", "ms_spectral", "ms_cf", "ms_qp", "gemm_flops", "reorth_elems")] + \
        [(n, ctypes.c_int32) for n in (
            "n_vectors", "n_sub_batches", "b_sub", "k_min", "k_max", "n_second_pass",
            "gpu_launches", "gemm1_splits")] + [("min_theta", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblgw.so once; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int32
    sig = {
        "lgw_status_string": ([I], ctypes.c_char_p),
        "lgw_create": ([ctypes.POINTER(P), ctypes.c_int, P], I),
        "lgw_destroy": ([P], I),
        "lgw_last_error": ([P, ctypes.c_char_p, ctypes.c_size_t], I),
        "lgw_prepare_system": ([P, ctypes.POINTER(lgw_system_desc), ctypes.POINTER(P)], I),
        "lgw_release_system": ([P], I),
        "lgw_apply_casida": ([P, P, I, P, P, I], I),
        "lgw_lanczos_coeffs": ([P, P, ctypes.POINTER(lgw_problem), ctypes.POINTER(lgw_options),
                                P, P, P, P], I),
        "lgw_sigma_from_coeffs": ([P, P, ctypes.POINTER(lgw_problem),
                                   ctypes.POINTER(lgw_options), P, P, P, P, P, P, P], I),
        "lgw_sigma_c": ([P, P, ctypes.POINTER(lgw_problem), ctypes.POINTER(lgw_options),
                         P, P, P, ctypes.POINTER(lgw_report)], I),
        "lgw_sigma_c_batched": ([P, I, P, ctypes.POINTER(lgw_problem),
                                 ctypes.POINTER(lgw_options), P, P, P,
                                 ctypes.POINTER(lgw_report)], I),
        "lgw_sigma_c_backward": ([P, P, ctypes.POINTER(lgw_problem),
                                  ctypes.POINTER(lgw_options), P, P, P], I),
        "lgw_sigma_c_tda_backward": ([P, P, ctypes.POINTER(lgw_problem),
                                      ctypes.POINTER(lgw_options), P, P, P], I),
        "lgw_sigma_c_poly_backward": ([P, P, ctypes.POINTER(lgw_problem),
                                       ctypes.POINTER(lgw_options), ctypes.POINTER(lgw_poly),
                                       P, P, P], I),
        "lgw_sigma_x": ([P, P, ctypes.POINTER(lgw_problem), P], I),
        "lgw_sigma_c_tda": ([P, P, ctypes.POINTER(lgw_problem), ctypes.POINTER(lgw_options),
                             P, P, P, ctypes.POINTER(lgw_report)], I),
        "lgw_sigma_offdiag": ([P, P, ctypes.POINTER(lgw_problem), ctypes.POINTER(lgw_options),
                               I, P, P], I),
        "lgw_fit_factors": ([P, I, I, P, P, P], I),
        "lgw_sigma_c_poly": ([P, P, ctypes.POINTER(lgw_problem), ctypes.POINTER(lgw_options),
                              ctypes.POINTER(lgw_poly), P, P, P, ctypes.POINTER(lgw_report)], I),
        "lgw_lanczos_coeffs_poly": ([P, P, ctypes.POINTER(lgw_problem),
                                     ctypes.POINTER(lgw_options), ctypes.POINTER(lgw_poly),
                                     P, P, P, P], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _ptr(x, dtype: str):
    """Raw address of a contiguous array of the given dtype ('f64' or 'i32')."""
    if x is None:
        return None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            want = torch.float64 if dtype == "f64" else torch.int32
            if x.dtype != want or not x.is_contiguous():
                raise TypeError(f"tensor must be contiguous {want}, got {x.dtype}")
            return x.data_ptr()
    except ImportError:
        pass
    if isinstance(x, np.ndarray):
        want = np.float64 if dtype == "f64" else np.int32
        if x.dtype != want or not x.flags["C_CONTIGUOUS"]:
            raise TypeError(f"array must be C-contiguous {np.dtype(want)}, got {x.dtype}")
        return x.ctypes.data
    raise TypeError(f"unsupported array type {type(x)}")


def _numel(x):
    return int(np.prod(x.shape)) if x is not None else 0


def _check(h, st):
    if st != LGW_OK:
        msg = lgw_last_error(h) if h is not None else ""
        raise LgwError(st, msg or lgw_status_string(st))


class Handle:
    def __init__(self, ptr: int, keep=None):
        self.ptr = ctypes.c_void_p(ptr)
        self._keep = keep

    def __enter__(self):
        return self

    def __exit__(self, *a):
        lgw_destroy(self)


class System:
    def __init__(self, ptr, handle, n_v, n_c, n_aux, kernel_factor):
        self.ptr = ctypes.c_void_p(ptr)
        self.handle = handle
        self.n_v, self.n_c, self.n_aux = n_v, n_c, n_aux
        self.kernel_factor = kernel_factor

    @property
    def n_vc(self):
        return self.n_v * self.n_c


@dataclass
class Problem:
    targets: object          # [n_t] int32
    m_idx: object            # [n_m] int32
    omega: object            # [n_freq] float64
    delta: float
    M: object = None         # [n_t, n_m, n_aux] float64
    V: object = None         # [n_t, n_m, n_vc] float64
    static_shift: object = None

    def to_c(self) -> lgw_problem:
        p = lgw_problem()
        p.n_t = _numel(self.targets)
        p.targets = _ptr(self.targets, "i32")
        p.n_m = _numel(self.m_idx)
        p.m_idx = _ptr(self.m_idx, "i32")
        p.M = _ptr(self.M, "f64")
        p.V = _ptr(self.V, "f64")
        p.n_freq = _numel(self.omega)
        p.omega = _ptr(self.omega, "f64")
        p.delta = float(self.delta)
        p.static_shift = _ptr(self.static_shift, "f64")
        return p


@dataclass
class Options:
    k: int
    precision: str = "bf16"
    reorth: str = "cgs2"
    b_sub: int = 0
    breakdown_tol: float = 0.0
    qp_max_iter: int = 0
    qp_tol: float = 0.0
    use_graph: int = 0
    reorth_arith: str = "auto"
    qp_mode: str = "graphical"
    ckpt_every: int = 0

    def to_c(self) -> lgw_options:
        o = lgw_options()
        o.k = int(self.k)
        o.precision = PRECISION[self.precision]
        o.reorth = REORTH[self.reorth]
        o.b_sub = int(self.b_sub)
        o.breakdown_tol = float(self.breakdown_tol)
        o.qp_max_iter = int(self.qp_max_iter)
        o.qp_tol = float(self.qp_tol)
        o.use_graph = int(self.use_graph)
        o.reorth_arith = REORTH_ARITH[self.reorth_arith]
        o.qp_mode = QP_MODE[self.qp_mode]
        o.ckpt_every = int(self.ckpt_every)
        return o


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def lgw_status_string(st: int) -> str:
    return load_library().lgw_status_string(int(st)).decode()


def lgw_last_error(h: Handle) -> str:
    buf = ctypes.create_string_buffer(512)
    load_library().lgw_last_error(h.ptr, buf, 512)
    return buf.value.decode()


def lgw_create(device: int = 0, stream=None) -> Handle:
    """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None for
    torch's current stream on ``device``."""
    lib = load_library()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(device)
    raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    out = ctypes.c_void_p()
    st = lib.lgw_create(ctypes.byref(out), int(device), ctypes.c_void_p(raw))
    if st != LGW_OK:
        raise LgwError(st, "lgw_create failed")
    return Handle(out.value, keep=stream)


def lgw_destroy(h: Handle) -> None:
    if h.ptr:
        load_library().lgw_destroy(h.ptr)
        h.ptr = ctypes.c_void_p()


def lgw_set_workspace_limit(h: Handle, nbytes: int) -> None:
    lib = load_library()
    fn = lib.lgw_set_workspace_limit
    fn.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
    fn.restype = ctypes.c_int32
    _check(h, fn(h.ptr, int(nbytes)))


def lgw_workspace_bytes(h: Handle) -> int:
    lib = load_library()
    fn = lib.lgw_workspace_bytes
    fn.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]
    fn.restype = ctypes.c_int32
    n = ctypes.c_size_t(0)
    _check(h, fn(h.ptr, ctypes.byref(n)))
    return int(n.value)


def lgw_release_workspace(h: Handle) -> None:
    lib = load_library()
    fn = lib.lgw_release_workspace
    fn.argtypes = [ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    _check(h, fn(h.ptr))


def lgw_selftest_bounded_wait(h: Handle, arrive: bool, seconds: float) -> None:
    lib = load_library()
    fn = lib.lgw_selftest_bounded_wait
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double]
    fn.restype = ctypes.c_int32
    _check(h, fn(h.ptr, 1 if arrive else 0, float(seconds)))


def lgw_prepare_system(h: Handle, n_v: int, n_c: int, n_aux: int, eps, L,
                       kernel_factor: float = 4.0, flags: int = 0) -> System:
    d = lgw_system_desc(int(n_v), int(n_c), int(n_aux), _ptr(eps, "f64"), _ptr(L, "f64"),
                        float(kernel_factor), int(flags))
    out = ctypes.c_void_p()
    _check(h, load_library().lgw_prepare_system(h.ptr, ctypes.byref(d), ctypes.byref(out)))
    return System(out.value, h, n_v, n_c, n_aux, kernel_factor)


def lgw_release_system(s: System) -> None:
    if s.ptr:
        load_library().lgw_release_system(s.ptr)
        s.ptr = ctypes.c_void_p()


def lgw_apply_casida(h: Handle, s: System, X, Y, precision: str = "fp64") -> None:
    n_vec = X.shape[0] if X is not None else 0
    _check(h, load_library().lgw_apply_casida(h.ptr, s.ptr, int(n_vec), _ptr(X, "f64"),
                                              _ptr(Y, "f64"), PRECISION[precision]))


def lgw_lanczos_coeffs(h: Handle, s: System, problem: Problem, options: Options,
                       alpha, beta, beta0, k_eff) -> None:
    p, o = problem.to_c(), options.to_c()
    _check(h, load_library().lgw_lanczos_coeffs(
        h.ptr, s.ptr, ctypes.byref(p), ctypes.byref(o), _ptr(alpha, "f64"), _ptr(beta, "f64"),
        _ptr(beta0, "f64"), _ptr(k_eff, "i32")))


def lgw_sigma_from_coeffs(h: Handle, s: System, problem: Problem, options: Options,
                          alpha, beta, beta0, k_eff, sigma, e_qp, z_qp=None) -> None:
    p, o = problem.to_c(), options.to_c()
    _check(h, load_library().lgw_sigma_from_coeffs(
        h.ptr, s.ptr, ctypes.byref(p), ctypes.byref(o), _ptr(alpha, "f64"), _ptr(beta, "f64"),
        _ptr(beta0, "f64"), _ptr(k_eff, "i32"), _ptr(sigma, "f64"), _ptr(e_qp, "f64"),
        _ptr(z_qp, "f64")))


def lgw_sigma_c(h: Handle, s: System, problem: Problem, options: Options, sigma, e_qp,
                z_qp=None, report: bool = False) -> Optional[dict]:
    p, o = problem.to_c(), options.to_c()
    rep = lgw_report()
    _check(h, load_library().lgw_sigma_c(
        h.ptr, s.ptr, ctypes.byref(p), ctypes.byref(o), _ptr(sigma, "f64"), _ptr(e_qp, "f64"),
        _ptr(z_qp, "f64"), ctypes.byref(rep) if report else None))
    return rep.as_dict() if report else None


def lgw_sigma_c_tda(h: Handle, s: System, problem: Problem, options: Options, sigma, e_qp,
                    z_qp=None, report: bool = False) -> Optional[dict]:
    p, o = problem.to_c(), options.to_c()
    rep = lgw_report()
    _check(h, load_library().lgw_sigma_c_tda(
        h.ptr, s.ptr, ctypes.byref(p), ctypes.byref(o), _ptr(sigma, "f64"), _ptr(e_qp, "f64"),
        _ptr(z_qp, "f64"), ctypes.byref(rep) if report else None))
    return rep.as_dict() if report else None


def lgw_sigma_offdiag(h: Handle, s: System, problem: Problem, options: Options, pairs,
                      sigma_od) -> None:
    p, o = problem.to_c(), options.to_c()
    n = _numel(pairs) // 2
    _check(h, load_library().lgw_sigma_offdiag(h.ptr, s.ptr, ctypes.byref(p), ctypes.byref(o),
                                               int(n), _ptr(pairs, "i32"), _ptr(sigma_od, "f64")))


def lgw_sigma_x(h: Handle, s: System, problem: Problem, sigma_x) -> None:
    p = problem.to_c()
    _check(h, load_library().lgw_sigma_x(h.ptr, s.ptr, ctypes.byref(p), _ptr(sigma_x, "f64")))


def lgw_fit_factors(h: Handle, C, metric, B) -> None:
    n_pairs, n_aux = (C.shape[0], C.shape[1]) if C is not None else (0, metric.shape[0])
    _check(h, load_library().lgw_fit_factors(h.ptr, int(n_pairs), int(n_aux), _ptr(C, "f64"),
                                             _ptr(metric, "f64"), _ptr(B, "f64")))


def lgw_sigma_c_poly(h: Handle, s: System, problem: Problem, options: Options, g: int,
                     x_lo: float, x_hi: float, sigma, e_qp, z_qp=None,
                     report: bool = False) -> Optional[dict]:
    p, o = problem.to_c(), options.to_c()
    pl = lgw_poly(int(g), float(x_lo), float(x_hi))
    rep = lgw_report()
    _check(h, load_library().lgw_sigma_c_poly(
        h.ptr, s.ptr, ctypes.byref(p), ctypes.byref(o), ctypes.byref(pl), _ptr(sigma, "f64"),
        _ptr(e_qp, "f64"), _ptr(z_qp, "f64"), ctypes.byref(rep) if report else None))
    return rep.as_dict() if report else None


def lgw_sigma_band(h: Handle, s: System, problem: Problem, options: Options, sigma,
                   report: bool = False) -> Optional[dict]:
    """Sigma_tt'(omega) of the request's targets by band Lanczos:
    sigma [n_t][n_t][n_freq][2]."""
    lib = load_library()
    fn = lib.lgw_sigma_band
    if fn.argtypes is None:
        P = ctypes.c_void_p
        fn.argtypes = [P, P, ctypes.POINTER(lgw_problem), ctypes.POINTER(lgw_options), P,
                       ctypes.POINTER(lgw_report)]
        fn.restype = ctypes.c_int32
    p, o = problem.to_c(), options.to_c()
    rep = lgw_report()
    _check(h, fn(h.ptr, s.ptr, ctypes.byref(p), ctypes.byref(o), _ptr(sigma, "f64"),
                 ctypes.byref(rep) if report else None))
    return rep.as_dict() if report else None


def lgw_spectral_interval(h: Handle, s: System, k: int = 32):
    """(x_lo, x_hi) around the spectrum of C for the polynomial fit."""
    lib = load_library()
    fn = lib.lgw_spectral_interval
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    fn.restype = ctypes.c_int32
    lo, hi = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(h, fn(h.ptr, s.ptr, int(k), ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def lgw_lanczos_coeffs_poly(h: Handle, s: System, problem: Problem, options: Options, g: int,
                            x_lo: float, x_hi: float, alpha, beta, beta0, k_eff) -> None:
    p, o = problem.to_c(), options.to_c()
    pl = lgw_poly(int(g), float(x_lo), float(x_hi))
    _check(h, load_library().lgw_lanczos_coeffs_poly(
        h.ptr, s.ptr, ctypes.byref(p), ctypes.byref(o), ctypes.byref(pl), _ptr(alpha, "f64"),
        _ptr(beta, "f64"), _ptr(beta0, "f64"), _ptr(k_eff, "i32")))


def lgw_sigma_c_batched(h: Handle, systems: Sequence[System], problems: Sequence[Problem],
                        options: Options, sigmas, e_qps, z_qps=None,
                        report: bool = False) -> Optional[dict]:
    n = len(systems)
    sys_arr = (ctypes.c_void_p * n)(*[s.ptr.value for s in systems])
    prob_arr = (lgw_problem * n)(*[p.to_c() for p in problems])
    sig_arr = (ctypes.c_void_p * n)(*[_ptr(x, "f64") for x in sigmas])
    e_arr = (ctypes.c_void_p * n)(*[_ptr(x, "f64") for x in e_qps])
    z_arr = (ctypes.c_void_p * n)(*[_ptr(x, "f64") for x in z_qps]) if z_qps else None
    o = options.to_c()
    rep = lgw_report()
    _check(h, load_library().lgw_sigma_c_batched(
        h.ptr, n, sys_arr, prob_arr, ctypes.byref(o), sig_arr, e_arr, z_arr,
        ctypes.byref(rep) if report else None))
    return rep.as_dict() if report else None


def lgw_sigma_c_backward(h: Handle, s: System, problem: Problem, options: Options, dE,
                         dL=None, deps=None) -> None:
    p, o = problem.to_c(), options.to_c()
    _check(h, load_library().lgw_sigma_c_backward(
        h.ptr, s.ptr, ctypes.byref(p), ctypes.byref(o), _ptr(dE, "f64"), _ptr(dL, "f64"),
        _ptr(deps, "f64")))


def lgw_sigma_c_tda_backward(h: Handle, s: System, problem: Problem, options: Options, dE,
                             dL=None, deps=None) -> None:
    p, o = problem.to_c(), options.to_c()
    _check(h, load_library().lgw_sigma_c_tda_backward(
        h.ptr, s.ptr, ctypes.byref(p), ctypes.byref(o), _ptr(dE, "f64"), _ptr(dL, "f64"),
        _ptr(deps, "f64")))


def lgw_sigma_c_poly_backward(h: Handle, s: System, problem: Problem, options: Options, g: int,
                              x_lo: float, x_hi: float, dE, dL=None, deps=None) -> None:
    p, o = problem.to_c(), options.to_c()
    pl = lgw_poly(int(g), float(x_lo), float(x_hi))
    _check(h, load_library().lgw_sigma_c_poly_backward(
        h.ptr, s.ptr, ctypes.byref(p), ctypes.byref(o), ctypes.byref(pl), _ptr(dE, "f64"),
        _ptr(dL, "f64"), _ptr(deps, "f64")))


def lgw_sigma_from_coeffs_noalloc(h: Handle, s: System, problem: Problem, options: Options,
                                  alpha, beta, beta0, k_eff, sigma, e_qp, z_qp=None) -> None:
    """Allocation-free lgw_sigma_from_coeffs: all arrays must be CUDA tensors;
    the library's scratch is a fixed 16 MiB static device array (see
    include/lgw.h for the size limit and the concurrency rule)."""
    lib = load_library()
    fn = lib.lgw_sigma_from_coeffs_noalloc
    if fn.argtypes is None:
        P = ctypes.c_void_p
        fn.argtypes = [P, P, ctypes.POINTER(lgw_problem), ctypes.POINTER(lgw_options),
                       P, P, P, P, P, P, P]
        fn.restype = ctypes.c_int32
    p, o = problem.to_c(), options.to_c()
    _check(h, fn(h.ptr, s.ptr, ctypes.byref(p), ctypes.byref(o), _ptr(alpha, "f64"),
                 _ptr(beta, "f64"), _ptr(beta0, "f64"), _ptr(k_eff, "i32"),
                 _ptr(sigma, "f64"), _ptr(e_qp, "f64"), _ptr(z_qp, "f64")))
