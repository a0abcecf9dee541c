"""Thin ctypes binding of libsfac (include/sfac.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module only converts
Python values and torch tensors to the C ABI's plain pointers and sizes. It
raises loudly when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

from . import _build

SFAC_OK, SFAC_EINVAL, SFAC_EUNSUPPORTED, SFAC_ENOMEM, SFAC_ECUDA, SFAC_ETIMEOUT = range(6)
SFAC_FP64, SFAC_FP32 = 0, 1
STATUS_NAMES = {0: "SFAC_OK", 1: "SFAC_EINVAL", 2: "SFAC_EUNSUPPORTED", 3: "SFAC_ENOMEM",
                4: "SFAC_ECUDA", 5: "SFAC_ETIMEOUT"}


class SfacParams(ctypes.Structure):
    """Mirror of struct sfac_params."""

    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("alpha", ctypes.c_double * 3),
                ("eps", ctypes.c_double), ("tau", ctypes.c_double), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("prec", ctypes.c_int), ("reserved", ctypes.c_int)]


class SfacError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libsfac.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and _build.is_stale():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libsfac is not built ({_build.LIB}); run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.POINTER
    vp, ll, d = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_double
    sig = {
        "sfac_plan_create": (ctypes.c_int, [P(SfacParams), vp, P(vp)]),
        "sfac_plan_destroy": (ctypes.c_int, [vp]),
        "sfac_step": (ctypes.c_int, [vp, vp, ll, vp]),
        "sfac_solve": (ctypes.c_int, [vp, vp, d, vp]),
        "sfac_step_host": (ctypes.c_int, [vp, vp, ll, vp]),
        "sfac_axis_pass": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]),
        "sfac_plan_tables": (ctypes.c_int, [P(SfacParams), ctypes.c_int, P(d), P(d), P(d), P(d)]),
        "sfac_last_error": (ctypes.c_char_p, []),
        "sfac_version": (ctypes.c_int, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != SFAC_OK:
        msg = load().sfac_last_error().decode(errors="replace")
        raise SfacError(status, where, msg)


def make_params(n: Sequence[int], alpha: Sequence[float], eps: float, tau: float,
                a: float = -1.0, b: float = 1.0, prec: int = SFAC_FP64) -> SfacParams:
    p = SfacParams()
    p.dim = len(n)
    for l in range(3):
        p.n[l] = int(n[l]) if l < len(n) else 1
        p.alpha[l] = float(alpha[l]) if l < len(alpha) else 1.5
    p.eps, p.tau, p.a, p.b = float(eps), float(tau), float(a), float(b)
    p.prec = int(prec)
    p.reserved = 0
    return p


def _ptr(x) -> int:
    """Device or host address of a torch tensor / numpy array / int."""
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("field must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("field must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> int:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- the C ABI, one function per entry point ---------------------------------

def sfac_plan_create(params: SfacParams, stream=None) -> int:
    out = ctypes.c_void_p()
    _check(load().sfac_plan_create(ctypes.byref(params), _stream(stream), ctypes.byref(out)),
           "sfac_plan_create")
    return out.value


def sfac_plan_destroy(plan: int) -> None:
    _check(load().sfac_plan_destroy(plan), "sfac_plan_destroy")


def sfac_step(plan: int, u, nsteps: int, stream=None) -> None:
    _check(load().sfac_step(plan, _ptr(u), int(nsteps), _stream(stream)), "sfac_step")


def sfac_solve(plan: int, u, T: float, stream=None) -> None:
    _check(load().sfac_solve(plan, _ptr(u), float(T), _stream(stream)), "sfac_solve")


def sfac_step_host(plan: int, u_host, nsteps: int, stream=None) -> None:
    _check(load().sfac_step_host(plan, _ptr(u_host), int(nsteps), _stream(stream)), "sfac_step_host")


def sfac_axis_pass(plan: int, u, axis: int, jq_in: int = 0, jq_out: int = 0, stream=None) -> None:
    _check(load().sfac_axis_pass(plan, _ptr(u), int(axis), int(jq_in), int(jq_out), _stream(stream)),
           "sfac_axis_pass")


def sfac_plan_tables(params: SfacParams, axis: int):
    """Host-only FP64 tables of one axis: (lambda, mu, b first column, J^Q constants)."""
    import numpy as np
    n = params.n[axis]
    lam, mu, bcol, jq = (np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(4))
    dp = lambda v: v.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(load().sfac_plan_tables(ctypes.byref(params), int(axis), dp(lam), dp(mu), dp(bcol), dp(jq)),
           "sfac_plan_tables")
    return lam, mu, bcol, jq


def sfac_last_error() -> str:
    return load().sfac_last_error().decode(errors="replace")


def sfac_version() -> int:
    return load().sfac_version()


# ---- convenience wrapper -------------------------------------------------------

class Plan:
    """Owns one sfac_plan. The field is a contiguous CUDA tensor of shape
    (n_d, ..., n_1) and dtype float64 (FP64 plans) or float32 (FP32 plans)."""

    def __init__(self, n: Sequence[int], alpha: Sequence[float], eps: float, tau: float,
                 a: float = -1.0, b: float = 1.0, prec: int = SFAC_FP64, stream=None):
        self.params = make_params(n, alpha, eps, tau, a, b, prec)
        self.n, self.prec = tuple(int(v) for v in n), prec
        self.handle = sfac_plan_create(self.params, stream)

    @classmethod
    def for_problem(cls, problem, prec: int = SFAC_FP64, stream=None) -> "Plan":
        return cls(problem.n, problem.alpha, problem.eps, problem.tau, problem.a, problem.b, prec, stream)

    @property
    def shape(self):
        return tuple(reversed(self.n))

    def _check_field(self, u):
        import torch
        want = torch.float64 if self.prec == SFAC_FP64 else torch.float32
        if u.dtype != want or not u.is_cuda or tuple(u.shape) != self.shape or not u.is_contiguous():
            raise ValueError(f"field must be a contiguous CUDA {want} tensor of shape {self.shape}")

    def step(self, u, nsteps: int, stream=None):
        self._check_field(u)
        sfac_step(self.handle, u, nsteps, stream)
        return u

    def solve(self, u, T: float, stream=None):
        self._check_field(u)
        sfac_solve(self.handle, u, T, stream)
        return u

    def axis_pass(self, u, axis: int, jq_in: int = 0, jq_out: int = 0, stream=None):
        self._check_field(u)
        sfac_axis_pass(self.handle, u, axis, jq_in, jq_out, stream)
        return u

    def step_host(self, u_host, nsteps: int, stream=None):
        sfac_step_host(self.handle, u_host, nsteps, stream)
        return u_host

    def close(self):
        if getattr(self, "handle", None):
            sfac_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
