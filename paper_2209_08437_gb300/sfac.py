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
        "sfac_diagnostics": (ctypes.c_int, [vp, vp, P(d), vp]),
        "sfac_plan_info": (ctypes.c_int, [vp, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int)]),
        "sfac_plan_kernel": (ctypes.c_int, [vp, ctypes.c_int, vp, P(ctypes.c_int)]),
        "sfac_plan_check": (ctypes.c_int, [vp, vp]),
        "sfac_plan_step_kernel": (ctypes.c_int, [vp, ll, P(ctypes.c_int)]),
        "sfac_plan_host_route": (ctypes.c_int, [vp, vp, ll, P(ctypes.c_int)]),
        "sfac_plan_set_wait_limit": (ctypes.c_int, [vp, ll, ctypes.c_int]),
        "sfac_plan_tables": (ctypes.c_int, [P(SfacParams), ctypes.c_int, P(d), P(d), P(d), P(d)]),
        "sfac_batch_create": (ctypes.c_int, [P(SfacParams), ctypes.c_int, vp, P(vp)]),
        "sfac_batch_destroy": (ctypes.c_int, [vp]),
        "sfac_batch_prepare": (ctypes.c_int, [vp, P(vp), P(ll), vp]),
        "sfac_batch_launch": (ctypes.c_int, [vp, vp]),
        "sfac_batch_wait": (ctypes.c_int, [vp, vp]),
        "sfac_batch_step": (ctypes.c_int, [vp, P(vp), P(ll), vp]),
        "sfac_batch_autotune": (ctypes.c_int, [vp, ctypes.c_int, vp, P(ctypes.c_int)]),
        "sfac_batch_set_config": (ctypes.c_int, [vp, ctypes.c_int]),
        "sfac_batch_get_config": (ctypes.c_int, [vp, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int),
                                                 P(ctypes.c_int)]),
        "sfac_batch_num_configs": (ctypes.c_int, []),
        "sfac_batch_set_wait_limit": (ctypes.c_int, [vp, ll, ctypes.c_int]),
        "sfac_batch_launch_noalloc": (ctypes.c_int, [vp, vp]),
        "sfac_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.c_int, vp, P(vp)]),
        "sfac_server_destroy": (ctypes.c_int, [vp]),
        "sfac_server_request_bytes": (ctypes.c_int, [P(SfacParams), P(ctypes.c_size_t)]),
        "sfac_server_admit": (ctypes.c_int, [vp, P(SfacParams), vp, ll, P(ctypes.c_int)]),
        "sfac_server_round": (ctypes.c_int, [vp, ll, ctypes.c_int, vp, P(ctypes.c_int)]),
        "sfac_server_set_wait_limit": (ctypes.c_int, [vp, ll, ctypes.c_int]),
        "sfac_server_wait": (ctypes.c_int, [vp, vp, P(ctypes.c_int), ctypes.c_int, P(ctypes.c_int)]),
        "sfac_server_fetch": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int]),
        "sfac_server_info": (ctypes.c_int, [vp, P(ctypes.c_size_t), P(ctypes.c_size_t), P(ctypes.c_int),
                                            P(ctypes.c_int)]),
        "sfac_probe_fma": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ll, vp, vp]),
        "sfac_probe_jq": (ctypes.c_int, [ctypes.c_int, vp, vp, ll, ctypes.c_double, ctypes.c_double, vp]),
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


def sfac_plan_info(plan: int, axis: int):
    """(FFT length, padded?) of the plan's pass along `axis`."""
    L, pad = ctypes.c_int(), ctypes.c_int()
    _check(load().sfac_plan_info(plan, int(axis), ctypes.byref(L), ctypes.byref(pad)), "sfac_plan_info")
    return L.value, bool(pad.value)


SFAC_KERNEL_CTA, SFAC_KERNEL_WARP, SFAC_KERNEL_STAGED = range(3)


def sfac_plan_kernel(plan: int, axis: int, u) -> int:
    """Which kernel (SFAC_KERNEL_*) a pass along `axis` would run for the field u."""
    kind = ctypes.c_int()
    _check(load().sfac_plan_kernel(plan, int(axis), _ptr(u), ctypes.byref(kind)), "sfac_plan_kernel")
    return kind.value


SFAC_STEP_PASSES, SFAC_STEP_WHOLE = range(2)


def sfac_plan_step_kernel(plan: int, nsteps: int) -> int:
    """SFAC_STEP_WHOLE if sfac_step runs a call of nsteps steps in one launch."""
    kind = ctypes.c_int()
    _check(load().sfac_plan_step_kernel(plan, int(nsteps), ctypes.byref(kind)), "sfac_plan_step_kernel")
    return kind.value


SFAC_HOST_COPY, SFAC_HOST_MAPPED, SFAC_HOST_MAPPED_IN = range(3)


def sfac_plan_host_route(plan: int, u_host, nsteps: int) -> int:
    """SFAC_HOST_* route that sfac_step_host takes for the host buffer u_host."""
    route = ctypes.c_int()
    _check(load().sfac_plan_host_route(plan, _ptr(u_host), int(nsteps), ctypes.byref(route)), "sfac_plan_host_route")
    return route.value


def sfac_plan_check(plan: int, stream=None) -> None:
    """Synchronise; raise SfacError(SFAC_ETIMEOUT) if a pass gave up a bounded wait."""
    _check(load().sfac_plan_check(plan, _stream(stream)), "sfac_plan_check")


def sfac_plan_set_wait_limit(plan: int, wait_cycles: int, hold: int = 0) -> None:
    """Per-wait limit (SM cycles) of the plan's bounded waits; hold=1 is the test hook."""
    _check(load().sfac_plan_set_wait_limit(plan, int(wait_cycles), int(hold)), "sfac_plan_set_wait_limit")


def sfac_diagnostics(plan: int, u, stream=None):
    """(max |u|, discrete energy) of the field u (Examples 4 and 5)."""
    out = (ctypes.c_double * 2)()
    _check(load().sfac_diagnostics(plan, _ptr(u), out, _stream(stream)), "sfac_diagnostics")
    return out[0], out[1]


def sfac_plan_tables(params: SfacParams, axis: int):
    """Host-only FP64 tables of one axis: (lambda, mu, b first column, J^Q constants)."""
    import numpy as np
    n = params.n[axis]
    lam, mu, bcol, jq = (np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(4))
    dp = lambda v: v.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(load().sfac_plan_tables(ctypes.byref(params), int(axis), dp(lam), dp(mu), dp(bcol), dp(jq)),
           "sfac_plan_tables")
    return lam, mu, bcol, jq


PROBE_THREADS, PROBE_CHAINS, PROBE_UNROLL = 256, 8, 16


def sfac_probe_fma(kind: int, blocks: int, iters: int, out_dev, stream=None) -> float:
    """Enqueue the multiply-add rate probe; returns the flops the launch performs."""
    _check(load().sfac_probe_fma(int(kind), int(blocks), int(iters), _ptr(out_dev), _stream(stream)),
           "sfac_probe_fma")
    lanes = 2 if kind == 2 else 1
    return 2.0 * lanes * blocks * PROBE_THREADS * PROBE_CHAINS * PROBE_UNROLL * iters


def sfac_probe_jq(prec: int, v_dev, out_dev, E: float, one_minus_E: float, stream=None) -> None:
    """Enqueue J^Q on the values of v_dev (the passes' own device code) into out_dev."""
    _check(load().sfac_probe_jq(int(prec), _ptr(v_dev), _ptr(out_dev), int(v_dev.numel()), float(E),
                                float(one_minus_E), _stream(stream)), "sfac_probe_jq")


def sfac_last_error() -> str:
    return load().sfac_last_error().decode(errors="replace")


def sfac_version() -> int:
    return load().sfac_version()


def _ptr_array(fields):
    arr = (ctypes.c_void_p * len(fields))()
    for i, f in enumerate(fields):
        arr[i] = _ptr(f)
    return arr


def _steps_array(nsteps):
    arr = (ctypes.c_longlong * len(nsteps))()
    for i, v in enumerate(nsteps):
        arr[i] = int(v)
    return arr


def sfac_batch_create(params_list, stream=None) -> int:
    arr = (SfacParams * len(params_list))(*params_list)
    out = ctypes.c_void_p()
    _check(load().sfac_batch_create(arr, len(params_list), _stream(stream), ctypes.byref(out)), "sfac_batch_create")
    return out.value


def sfac_batch_destroy(batch: int) -> None:
    _check(load().sfac_batch_destroy(batch), "sfac_batch_destroy")


def sfac_batch_prepare(batch: int, fields, nsteps, stream=None) -> None:
    _check(load().sfac_batch_prepare(batch, _ptr_array(fields), _steps_array(nsteps), _stream(stream)),
           "sfac_batch_prepare")


def sfac_batch_launch(batch: int, stream=None) -> None:
    _check(load().sfac_batch_launch(batch, _stream(stream)), "sfac_batch_launch")


def sfac_batch_launch_noalloc(batch: int, stream=None) -> None:
    """sfac_batch_launch without any allocation: the counters live in the
    library's fixed device array (for callers that cannot allocate at launch)."""
    _check(load().sfac_batch_launch_noalloc(batch, _stream(stream)), "sfac_batch_launch_noalloc")


def sfac_batch_wait(batch: int, stream=None) -> None:
    _check(load().sfac_batch_wait(batch, _stream(stream)), "sfac_batch_wait")


def sfac_batch_step(batch: int, fields, nsteps, stream=None) -> None:
    _check(load().sfac_batch_step(batch, _ptr_array(fields), _steps_array(nsteps), _stream(stream)),
           "sfac_batch_step")


def sfac_batch_autotune(batch: int, max_steps: int, stream=None) -> int:
    choice = ctypes.c_int(-1)
    _check(load().sfac_batch_autotune(batch, int(max_steps), _stream(stream), ctypes.byref(choice)),
           "sfac_batch_autotune")
    return choice.value


def sfac_batch_set_config(batch: int, config: int) -> None:
    _check(load().sfac_batch_set_config(batch, int(config)), "sfac_batch_set_config")


def sfac_batch_get_config(batch: int):
    vals = [ctypes.c_int() for _ in range(4)]
    _check(load().sfac_batch_get_config(batch, *[ctypes.byref(v) for v in vals]), "sfac_batch_get_config")
    return tuple(v.value for v in vals)


def sfac_batch_num_configs() -> int:
    return load().sfac_batch_num_configs()


def sfac_batch_set_wait_limit(batch: int, spin_limit: int, hold_instance: int = -1) -> None:
    _check(load().sfac_batch_set_wait_limit(batch, int(spin_limit), int(hold_instance)),
           "sfac_batch_set_wait_limit")


def sfac_server_create(arena_bytes: int, max_slots: int, prec: int = SFAC_FP32, stream=None) -> int:
    out = ctypes.c_void_p()
    _check(load().sfac_server_create(int(arena_bytes), int(max_slots), int(prec), _stream(stream),
                                     ctypes.byref(out)), "sfac_server_create")
    return out.value


def sfac_server_destroy(server: int) -> None:
    _check(load().sfac_server_destroy(server), "sfac_server_destroy")


def sfac_server_request_bytes(params: SfacParams) -> int:
    out = ctypes.c_size_t()
    _check(load().sfac_server_request_bytes(ctypes.byref(params), ctypes.byref(out)), "sfac_server_request_bytes")
    return out.value


def sfac_server_admit(server: int, params: SfacParams, u0_host, nsteps: int):
    """Slot number, or None when no slot or arena block is free (SFAC_ENOMEM)."""
    slot = ctypes.c_int(-1)
    st = load().sfac_server_admit(server, ctypes.byref(params), _ptr(u0_host), int(nsteps), ctypes.byref(slot))
    if st == SFAC_ENOMEM:
        return None
    _check(st, "sfac_server_admit")
    return slot.value


def sfac_server_round(server: int, chunk: int, shape: int = 0, stream=None) -> bool:
    """Enqueue a round; False when no slot had open steps (nothing enqueued)."""
    launched = ctypes.c_int(0)
    _check(load().sfac_server_round(server, int(chunk), int(shape), _stream(stream), ctypes.byref(launched)),
           "sfac_server_round")
    return bool(launched.value)


def sfac_server_wait(server: int, capacity: int, stream=None):
    """Finished slots of the oldest round in flight. If that round gave up
    (SFAC_ETIMEOUT), raises SfacError whose `finished` lists the finished
    slots, failed ones included (fetching those raises SFAC_ETIMEOUT)."""
    buf = (ctypes.c_int * max(capacity, 1))()
    n = ctypes.c_int(0)
    st = load().sfac_server_wait(server, _stream(stream), buf, capacity, ctypes.byref(n))
    done = [buf[i] for i in range(min(n.value, capacity))]
    if st != SFAC_OK:
        err = SfacError(st, "sfac_server_wait", load().sfac_last_error().decode(errors="replace"))
        err.finished = done
        raise err
    return done


def sfac_server_set_wait_limit(server: int, spin_limit: int, hold_slot: int = -1) -> None:
    _check(load().sfac_server_set_wait_limit(server, int(spin_limit), int(hold_slot)), "sfac_server_set_wait_limit")


def sfac_server_fetch(server: int, slot: int, u_host=None, release: bool = True) -> None:
    _check(load().sfac_server_fetch(server, int(slot), _ptr(u_host) if u_host is not None else None,
                                    1 if release else 0), "sfac_server_fetch")


def sfac_server_info(server: int) -> dict:
    fb, lf, act, cap = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int()
    _check(load().sfac_server_info(server, ctypes.byref(fb), ctypes.byref(lf), ctypes.byref(act),
                                   ctypes.byref(cap)), "sfac_server_info")
    return {"free_bytes": fb.value, "largest_free": lf.value, "active": act.value, "capacity": cap.value}


# ---- convenience wrappers ------------------------------------------------------

class Server:
    """Owns one sfac_server (continuous batching of requests of different sizes)."""

    def __init__(self, arena_bytes: int, max_slots: int, prec: int = SFAC_FP32, stream=None):
        self.prec, self.capacity = prec, int(max_slots)
        self.handle = sfac_server_create(arena_bytes, max_slots, prec, stream)

    def admit(self, problem, u0_host, nsteps: int):
        p = make_params(problem.n, problem.alpha, problem.eps, problem.tau, problem.a, problem.b, self.prec)
        return sfac_server_admit(self.handle, p, u0_host, nsteps)

    def round(self, chunk: int, shape: int = 0, stream=None) -> bool:
        return sfac_server_round(self.handle, chunk, shape, stream)

    def set_wait_limit(self, spin_limit: int, hold_slot: int = -1):
        sfac_server_set_wait_limit(self.handle, spin_limit, hold_slot)

    def wait(self, stream=None):
        return sfac_server_wait(self.handle, self.capacity, stream)

    def fetch(self, slot: int, u_host=None, release: bool = True):
        sfac_server_fetch(self.handle, slot, u_host, release)

    def info(self) -> dict:
        return sfac_server_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            sfac_server_destroy(self.handle)
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


class Batch:
    """Owns one sfac_batch: many independent problems in one persistent launch.
    `problems` are sfac_inputs.Problem-like objects (n, alpha, eps, tau, a, b)."""

    def __init__(self, problems, prec: int = SFAC_FP32, stream=None):
        self.params = [make_params(p.n, p.alpha, p.eps, p.tau, p.a, p.b, prec) for p in problems]
        self.shapes = [tuple(reversed(tuple(int(v) for v in p.n))) for p in problems]
        self.prec = prec
        self.handle = sfac_batch_create(self.params, stream)

    def step(self, fields, nsteps, stream=None):
        sfac_batch_step(self.handle, fields, nsteps, stream)

    def prepare(self, fields, nsteps, stream=None):
        sfac_batch_prepare(self.handle, fields, nsteps, stream)

    def launch(self, stream=None):
        sfac_batch_launch(self.handle, stream)

    def wait(self, stream=None):
        sfac_batch_wait(self.handle, stream)

    def autotune(self, max_steps: int = 10, stream=None) -> int:
        return sfac_batch_autotune(self.handle, max_steps, stream)

    def close(self):
        if getattr(self, "handle", None):
            sfac_batch_destroy(self.handle)
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

    def diagnostics(self, u, stream=None):
        """(max |u|, discrete energy E(u)) of a field of this plan."""
        self._check_field(u)
        return sfac_diagnostics(self.handle, u, stream)

    def step_host(self, u_host, nsteps: int, stream=None):
        sfac_step_host(self.handle, u_host, nsteps, stream)
        return u_host

    def kernel(self, axis: int, u) -> int:
        """SFAC_KERNEL_* that a pass along `axis` runs for the field u."""
        return sfac_plan_kernel(self.handle, axis, u)

    def host_route(self, u_host, nsteps: int) -> int:
        """SFAC_HOST_* route that step_host takes for the host buffer u_host."""
        return sfac_plan_host_route(self.handle, u_host, nsteps)

    def step_kernel(self, nsteps: int) -> int:
        """SFAC_STEP_* that sfac_step uses for a call of nsteps steps."""
        return sfac_plan_step_kernel(self.handle, nsteps)

    def check(self, stream=None):
        """Synchronise `stream` and raise if a pass gave up a bounded wait."""
        sfac_plan_check(self.handle, stream)

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
