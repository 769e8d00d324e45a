"""GB300 (sm_103a) explicit finite-difference stepper for phase-field and
reaction-diffusion models on periodic grids (SymPhas 2.0, arXiv 2511.10508).

The Python layer only marshals arguments into ``libsp.so`` (``include/sp.h``);
fields live in device memory and every step runs in the library's CUDA
kernels.  Streams may be torch CUDA streams (``torch.cuda.Stream``) or raw
``cudaStream_t`` integers.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as N
from ._native import (ALLEN_CAHN, BF16_F32, CAHN_HILLIARD, F32, F64, FLAG_AUTOTUNE, FLAG_BF16_NO_BOUND, FREE_ENERGY, GRAY_SCOTT, IC_CONSTANT,
                      IC_NOISE, LAP_5, LAP_7, LAP_9BOX, LAP_9CROSS4, LAP_13CROSS4, LAP_27, LAP_DEFAULT, LAP_GENERATED, MASS,
                      MAX_U, MIN_U, MODEL_C, MODEL_H, SCHEME_FD, SCHEME_SPECTRAL, SUM_U, SUM_V, SUMSQ_U, SpError)

__all__ = ["Simulation", "Server", "Result", "params", "admission_order", "check_stability", "SpError", "ALLEN_CAHN", "CAHN_HILLIARD", "GRAY_SCOTT",
           "MODEL_C", "MODEL_H", "SCHEME_FD", "SCHEME_SPECTRAL",
           "LAP_5", "LAP_9BOX", "LAP_9CROSS4", "LAP_7", "LAP_27", "LAP_13CROSS4", "LAP_DEFAULT", "LAP_GENERATED",
           "stencil_weights", "F64", "F32",
           "BF16_F32", "IC_NOISE", "IC_CONSTANT", "FLAG_AUTOTUNE", "FLAG_BF16_NO_BOUND", "MASS", "FREE_ENERGY", "SUM_U", "SUM_V", "MIN_U", "MAX_U",
           "SUMSQ_U"]

_STORAGE = {F64: np.float64, F32: np.float32, BF16_F32: np.uint16}


def params(model: int, dims: int, **kw) -> N.sp_params:
    """sp_params with the library defaults, overridden by keyword arguments."""
    p = N.sp_params()
    N.lib().sp_params_default(model, dims, ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(f"sp_params has no field {k!r}")
        setattr(p, k, v)
    return p


def stencil_weights(order: int, dims: int):
    """Kernel weights (dims w_0, w_1, ..., w_r) and lambda_max of the generated cross
    Laplacian of accuracy ``order`` (see sp_stencil_weights)."""
    w = (ctypes.c_double * 5)()
    lm = ctypes.c_double(0.0)
    N.check(N.lib().sp_stencil_weights(int(order), int(dims), w, ctypes.byref(lm)), "sp_stencil_weights")
    return [w[i] for i in range(order // 2 + 1)], lm.value


def check_stability(model: int, dims: int, h: float, dt: float, prm: N.sp_params | None = None):
    """(stable, dt*max|sigma|) from the library's host-only check."""
    prm = prm if prm is not None else params(model, dims)
    f = ctypes.c_double(0.0)
    rc = N.lib().sp_check_stability(model, dims, h, dt, ctypes.byref(prm), ctypes.byref(f))
    if rc not in (N.SP_OK, N.SP_EUNSTABLE):
        raise SpError(rc, "sp_check_stability")
    return rc == N.SP_OK, f.value


def probe_fp64_rate(stream=None) -> float:
    """Sustained FP64 FMA rate of the current device in Gop/s (sp_probe_fp64_rate)."""
    g = ctypes.c_double(0.0)
    N.check(N.lib().sp_probe_fp64_rate(_stream_ptr(stream), ctypes.byref(g)), "sp_probe_fp64_rate")
    return g.value


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


class Simulation:
    """One resident grid.  ``shape`` is numpy order: (ny, nx) or (nz, ny, nx)."""

    def __init__(self, model: int, shape, *, h: float = 1.0, dt: float, prm: N.sp_params | None = None, **kw):
        self.model = model
        self.shape = tuple(int(s) for s in shape)
        self.dims = len(self.shape)
        self.prm = prm if prm is not None else params(model, self.dims, **kw)
        xyz = (ctypes.c_int64 * 3)(*(list(self.shape[::-1]) + [1] * (3 - self.dims)))
        h_ = ctypes.c_void_p()
        N.check(N.lib().sp_create(model, self.dims, xyz, h, dt, ctypes.byref(self.prm), ctypes.byref(h_)),
                "sp_create")
        self._h = h_
        self.nfields = (1 + len(shape)) if model == MODEL_H else (2 if model in (GRAY_SCOTT, MODEL_C) else 1)
        self.dtype = self.prm.dtype

    # -- lifecycle
    def close(self) -> None:
        if getattr(self, "_h", None):
            N.lib().sp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls
    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def step(self, n: int = 1, stream=None) -> None:
        N.check(N.lib().sp_step(self._h, int(n), _stream_ptr(stream)), "sp_step")

    def read(self, field: int = 0, as_f64: bool = True, stream=None) -> np.ndarray:
        dt = np.float64 if as_f64 else _STORAGE[self.dtype]
        out = np.empty(self.shape, dtype=dt)
        N.check(N.lib().sp_read(self._h, field, out.ctypes.data, out.nbytes, int(as_f64), _stream_ptr(stream)),
                "sp_read")
        return out

    def write(self, field: int, values, stream=None) -> None:
        arr = np.ascontiguousarray(values)
        is_f64 = arr.dtype == np.float64
        if not is_f64 and arr.dtype != _STORAGE[self.dtype]:
            raise TypeError(f"write expects float64 or the storage dtype, got {arr.dtype}")
        if arr.shape != self.shape:
            raise ValueError(f"shape {arr.shape} != {self.shape}")
        N.check(N.lib().sp_write(self._h, field, arr.ctypes.data, arr.nbytes, int(is_f64), _stream_ptr(stream)),
                "sp_write")

    def reduce(self, what: int, stream=None) -> float:
        out = ctypes.c_double(0.0)
        N.check(N.lib().sp_reduce(self._h, what, ctypes.byref(out), _stream_ptr(stream)), "sp_reduce")
        return out.value

    def devptr(self, field: int = 0) -> int:
        p = ctypes.c_void_p()
        N.check(N.lib().sp_field_devptr(self._h, field, ctypes.byref(p)), "sp_field_devptr")
        return int(p.value)

    def autotune(self, stream=None) -> int:
        """Pick the fastest launch configuration for this grid by timing the
        candidates; returns the time steps taken meanwhile (see sp_autotune)."""
        n = ctypes.c_int64(0)
        N.check(N.lib().sp_autotune(self._h, _stream_ptr(stream), ctypes.byref(n)), "sp_autotune")
        return n.value

    @property
    def launch_config(self):
        """(steps fused per launch, kernel family) currently used."""
        a, b = ctypes.c_int(0), ctypes.c_int(0)
        N.check(N.lib().sp_launch_config(self._h, ctypes.byref(a), ctypes.byref(b)), "sp_launch_config")
        return a.value, b.value

    @launch_config.setter
    def launch_config(self, cfg) -> None:
        spl, variant = cfg
        N.check(N.lib().sp_set_launch_config(self._h, int(spl), int(variant)), "sp_set_launch_config")

    @property
    def steps_taken(self) -> int:
        s = ctypes.c_int64(0)
        N.check(N.lib().sp_steps_taken(self._h, ctypes.byref(s)), "sp_steps_taken")
        return s.value

    def field_tensor(self, field: int = 0):
        """Zero-copy torch view of the current level (valid until the next step).

        The view is read on torch's stream; steps enqueued on another stream (the
        simulation's own one when ``stream`` was None) must have completed first,
        e.g. after ``torch.cuda.synchronize()``."""
        import torch

        tdt = {F64: torch.float64, F32: torch.float32, BF16_F32: torch.bfloat16}[self.dtype]
        esize = {F64: 8, F32: 4, BF16_F32: 2}[self.dtype]
        strides = []
        acc = 1
        for s in reversed(self.shape):
            strides.append(acc * esize)
            acc *= s
        typestr = {F64: "<f8", F32: "<f4", BF16_F32: "<u2"}[self.dtype]

        class _CAI:
            __cuda_array_interface__ = {"shape": self.shape, "typestr": typestr,
                                        "data": (self.devptr(field), False), "version": 2,
                                        "strides": tuple(reversed(strides))}

        t = torch.as_tensor(_CAI(), device="cuda")
        return t.view(tdt) if self.dtype == BF16_F32 else t


class Result:
    """Outcome of a served request (a copy; the server's buffers may be released)."""

    def __init__(self, res: N.sp_result, shape, nfields: int):
        self.status = res.status
        self.steps_done = res.steps_done
        self.t_submit, self.t_admit, self.t_finish = res.t_submit, res.t_admit, res.t_finish
        self.mass = res.mass
        self.fields = None
        if res.fields and res.n_values:
            flat = np.ctypeslib.as_array(res.fields, shape=(res.n_values,)).copy()
            self.fields = flat.reshape((nfields,) + tuple(shape))

    @property
    def latency(self) -> float:
        """Time to result: finish - submit (seconds)."""
        return self.t_finish - self.t_submit


def set_wait_polls(polls: int) -> None:
    """Test hook: polls before the kernels' bounded device waits give up (0 the
    default, negative: give up at once); a step whose wait gave up makes the next
    read or reduction of that simulation raise SpError(SP_ETIMEOUT)."""
    N.lib().sp_set_wait_polls(int(polls))


def admission_order(bytes_, priorities, free_bytes: int, free_slots: int) -> list[int]:
    """The server's admission rule (sp_admission_order): indices of the pending
    requests admitted now, in admission order."""
    n = len(bytes_)
    b = (ctypes.c_size_t * max(n, 1))(*[int(x) for x in bytes_])
    p = (ctypes.c_int * max(n, 1))(*[int(x) for x in priorities])
    o = (ctypes.c_int * max(n, 1))()
    k = N.lib().sp_admission_order(n, b, p, int(free_bytes), int(free_slots), o)
    if k < 0:
        raise SpError(N.SP_EINVAL, "sp_admission_order")
    return [o[i] for i in range(k)]


class Server:
    """Continuous-batching server (``sp_server_*``): submit grids at any time,
    collect results by ticket."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 256, quantum_steps: int = 50):
        h = ctypes.c_void_p()
        N.check(N.lib().sp_server_create(int(hbm_budget_bytes), int(max_slots), int(quantum_steps),
                                         ctypes.byref(h)), "sp_server_create")
        self._h = h
        self._meta = {}

    def submit(self, model: int, shape, *, dt: float, nsteps: int, h: float = 1.0, prm: N.sp_params | None = None,
               return_fields: bool = False, fault: int = 0, priority: int = 0, **kw) -> int:
        shape = tuple(int(s) for s in shape)
        dims = len(shape)
        r = N.sp_request()
        r.model, r.dims = model, dims
        xyz = list(shape[::-1]) + [1] * (3 - dims)
        for i in range(3):
            r.shape[i] = xyz[i]
        r.h, r.dt = h, dt
        r.params = prm if prm is not None else params(model, dims, **kw)
        r.nsteps = int(nsteps)
        r.return_fields = int(bool(return_fields))
        r.fault = int(fault)
        r.priority = int(priority)
        t = ctypes.c_uint64(0)
        N.check(N.lib().sp_submit(self._h, ctypes.byref(r), ctypes.byref(t)), "sp_submit")
        self._meta[t.value] = (shape, 2 if model in (GRAY_SCOTT, MODEL_C) else 1)
        return t.value

    def poll(self, ticket: int):
        """(status, Result or None): SP_PENDING (8) while running."""
        res = N.sp_result()
        rc = N.lib().sp_poll(self._h, ticket, ctypes.byref(res))
        if rc == N.SP_PENDING:
            return rc, None
        shape, nf = self._meta[ticket]
        return rc, Result(res, shape, nf)

    def wait(self, ticket: int, timeout: float = 600.0) -> Result:
        res = N.sp_result()
        rc = N.lib().sp_wait(self._h, ticket, float(timeout), ctypes.byref(res))
        if rc == N.SP_ETIMEOUT:
            raise TimeoutError(f"ticket {ticket} not done after {timeout} s")
        shape, nf = self._meta[ticket]
        out = Result(res, shape, nf)
        if rc != N.SP_OK:
            raise SpError(rc, f"request {ticket}")
        return out

    def release(self, ticket: int) -> None:
        N.check(N.lib().sp_release(self._h, ticket), "sp_release")
        self._meta.pop(ticket, None)

    def stats(self) -> dict:
        st = N.sp_server_stats()
        N.check(N.lib().sp_server_get_stats(self._h, ctypes.byref(st)), "sp_server_get_stats")
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self) -> None:
        if getattr(self, "_h", None):
            N.lib().sp_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
