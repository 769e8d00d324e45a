"""FP64 CPU oracle for the explicit finite-difference step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The GPU library never imports it and it imports
nothing of the GPU library: the two share no code.

The arithmetic lives in ``sp_oracle.c`` (plain C, OpenMP over rows, FP64,
compiled with ``-ffp-contract=off``); this module compiles it and wraps it for
numpy arrays.  See the C file's header for the equations (SymPhas 2.0, Eq.
(model-a), Eq. (model-b), Gray-Scott in Pearson's form), the stencils and the
fixed evaluation order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

AC, CH, GS, MC, MH = 0, 1, 2, 3, 4
TWO_FIELD = (GS, MC)
S1, S2, S3, S4, S5, S6 = range(6)
STENCIL_DIMS = {S1: 2, S2: 2, S3: 2, S4: 3, S5: 3, S6: 3}
STENCIL_RADIUS = {S1: 1, S2: 1, S3: 2, S4: 1, S5: 1, S6: 2}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, no GPU needed)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    """The loaded oracle library.  ``SP_ORACLE_LIB`` names another build of the same
    source (used by the mutation test, which plants mistakes in a copy)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("SP_ORACLE_LIB")
            if not path:
                path = build()
            L = ctypes.CDLL(path)
            i64, dbl, ptr, u64 = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_uint64
            c_int = ctypes.c_int
            L.or_num_threads.restype = c_int
            L.or_stencil_q.restype = c_int
            L.or_stencil_q.argtypes = [c_int]
            L.or_stencil_sum.argtypes = [c_int, i64, i64, i64, ptr, ptr]
            L.or_laplacian.argtypes = [c_int, i64, i64, i64, dbl, ptr, ptr]
            L.or_chemical_potential.argtypes = [c_int, i64, i64, i64, dbl, ptr, ptr, ptr]
            L.or_step.argtypes = [c_int, c_int, i64, i64, i64, dbl, dbl, ptr, ptr, ptr, i64]
            L.or_splitmix64_nth.restype = u64
            L.or_splitmix64_nth.argtypes = [u64, u64]
            L.or_u01.restype = dbl
            L.or_u01.argtypes = [u64, u64]
            L.or_initial_condition.argtypes = [c_int, c_int, i64, i64, i64, u64, dbl, dbl, i64, i64, ptr, ptr]
            L.or_initial_condition_window.argtypes = [c_int, c_int, i64, i64, i64, u64, dbl, dbl, i64, i64,
                                                      i64, i64, i64, i64, i64, i64, ptr, ptr]
            L.or_sum.restype = dbl
            L.or_sum.argtypes = [ptr, i64]
            L.or_mass.restype = dbl
            L.or_mass.argtypes = [c_int, i64, i64, i64, dbl, ptr]
            L.or_free_energy.restype = dbl
            L.or_free_energy.argtypes = [c_int, i64, i64, i64, dbl, dbl, dbl, ptr]
            L.or_step_gen.restype = c_int
            L.or_step_gen.argtypes = [c_int, c_int, c_int, ptr, i64, i64, i64, dbl, dbl, ptr, ptr, ptr, i64]
            L.or_step_h.restype = c_int
            L.or_step_h.argtypes = [c_int, i64, i64, i64, dbl, dbl, ptr, ptr, ptr, ptr, ptr, i64]
            L.or_initial_condition_h.restype = c_int
            L.or_initial_condition_h.argtypes = [c_int, i64, i64, i64, ctypes.c_uint64, dbl, dbl, ptr, ptr, ptr, ptr]
            L.or_free_energy_h.restype = dbl
            L.or_free_energy_h.argtypes = [c_int, i64, i64, i64, dbl, dbl, dbl, ptr, ptr, ptr, ptr]
            L.or_free_energy_c.restype = dbl
            L.or_free_energy_c.argtypes = [c_int, i64, i64, i64, dbl, dbl, dbl, dbl, ptr, ptr]
            L.or_rel_l2.restype = dbl
            L.or_rel_l2.argtypes = [ptr, ptr, i64]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _shape3(a: np.ndarray, dims: int):
    """numpy shape (ny, nx) or (nz, ny, nx) -> (nx, ny, nz)."""
    if dims == 2:
        ny, nx = a.shape
        return nx, ny, 1
    nz, ny, nx = a.shape
    return nx, ny, nz


def params(c1=1.0, c2=1.0, kappa=1.0, Du=0.16, Dv=0.08, F=0.035, k=0.065, c3=0.5) -> np.ndarray:
    """Parameter vector in the oracle's order: c1, c2, kappa, Du, Dv, F, k, c3."""
    return np.array([c1, c2, kappa, Du, Dv, F, k, c3], dtype=np.float64)


def num_threads() -> int:
    return lib().or_num_threads()


def stencil_q(st: int) -> int:
    return lib().or_stencil_q(st)


def stencil_sum(st: int, f) -> np.ndarray:
    f = _f64(f)
    out = np.empty_like(f)
    nx, ny, nz = _shape3(f, STENCIL_DIMS[st])
    if lib().or_stencil_sum(st, nx, ny, nz, _p(f), _p(out)):
        raise ValueError("or_stencil_sum: bad arguments")
    return out


def laplacian(st: int, f, h: float = 1.0) -> np.ndarray:
    f = _f64(f)
    out = np.empty_like(f)
    nx, ny, nz = _shape3(f, STENCIL_DIMS[st])
    if lib().or_laplacian(st, nx, ny, nz, h, _p(f), _p(out)):
        raise ValueError("or_laplacian: bad arguments")
    return out


def chemical_potential(st: int, f, h: float = 1.0, prm=None) -> np.ndarray:
    f = _f64(f)
    prm = params() if prm is None else _f64(prm)
    out = np.empty_like(f)
    nx, ny, nz = _shape3(f, STENCIL_DIMS[st])
    if lib().or_chemical_potential(st, nx, ny, nz, h, _p(prm), _p(f), _p(out)):
        raise ValueError("or_chemical_potential: bad arguments")
    return out


def step(model: int, st: int, u, v=None, *, h: float = 1.0, dt: float, prm=None, nsteps: int = 1):
    """Return the fields after ``nsteps`` forward-Euler steps (copies; inputs untouched)."""
    u = np.array(u, dtype=np.float64, copy=True, order="C")
    vv = None if v is None else np.array(v, dtype=np.float64, copy=True, order="C")
    prm = params() if prm is None else _f64(prm)
    nx, ny, nz = _shape3(u, STENCIL_DIMS[st])
    rc = lib().or_step(model, st, nx, ny, nz, h, dt, _p(prm), _p(u),
                       None if vv is None else _p(vv), int(nsteps))
    if rc:
        raise ValueError("or_step: bad arguments or out of memory")
    return u if model not in TWO_FIELD else (u, vv)


def splitmix64_nth(seed: int, n: int) -> int:
    return int(lib().or_splitmix64_nth(seed, n))


def u01(seed: int, n: int) -> float:
    return float(lib().or_u01(seed, n))


def initial_condition(model: int, shape, *, seed: int, mean: float = 0.0, amp: float = 0.01,
                      patches: int = 0, patch: int = 0):
    """Seeded initial fields; ``shape`` is (ny, nx) or (nz, ny, nx)."""
    dims = len(shape)
    u = np.empty(shape, dtype=np.float64)
    v = np.empty(shape, dtype=np.float64) if model in TWO_FIELD else None
    nx, ny, nz = _shape3(u, dims)
    rc = lib().or_initial_condition(model, dims, nx, ny, nz, seed, mean, amp, patches, patch,
                                    _p(u), None if v is None else _p(v))
    if rc:
        raise ValueError("or_initial_condition: bad arguments")
    return u if model not in TWO_FIELD else (u, v)


def initial_condition_window(model: int, shape, origin, wshape, *, seed: int, mean: float = 0.0,
                             amp: float = 0.01, patches: int = 0, patch: int = 0):
    """Initial condition of the full grid ``shape`` evaluated on the periodic window
    with lower corner ``origin`` and size ``wshape`` (all numpy order)."""
    dims = len(shape)
    full = list(shape[::-1]) + [1] * (3 - dims)
    org = list(origin[::-1]) + [0] * (3 - dims)
    win = list(wshape[::-1]) + [1] * (3 - dims)
    u = np.empty(wshape, dtype=np.float64)
    v = np.empty(wshape, dtype=np.float64) if model in TWO_FIELD else None
    rc = lib().or_initial_condition_window(model, dims, full[0], full[1], full[2], seed, mean, amp, patches, patch,
                                           org[0], org[1], org[2], win[0], win[1], win[2], _p(u),
                                           None if v is None else _p(v))
    if rc:
        raise ValueError("or_initial_condition_window: bad arguments")
    return u if model not in TWO_FIELD else (u, v)


def kahan_sum(f) -> float:
    f = _f64(f).ravel()
    return lib().or_sum(_p(f), f.size)


def mass(f, h: float = 1.0) -> float:
    f = _f64(f)
    dims = f.ndim
    nx, ny, nz = _shape3(f, dims)
    return lib().or_mass(dims, nx, ny, nz, h, _p(f))


def free_energy(f, h: float = 1.0, c1: float = 1.0, c2: float = 1.0) -> float:
    f = _f64(f)
    dims = f.ndim
    nx, ny, nz = _shape3(f, dims)
    return lib().or_free_energy(dims, nx, ny, nz, h, c1, c2, _p(f))


def free_energy_c(phi, rho, h: float = 1.0, c1: float = 1.0, c2: float = 1.0, c3: float = 0.5) -> float:
    """Discrete Model C free energy of (phi, rho) (see or_free_energy_c)."""
    phi, rho = _f64(phi), _f64(rho)
    dims = phi.ndim
    nx, ny, nz = _shape3(phi, dims)
    return lib().or_free_energy_c(dims, nx, ny, nz, h, c1, c2, c3, _p(phi), _p(rho))


def rel_l2(a, b) -> float:
    a = _f64(a).ravel()
    b = _f64(b).ravel()
    assert a.size == b.size
    return lib().or_rel_l2(_p(a), _p(b), a.size)


def step_h(st: int, m, j, *, h: float = 1.0, dt: float, prm=None, nsteps: int = 1):
    """Model H: return (m, [j_x, j_y(, j_z)]) after ``nsteps`` steps (copies)."""
    m = np.array(m, dtype=np.float64, copy=True, order="C")
    js = [np.array(c, dtype=np.float64, copy=True, order="C") for c in j]
    prm = params() if prm is None else _f64(prm)
    dims = STENCIL_DIMS[st]
    if len(js) != dims or any(c.shape != m.shape for c in js):
        raise ValueError("step_h: j needs one array per axis, shaped like m")
    nx, ny, nz = _shape3(m, dims)
    rc = lib().or_step_h(st, nx, ny, nz, h, dt, _p(prm), _p(m), _p(js[0]), _p(js[1]),
                         _p(js[2]) if dims == 3 else None, int(nsteps))
    if rc:
        raise ValueError("or_step_h: bad arguments or out of memory")
    return m, js


def initial_condition_h(shape, *, seed: int, mean: float = 0.0, amp: float = 0.01):
    """Model H initial fields (m, [j_x, j_y(, j_z)])."""
    dims = len(shape)
    m = np.empty(shape, dtype=np.float64)
    js = [np.empty(shape, dtype=np.float64) for _ in range(dims)]
    nx, ny, nz = _shape3(m, dims)
    rc = lib().or_initial_condition_h(dims, nx, ny, nz, seed, mean, amp, _p(m), _p(js[0]), _p(js[1]),
                                      _p(js[2]) if dims == 3 else None)
    if rc:
        raise ValueError("or_initial_condition_h: bad arguments")
    return m, js


def free_energy_h(m, j, h: float = 1.0, c1: float = 1.0, c2: float = 1.0) -> float:
    m = _f64(m)
    js = [_f64(c) for c in j]
    dims = m.ndim
    nx, ny, nz = _shape3(m, dims)
    return lib().or_free_energy_h(dims, nx, ny, nz, h, c1, c2, _p(m), _p(js[0]), _p(js[1]),
                                  _p(js[2]) if dims == 3 else None)


def step_gen(model: int, order: int, u, v=None, *, h: float = 1.0, dt: float, prm=None, nsteps: int = 1):
    """Steps with the generated cross Laplacian of accuracy ``order`` (weights from
    oracle/stencil_gen.py); returns copies like ``step``."""
    from .stencil_gen import kernel_weights

    u = np.array(u, dtype=np.float64, copy=True, order="C")
    vv = None if v is None else np.array(v, dtype=np.float64, copy=True, order="C")
    prm = params() if prm is None else _f64(prm)
    dims = u.ndim
    wk = np.array(kernel_weights(order, dims), dtype=np.float64)
    nx, ny, nz = _shape3(u, dims)
    rc = lib().or_step_gen(model, dims, order // 2, _p(wk), nx, ny, nz, h, dt, _p(prm), _p(u),
                           None if vv is None else _p(vv), int(nsteps))
    if rc:
        raise ValueError("or_step_gen: bad arguments or out of memory")
    return u if model not in TWO_FIELD else (u, vv)
