"""sp_reduce_field_noalloc against sp_reduce, through the C ABI.

sp_reduce_field_noalloc serves callers that cannot allocate device memory when
they need a diagnostic (a memory pool that already owns nearly all of HBM, a
latency-critical loop where cudaMalloc/cudaFree would stall the device, fields
held by the caller's own allocator).  It reduces a caller-owned field with its
block partials in a fixed device array of the library.  Here a simulation
handle (created by the ordinary, allocating API) provides the fields; each
reduction of the no-allocation entry point must agree with sp_reduce on the
same field within the tolerance of the other reduction tests, on two calls in
a row.  This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    import __graft_entry__

    __graft_entry__._load_builder().build()
    import paper_2511_10508_gb300 as sp

    return sp


def noalloc(sp, what, sim, field=0):
    from paper_2511_10508_gb300 import _native as N

    f = N.lib().sp_reduce_field_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                  ctypes.c_void_p]
    shape = (ctypes.c_int64 * 3)(*(list(sim.shape[::-1]) + [1] * (3 - sim.dims)))
    out = ctypes.c_double(np.nan)
    rc = f(what, sim.dtype, sim.devptr(field), sim.dims, shape, sim.h, sim.prm.c1, sim.prm.c2, ctypes.byref(out),
           None)
    assert rc == N.SP_OK, rc
    return out.value


@pytest.mark.parametrize("model,shape,stencil,dtype,h", [
    (1, (70, 301), 0, 0, 1.0),            # Cahn-Hilliard 2D, FP64
    (0, (37, 45, 70), 3, 1, 0.5),         # Allen-Cahn 3D, FP32
    (2, (64, 96), 0, 2, 1.0),             # Gray-Scott 2D, BF16 storage (u and v)
    (1, (512, 512), 0, 0, 0.7),           # enough points for the full block count
])
def test_noalloc_reduction_matches_sp_reduce(sp, model, shape, stencil, dtype, h):
    dt = {0: 0.01, 1: 0.002, 2: 0.5}[model]
    kw = dict(stencil=stencil, dtype=dtype, seed=21, ic_amp=0.3 if model != 2 else 0.01,
              flags=sp.FLAG_BF16_NO_BOUND if dtype == 2 else 0)
    if model == 2:
        kw.update(gs_patches=4, gs_patch=5)
    with sp.Simulation(model, shape, h=h, dt=dt, **kw) as sim:
        sim.h = h
        whats = [sp.MASS, sp.FREE_ENERGY, sp.SUM_U, sp.SUMSQ_U, sp.MIN_U, sp.MAX_U]
        for call in range(2):  # two calls in a row, the field advancing in between
            sim.step(3)
            u = sim.read(0)
            scale = np.abs(u).sum() + 1.0
            for what in whats:
                a = sim.reduce(what)
                b = noalloc(sp, what, sim)
                tol = 1e-12 * (abs(a) + scale) if what == sp.FREE_ENERGY else 1e-13 * scale
                assert abs(a - b) <= tol, (call, what, a, b)
            if model == 2:
                v = sim.read(1)
                a = sim.reduce(sp.SUM_V)
                b = noalloc(sp, sp.SUM_U, sim, field=1)
                assert abs(a - b) <= 1e-13 * (np.abs(v).sum() + 1.0), (call, a, b)


def test_noalloc_rejects_bad_arguments(sp):
    from paper_2511_10508_gb300 import _native as N

    with sp.Simulation(sp.ALLEN_CAHN, (16, 16), dt=0.01) as sim:
        f = N.lib().sp_reduce_field_noalloc
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                      ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                      ctypes.c_void_p]
        shape = (ctypes.c_int64 * 3)(16, 16, 1)
        out = ctypes.c_double(0)
        ptr = sim.devptr(0)
        assert f(sp.SUM_V, 0, ptr, 2, shape, 1.0, 1.0, 1.0, ctypes.byref(out), None) == N.SP_EINVAL
        assert f(sp.MASS, 7, ptr, 2, shape, 1.0, 1.0, 1.0, ctypes.byref(out), None) == N.SP_EINVAL
        assert f(sp.MASS, 0, None, 2, shape, 1.0, 1.0, 1.0, ctypes.byref(out), None) == N.SP_EINVAL
        assert f(sp.MASS, 0, ptr, 2, shape, 0.0, 1.0, 1.0, ctypes.byref(out), None) == N.SP_EINVAL
        assert f(sp.MASS, 0, ptr, 2, (ctypes.c_int64 * 3)(16, 16, 2), 1.0, 1.0, 1.0, ctypes.byref(out),
                 None) == N.SP_EINVAL
        # an FP64 field must be 8-byte aligned (checked on the host, nothing is launched)
        assert f(sp.MASS, 0, ptr + 4, 2, (ctypes.c_int64 * 3)(8, 8, 1), 1.0, 1.0, 1.0, ctypes.byref(out),
                 None) == N.SP_EINVAL
        # a 3D plane beyond sp_create's limit
        assert f(sp.MASS, 0, ptr, 3, (ctypes.c_int64 * 3)(1 << 20, 1 << 20, 1 << 20), 1.0, 1.0, 1.0,
                 ctypes.byref(out), None) == N.SP_EINVAL
        assert f(sp.MASS, 0, ptr, 2, shape, 1.0, 1.0, 1.0, ctypes.byref(out), None) == N.SP_OK


def test_noalloc_rejects_a_capturing_stream(sp):
    """The result is copied to the host and the stream synchronised, which a
    stream under capture does not allow: the call must refuse before touching it,
    and the capture must still end cleanly."""
    import torch
    from paper_2511_10508_gb300 import _native as N

    with sp.Simulation(sp.ALLEN_CAHN, (32, 32), dt=0.01, seed=3) as sim:
        sim.h = 1.0
        f = N.lib().sp_reduce_field_noalloc
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                      ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                      ctypes.c_void_p]
        shape = (ctypes.c_int64 * 3)(32, 32, 1)
        out = ctypes.c_double(0)
        expect = noalloc(sp, sp.MASS, sim)  # first call in this context, outside any capture
        ptr = sim.devptr(0)
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        x = torch.zeros(4, device="cuda")
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            g.capture_begin()
            x += 1.0
            rc = f(sp.MASS, 0, ptr, 2, shape, 1.0, 1.0, 1.0, ctypes.byref(out), s.cuda_stream)
            g.capture_end()
        assert rc == N.SP_EINVAL
        g.replay()
        torch.cuda.synchronize()
        assert x.tolist() == [1.0] * 4
        assert noalloc(sp, sp.MASS, sim) == expect
