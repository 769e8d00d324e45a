"""Host-side tests of the C ABI (no GPU): the library loads, exports every
function that include/sp.h declares, rejects bad arguments before touching the
device, and its forward-Euler stability check matches the stencils' spectra."""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sp():
    import __graft_entry__

    __graft_entry__._load_builder().build()
    import paper_2511_10508_gb300 as sp

    return sp


def test_library_exports_every_declared_function(sp):
    from paper_2511_10508_gb300 import _native as N

    names = N.header_functions()
    assert len(names) >= 12
    lib = ctypes.CDLL(N.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", N.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(names) <= exported


@pytest.mark.gpu
def test_library_is_built_for_sm103a(sp):
    """The library reports the architecture of the device code the runtime loaded."""
    from paper_2511_10508_gb300 import _native as N

    v = ctypes.c_int(0)
    assert N.lib().sp_binary_version(ctypes.byref(v)) == N.SP_OK
    assert v.value == 103


def test_params_default(sp):
    p = sp.params(sp.GRAY_SCOTT, 2)
    assert (p.c1, p.c2, p.kappa) == (1.0, 1.0, 1.0)
    assert (p.Du, p.Dv, p.F, p.k) == (0.16, 0.08, 0.035, 0.065)
    assert p.stencil == sp.LAP_5 and p.dtype == sp.F64
    assert (p.gs_patches, p.gs_patch) == (64, 20)
    assert sp.params(sp.CAHN_HILLIARD, 3).stencil == sp.LAP_7


@pytest.mark.parametrize("bad", [
    dict(model=7), dict(dims=4), dict(stencil=9),
    dict(h=0.0), dict(dt=-1.0), dict(h=float("nan")), dict(dtype=5), dict(flags=4), dict(scheme=2),
    dict(dtype=2),  # BF16 storage without SP_FLAG_BF16_NO_BOUND
    dict(scheme=1, model=2), dict(scheme=1, model=3), dict(scheme=1, dtype=2),
    dict(stencil=3),  # 3D stencil on a 2D grid
])
def test_invalid_arguments_rejected_before_device(sp, bad):
    from paper_2511_10508_gb300 import _native as N

    model = bad.get("model", sp.ALLEN_CAHN)
    dims = bad.get("dims", 2)
    p = N.sp_params()
    N.lib().sp_params_default(0, 2, ctypes.byref(p))
    for k in ("stencil", "dtype", "flags", "scheme"):
        if k in bad:
            setattr(p, k, bad[k])
    shape = (ctypes.c_int64 * 3)(16, 16, 1)
    h = ctypes.c_void_p()
    rc = N.lib().sp_create(model, dims, shape, bad.get("h", 1.0), bad.get("dt", 0.01), ctypes.byref(p),
                           ctypes.byref(h))
    assert rc == N.SP_EINVAL, (rc, N.lib().sp_last_error())
    assert not h.value
    assert N.lib().sp_last_error()


def test_bad_shapes_rejected(sp):
    from paper_2511_10508_gb300 import _native as N

    p = N.sp_params()
    N.lib().sp_params_default(0, 2, ctypes.byref(p))
    h = ctypes.c_void_p()
    for shp in ((0, 5, 1), (5, -1, 1), (5, 5, 3)):
        rc = N.lib().sp_create(0, 2, (ctypes.c_int64 * 3)(*shp), 1.0, 0.01, ctypes.byref(p), ctypes.byref(h))
        assert rc == N.SP_EINVAL
    p.gs_patches = 5000
    rc = N.lib().sp_create(2, 2, (ctypes.c_int64 * 3)(64, 64, 1), 1.0, 0.5, ctypes.byref(p), ctypes.byref(h))
    assert rc == N.SP_EINVAL


def test_unstable_dt_rejected(sp):
    from paper_2511_10508_gb300 import _native as N

    p = sp.params(sp.ALLEN_CAHN, 2)
    h = ctypes.c_void_p()
    rc = N.lib().sp_create(0, 2, (ctypes.c_int64 * 3)(32, 32, 1), 1.0, 0.25, ctypes.byref(p), ctypes.byref(h))
    assert rc == N.SP_EUNSTABLE


def _oracle_lambda_max(st):
    """max over all modes of an 8^d grid (contains theta = pi) of the eigenvalue of
    -h^2 L_h, measured by applying the oracle's stencil to each cosine mode."""
    dims = O.STENCIL_DIMS[st]
    n = 8
    shape = (n,) * dims
    best = 0.0
    idx = np.meshgrid(*[np.arange(n)] * dims, indexing="ij")
    for ks in np.ndindex(*shape):
        ph = sum(2 * np.pi * k * i / n for k, i in zip(ks, idx))
        f = np.cos(ph)
        L = O.laplacian(st, f, 1.0)
        j = np.unravel_index(np.argmax(np.abs(f)), f.shape)
        best = max(best, -L[j] / f[j])
    return best


@pytest.mark.parametrize("st", [0, 1, 2, 3, 4, 5])
def test_stability_bound_matches_stencil_spectrum(sp, st):
    """With c1 = c2 = 0 the Allen-Cahn growth bound is lambda_max / h^2: the library's
    table must equal the maximum eigenvalue of the oracle's stencil."""
    dims = O.STENCIL_DIMS[st]
    p = sp.params(sp.ALLEN_CAHN, dims, stencil=st, c1=0.0, c2=0.0)
    ok, f = sp.check_stability(sp.ALLEN_CAHN, dims, 0.5, 0.01, p)
    lam_lib = f / 0.01 * 0.25
    assert lam_lib == pytest.approx(_oracle_lambda_max(st), rel=1e-12)


def test_stability_of_the_benchmark_configurations(sp):
    cases = [
        (sp.ALLEN_CAHN, 2, dict(), 0.05, 0.5),                              # 256^2 AC
        (sp.CAHN_HILLIARD, 2, dict(stencil=sp.LAP_5), 0.01, 0.8),           # 4096^2 CH 5-point
        (sp.CAHN_HILLIARD, 2, dict(stencil=sp.LAP_9CROSS4), 0.01, 0.01 * 32 / 3 * (32 / 3 + 2)),
        (sp.GRAY_SCOTT, 2, dict(), 1.0, 0.16 * 8 + 0.035),                  # 32768^2 GS
        (sp.CAHN_HILLIARD, 3, dict(stencil=sp.LAP_7), 0.005, 0.005 * 12 * 14),
        (sp.CAHN_HILLIARD, 3, dict(stencil=sp.LAP_27), 0.005, 0.005 * 92 / 15 * (92 / 15 + 2)),
        (sp.CAHN_HILLIARD, 3, dict(stencil=sp.LAP_13CROSS4), 0.005, 0.005 * 16 * 18),
    ]
    for model, dims, kw, dt, want in cases:
        ok, f = sp.check_stability(model, dims, 1.0, dt, sp.params(model, dims, **kw))
        assert ok and f == pytest.approx(want, rel=1e-12), (model, dims, kw, f, want)
    ok, f = sp.check_stability(sp.CAHN_HILLIARD, 2, 1.0, 0.03, sp.params(sp.CAHN_HILLIARD, 2))
    assert not ok and f == pytest.approx(2.4)


def test_spectral_scheme_stability_bound(sp):
    """Semi-implicit spectral scheme: the step needs 1 - dt L(k) > 0 for all k, i.e.
    dt c1 < 1 (Allen-Cahn) and dt c1^2 / (4 kappa) < 1 (Cahn-Hilliard); the stencil
    bound of forward Euler does not apply (dt = 5 is fine for Cahn-Hilliard)."""
    ok, f = sp.check_stability(sp.ALLEN_CAHN, 2, 1.0, 0.99, sp.params(sp.ALLEN_CAHN, 2, scheme=sp.SCHEME_SPECTRAL))
    assert ok and abs(f - 0.99) < 1e-15
    ok, _ = sp.check_stability(sp.ALLEN_CAHN, 2, 1.0, 1.0, sp.params(sp.ALLEN_CAHN, 2, scheme=sp.SCHEME_SPECTRAL))
    assert not ok
    ok, f = sp.check_stability(sp.CAHN_HILLIARD, 3, 1.0, 3.9, sp.params(sp.CAHN_HILLIARD, 3, scheme=sp.SCHEME_SPECTRAL))
    assert ok and abs(f - 3.9 / 4) < 1e-15
    ok, _ = sp.check_stability(sp.CAHN_HILLIARD, 3, 1.0, 4.0, sp.params(sp.CAHN_HILLIARD, 3, scheme=sp.SCHEME_SPECTRAL))
    assert not ok
    ok, _ = sp.check_stability(sp.CAHN_HILLIARD, 2, 1.0, 0.5, sp.params(sp.CAHN_HILLIARD, 2))
    assert not ok  # forward Euler with the 5-point stencil is unstable at this dt


@pytest.mark.parametrize("order", [2, 4, 6, 8])
@pytest.mark.parametrize("dims", [2, 3])
def test_generated_stencil_weights_equal_the_oracles(sp, order, dims):
    """The library solves the interpolation system in its own exact rational
    arithmetic; the weights it rounds to FP64 equal the oracle's bit for bit, so
    FP64 steps with generated stencils can be compared bit for bit."""
    from oracle import stencil_gen as G

    w, lm = sp.stencil_weights(order, dims)
    assert w == G.kernel_weights(order, dims)
    assert lm == G.lambda_max(order, dims)


def test_generated_stencil_rejections(sp):
    from paper_2511_10508_gb300 import _native as N

    w = (ctypes.c_double * 5)()
    for order, dims in [(3, 2), (0, 2), (10, 3), (4, 4)]:
        assert N.lib().sp_stencil_weights(order, dims, w, None) == N.SP_EINVAL
    for order in (1, 5, 12):
        p = sp.params(sp.CAHN_HILLIARD, 2, stencil=sp.LAP_GENERATED, stencil_order=order)
        ok = N.lib().sp_check_stability(sp.CAHN_HILLIARD, 2, 1.0, 1e-4, ctypes.byref(p), None)
        assert ok == N.SP_EINVAL
    p = sp.params(sp.MODEL_H, 2, stencil=sp.LAP_GENERATED, stencil_order=4)
    assert N.lib().sp_check_stability(sp.MODEL_H, 2, 1.0, 1e-4, ctypes.byref(p), None) == N.SP_EINVAL
    # stability uses the generated stencil's lambda_max: order 8 in 3D
    _, lm = sp.stencil_weights(8, 3)
    p = sp.params(sp.ALLEN_CAHN, 3, stencil=sp.LAP_GENERATED, stencil_order=8)
    ok, f = sp.check_stability(sp.ALLEN_CAHN, 3, 1.0, 0.01, p)
    assert ok and abs(f - 0.01 * max(1.0, abs(1.0 - lm), 2.0, abs(-2.0 - lm))) < 1e-12


def test_admission_order_by_priority(sp):
    """The server's admission rule on the host: higher priority first, arrival
    order within a priority, requests that do not fit let later ones pass, and
    the slot limit stops admission."""
    order = sp.admission_order
    # everything fits: priority, then arrival
    assert order([10, 10, 10, 10], [0, 2, 1, 2], 100, 10) == [1, 3, 2, 0]
    # the high-priority request is too large for now: smaller ones pass it
    assert order([80, 30, 30, 30], [5, 0, 1, 0], 70, 10) == [2, 1]
    # the budget is consumed in admission order
    assert order([40, 40, 40], [0, 0, 9], 90, 10) == [2, 0]
    # slots
    assert order([1, 1, 1, 1], [3, 2, 1, 0], 100, 2) == [0, 1]
    assert order([1, 1], [0, 0], 100, 0) == []
    assert order([], [], 100, 4) == []
    # negative priorities come after the default 0
    assert order([1, 1, 1], [-1, 0, -5], 100, 10) == [1, 0, 2]


def test_wait_poll_hook_needs_no_device():
    """The bounded-wait test hook only sets a process-wide value: callable
    without a GPU, every value accepted, 0 restores the default."""
    import paper_2511_10508_gb300._native as N

    for v in (5, -1, 0):
        assert N.lib().sp_set_wait_polls(v) == 0
