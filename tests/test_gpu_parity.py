"""GPU path (through the C ABI) against the FP64 oracle.

FP64: the kernels evaluate the same expressions in the same order as the
oracle, with no contraction, so fields must be equal bit for bit.
FP32 / BF16-storage: compared with the FP64 oracle started from the same
(rounded) initial field; the bounds are stated per test.
Grids are ragged (sides not multiples of the tile) and span several tiles and
several slabs along the streamed axis.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

MODELS = {0: "AC", 1: "CH", 2: "GS"}
DT = {0: 0.05, 1: 0.005, 2: 0.5, 3: 0.02}
DT3 = {0: 0.05, 1: 0.002, 2: 0.25, 3: 0.02}
TWO = (2, 3)  # two-field models: Gray-Scott, Model C


@pytest.fixture(scope="module")
def sp():
    import __graft_entry__

    __graft_entry__._load_builder().build()
    import paper_2511_10508_gb300 as sp

    return sp


def make(sp, model, shape, st, dtype=0, dt=None, **kw):
    dims = len(shape)
    dt = dt if dt is not None else (DT if dims == 2 else DT3)[model]
    base = dict(stencil=st, dtype=dtype, seed=kw.pop("seed", 12345))
    if model == 2:
        base.update(gs_patches=kw.pop("gs_patches", 6), gs_patch=kw.pop("gs_patch", 5), ic_amp=kw.pop("ic_amp", 0.01))
    else:
        base.update(ic_amp=kw.pop("ic_amp", 0.5))
    base.update(kw)
    if dtype == 2:  # BF16 storage has no accuracy bound and must be asked for explicitly
        base["flags"] = base.get("flags", 0) | sp.FLAG_BF16_NO_BOUND
    return sp.Simulation(model, shape, dt=dt, **base), dt


def oracle_ic(model, shape, prm):
    if model == 2:
        return O.initial_condition(O.GS, shape, seed=prm.seed, amp=prm.ic_amp, patches=prm.gs_patches,
                                   patch=prm.gs_patch)
    return O.initial_condition(model, shape, seed=prm.seed, mean=prm.ic_mean, amp=prm.ic_amp)


def oparams(prm):
    return O.params(c1=prm.c1, c2=prm.c2, kappa=prm.kappa, Du=prm.Du, Dv=prm.Dv, F=prm.F, k=prm.k, c3=prm.c3)


CASES_2D = [(m, s) for m in (0, 1, 2, 3) for s in (0, 1, 2)]
CASES_3D = [(m, s) for m in (0, 1, 2, 3) for s in (3, 4, 5)]


@pytest.mark.parametrize("model,st", CASES_2D + CASES_3D)
def test_fp64_bitwise(sp, model, st):
    dims = O.STENCIL_DIMS[st]
    shape = (70, 301) if dims == 2 else (37, 45, 70)
    sim, dt = make(sp, model, shape, st)
    with sim:
        ic = oracle_ic(model, shape, sim.prm)
        u0 = sim.read(0)
        if model in TWO:
            assert np.array_equal(u0, ic[0]) and np.array_equal(sim.read(1), ic[1])
        else:
            assert np.array_equal(u0, ic)
        n = 9
        sim.step(n)
        assert sim.steps_taken == n
        if model in TWO:
            ru, rv = O.step(model, st, ic[0], ic[1], dt=dt, prm=oparams(sim.prm), nsteps=n)
            gu, gv = sim.read(0), sim.read(1)
            assert np.array_equal(gu, ru), np.abs(gu - ru).max()
            assert np.array_equal(gv, rv), np.abs(gv - rv).max()
        else:
            ref = O.step(model, st, ic, dt=dt, prm=oparams(sim.prm), nsteps=n)
            g = sim.read(0)
            assert np.array_equal(g, ref), np.abs(g - ref).max()


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (2, 7), (5, 1), (33, 257), (1, 1, 1), (2, 3, 5), (3, 1, 4),
                                   (40, 33, 65)])
@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_fp64_bitwise_small_and_degenerate(sp, shape, model):
    """Sides smaller than the stencil radius (neighbours wrap several times), a
    single point, and sides one past a tile boundary."""
    dims = len(shape)
    for st in ((0, 2) if dims == 2 else (3, 4, 5)):
        kw = dict(gs_patches=1, gs_patch=1) if model == 2 else {}
        sim, dt = make(sp, model, shape, st, **kw)
        with sim:
            ic = oracle_ic(model, shape, sim.prm)
            sim.step(5)
            if model in TWO:
                ru, rv = O.step(model, st, ic[0], ic[1], dt=dt, prm=oparams(sim.prm), nsteps=5)
                assert np.array_equal(sim.read(0), ru) and np.array_equal(sim.read(1), rv)
            else:
                ref = O.step(model, st, ic, dt=dt, prm=oparams(sim.prm), nsteps=5)
                assert np.array_equal(sim.read(0), ref)


def test_fp64_long_slab_streaming(sp):
    """A tall grid is split into several slabs along the streamed axis; the slab
    seams must be invisible (bitwise) over many steps."""
    for model, st, shape in [(1, 0, (1500, 300)), (1, 2, (900, 257)), (1, 3, (200, 40, 70)), (2, 4, (150, 33, 66)),
                             (3, 0, (1200, 300)), (3, 4, (150, 33, 66))]:
        sim, dt = make(sp, model, shape, st)
        with sim:
            ic = oracle_ic(model, shape, sim.prm)
            sim.step(12)
            if model in TWO:
                ru, rv = O.step(model, st, ic[0], ic[1], dt=dt, prm=oparams(sim.prm), nsteps=12)
                assert np.array_equal(sim.read(0), ru) and np.array_equal(sim.read(1), rv)
            else:
                ref = O.step(model, st, ic, dt=dt, prm=oparams(sim.prm), nsteps=12)
                assert np.array_equal(sim.read(0), ref)


# FP32 arithmetic: per-step relative rounding ~6e-8; over these short runs the
# relative L2 error against the FP64 oracle stays below 1e-5.
# BF16 storage: every store rounds to 8 significant bits (relative 2^-9); the
# error after a few steps is of that order, bounded here by 1e-2.
TOL = {1: 1e-5, 2: 1e-2}


@pytest.mark.parametrize("dtype", [1, 2])
@pytest.mark.parametrize("model,st", [(0, 0), (1, 0), (1, 2), (2, 0), (0, 3), (1, 3), (1, 4), (2, 3), (1, 5),
                                      (3, 0), (3, 2), (3, 3), (3, 4)])
def test_reduced_precision_against_fp64_oracle(sp, dtype, model, st):
    dims = O.STENCIL_DIMS[st]
    shape = (60, 1100) if dims == 2 else (36, 40, 72)
    sim, dt = make(sp, model, shape, st, dtype=dtype)
    with sim:
        u0 = sim.read(0)  # the rounded initial field, widened exactly
        ic = oracle_ic(model, shape, sim.prm)
        first = ic[0] if model in TWO else ic
        # initial condition: the FP64 value rounded once to the storage type
        ulp = 2.0 ** -24 if dtype == 1 else 2.0 ** -8
        assert np.all(np.abs(u0 - first) <= ulp * np.abs(first) + 1e-300)
        n = 10
        if model in TWO:
            v0 = sim.read(1)
            ru, rv = O.step(model, st, u0, v0, dt=dt, prm=oparams(sim.prm), nsteps=n)
            sim.step(n)
            eu, ev = O.rel_l2(sim.read(0), ru), O.rel_l2(sim.read(1), rv)
            assert eu < TOL[dtype] and ev < TOL[dtype], (eu, ev)
        else:
            ref = O.step(model, st, u0, dt=dt, prm=oparams(sim.prm), nsteps=n)
            sim.step(n)
            e = O.rel_l2(sim.read(0), ref)
            assert e < TOL[dtype], e


@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_reductions(sp, dtype):
    for model, shape, st in [(1, (70, 301), 0), (0, (37, 45, 70), 3), (2, (64, 96), 0)]:
        sim, dt = make(sp, model, shape, st, dtype=dtype)
        with sim:
            sim.step(3)
            u = sim.read(0)
            scale = np.abs(u).sum() + 1.0
            assert abs(sim.reduce(sp.MASS) - O.mass(u)) <= 1e-13 * scale
            assert abs(sim.reduce(sp.SUM_U) - O.kahan_sum(u)) <= 1e-13 * scale
            assert abs(sim.reduce(sp.SUMSQ_U) - O.kahan_sum(u * u)) <= 1e-13 * (u * u).sum()
            assert sim.reduce(sp.MIN_U) == u.min() and sim.reduce(sp.MAX_U) == u.max()
            fe = O.free_energy(u, h=1.0, c1=sim.prm.c1, c2=sim.prm.c2)
            assert abs(sim.reduce(sp.FREE_ENERGY) - fe) <= 1e-12 * (abs(fe) + scale)
            if model == 2:
                v = sim.read(1)
                assert abs(sim.reduce(sp.SUM_V) - O.kahan_sum(v)) <= 1e-13 * (np.abs(v).sum() + 1)


@pytest.mark.parametrize("dtype", [1, 2])
def test_fixed_point_sums_adversarial(sp, dtype):
    """FP32 / BF16 mass and sums take exact fixed-point block sums: against the
    exact sum of the stored values (math.fsum, correctly rounded) the error stays
    within u|S| + 5u sum|x| (u = 2^-53) on values spanning 60 decades, with
    denormals, zeros of both signs, cancelling pairs and a ragged tail; an
    infinity propagates."""
    import math

    rng = np.random.default_rng(3)
    shape = (37, 64, 65)
    n = int(np.prod(shape))
    mag = 10.0 ** rng.uniform(-30, 30, n)
    vals = np.where(rng.random(n) < 0.5, -mag, mag)
    vals[rng.random(n) < 0.02] = 1e-40 if dtype == 1 else 1e-38   # denormal in FP32
    vals[rng.random(n) < 0.02] = 0.0
    vals[rng.random(n) < 0.01] = -0.0
    half = n // 4
    vals[half:2 * half] = -vals[:half]                              # exact cancellation
    vals = vals.reshape(shape)
    u = 2.0 ** -53
    with sp.Simulation(sp.ALLEN_CAHN, shape, dt=0.01, dtype=dtype, flags=sp.FLAG_BF16_NO_BOUND if dtype == 2 else 0, stencil=3) as sim:
        sim.write(0, vals)
        stored = sim.read(0)                                        # the values as rounded to storage
        exact = math.fsum(stored.ravel().tolist())
        bound = u * abs(exact) + 5 * u * np.abs(stored).sum()
        for what in (sp.MASS, sp.SUM_U):
            got = sim.reduce(what)
            assert abs(got - exact) <= bound, (what, got, exact, bound)
        inf_vals = stored.copy()
        inf_vals[5, 7, 9] = np.inf
        sim.write(0, inf_vals)
        assert sim.reduce(sp.MASS) == np.inf


def test_reductions_with_h(sp):
    """Cell volume h^d and the 1/h of the gradient enter mass and free energy."""
    shape = (48, 80)
    with sp.Simulation(sp.CAHN_HILLIARD, shape, h=0.7, dt=0.001, seed=4, ic_amp=0.3) as sim:
        u = sim.read(0)
        assert abs(sim.reduce(sp.MASS) - O.mass(u, h=0.7)) <= 1e-13 * np.abs(u).sum()
        fe = O.free_energy(u, h=0.7)
        assert abs(sim.reduce(sp.FREE_ENERGY) - fe) <= 1e-12 * abs(fe)


def test_write_read_roundtrip_and_resume(sp):
    """sp_write + sp_read round-trip bit for bit (FP64) and resuming from a written
    state equals continuing the run (checkpoint / resume)."""
    shape = (50, 130)
    with sp.Simulation(sp.CAHN_HILLIARD, shape, dt=0.005, seed=8, ic_amp=0.4) as a, \
            sp.Simulation(sp.CAHN_HILLIARD, shape, dt=0.005, seed=99, ic_amp=0.4) as b:
        a.step(6)
        snap = a.read(0)
        b.write(0, snap)
        assert np.array_equal(b.read(0), snap)
        a.step(7)
        b.step(7)
        assert np.array_equal(a.read(0), b.read(0))


def bf16_round(x):
    """Round FP64 values to the nearest BF16 value (ties to even), exactly: a BF16
    number is m * 2^(e-7) with an integer significand m in [128, 256)."""
    x = np.asarray(x, dtype=np.float64)
    e = np.floor(np.log2(np.abs(np.where(x == 0, 1.0, x))))
    scale = np.exp2(e - 7)
    return np.where(x == 0, 0.0, np.round(x / scale) * scale)


@pytest.mark.parametrize("dtype", [1, 2])
def test_write_rounds_to_storage(sp, dtype):
    shape = (16, 40)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(shape)
    with sp.Simulation(sp.ALLEN_CAHN, shape, dt=0.01, dtype=dtype, flags=sp.FLAG_BF16_NO_BOUND if dtype == 2 else 0) as s:
        s.write(0, x)
        y = s.read(0)
        if dtype == 1:
            assert np.array_equal(y, x.astype(np.float32).astype(np.float64))
        else:
            assert np.array_equal(y, bf16_round(x))
        raw = s.read(0, as_f64=False)
        assert raw.dtype == (np.float32 if dtype == 1 else np.uint16)


def test_periodic_shift_equivariance_gpu(sp):
    shape = (64, 96)
    rng = np.random.default_rng(1)
    x = rng.uniform(-0.5, 0.5, shape)
    with sp.Simulation(sp.CAHN_HILLIARD, shape, dt=0.005, stencil=sp.LAP_9CROSS4) as a, \
            sp.Simulation(sp.CAHN_HILLIARD, shape, dt=0.005, stencil=sp.LAP_9CROSS4) as b:
        a.write(0, x)
        b.write(0, np.roll(x, (5, -17), (0, 1)))
        a.step(10)
        b.step(10)
        assert np.array_equal(np.roll(a.read(0), (5, -17), (0, 1)), b.read(0))


def test_torch_stream_and_zero_copy_view(sp):
    torch = pytest.importorskip("torch")
    shape = (40, 300)
    s = torch.cuda.Stream()
    with sp.Simulation(sp.ALLEN_CAHN, shape, dt=0.05, seed=2, ic_amp=0.1) as sim:
        ic = O.initial_condition(O.AC, shape, seed=2, amp=0.1)
        sim.step(4, stream=s)
        s.synchronize()
        t = sim.field_tensor(0)
        ref = O.step(O.AC, O.S1, ic, dt=0.05, nsteps=4)
        assert np.array_equal(t.cpu().numpy(), ref)


def test_mass_conservation_cahn_hilliard_gpu(sp):
    with sp.Simulation(sp.CAHN_HILLIARD, (256, 256), dt=0.01, seed=1, ic_amp=0.01) as sim:
        m0 = sim.reduce(sp.MASS)
        sim.step(500)
        m1 = sim.reduce(sp.MASS)
        u = sim.read(0)
        assert abs(m1 - m0) <= 500 * 1e-15 * u.size * np.abs(u).max()


def test_reduction_of_unaligned_field_pointer(sp):
    """sp_reduce_field_noalloc takes any caller pointer: an element-aligned but not
    16-byte-aligned base must take the scalar path and give the same sum."""
    import ctypes
    from paper_2511_10508_gb300 import _native as N

    with sp.Simulation(sp.ALLEN_CAHN, (33, 65), dt=0.01, dtype=sp.F32, seed=3, ic_amp=0.4) as sim:
        u = sim.read(0)
        f = N.lib().sp_reduce_field_noalloc
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                      ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                      ctypes.c_void_p]
        out = ctypes.c_double(0)
        # skip the first element: a 4-byte-aligned base; reduce the remaining 33*65-1 values as a 1-row grid
        n = u.size - 1
        rc = f(sp.SUM_U, sp.F32, sim.devptr(0) + 4, 2, (ctypes.c_int64 * 3)(n, 1, 1), 1.0, 1.0, 1.0,
               ctypes.byref(out), None)
        assert rc == N.SP_OK
        ref = O.kahan_sum(u.ravel()[1:])
        assert abs(out.value - ref) <= 1e-13 * np.abs(u).sum()


@pytest.mark.parametrize("model,shape,dtype", [(1, (70, 301), 0), (2, (40, 33, 65), 1), (0, (64, 64), 0)])
def test_graph_replay_equals_eager(sp, model, shape, dtype):
    """sp_step issues long runs as replays of a captured multi-step graph; the
    result equals stepping one launch at a time, bit for bit."""
    st = 0 if len(shape) == 2 else 3
    a, dt = make(sp, model, shape, st, dtype=dtype)
    b, _ = make(sp, model, shape, st, dtype=dtype)
    with a, b:
        a.step(133)
        for _ in range(133):
            b.step(1)
        for f in range(2 if model in TWO else 1):
            assert np.array_equal(a.read(f), b.read(f))
        assert a.steps_taken == b.steps_taken == 133


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("model,st", [(m, s) for m in (0, 1, 2, 3) for s in (0, 1, 2)])
def test_temporal_blocking_equals_single_steps(sp, dtype, model, st):
    """K steps fused in one launch (intermediate values rounded to the storage type
    in shared memory) equal K single-step launches bit for bit; FP64 equals the
    oracle bit for bit."""
    shape = (70, 301)
    outs = []
    for spl in (1, 2, 4):
        sim, dt = make(sp, model, shape, st, dtype=dtype, steps_per_launch=spl)
        with sim:
            assert sim.launch_config[0] == spl
            sim.step(1)       # first step of a handle is a single-step launch
            sim.step(12)      # blocked launches (and single steps for the rest)
            outs.append([sim.read(f, as_f64=False) for f in range(2 if model in TWO else 1)])
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)
    if dtype == 0:
        ic = oracle_ic(model, shape, sim.prm)
        if model in TWO:
            ref = O.step(model, st, ic[0], ic[1], dt=dt, prm=oparams(sim.prm), nsteps=13)
        else:
            ref = (O.step(model, st, ic, dt=dt, prm=oparams(sim.prm), nsteps=13),)
        for a, b in zip(outs[-1], ref):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("dtype", [1, 2])
@pytest.mark.parametrize("model,st", [(m, s) for m in (0, 2, 3) for s in (3, 4, 5)])
@pytest.mark.parametrize("shape", [(37, 45, 124), (6, 5, 8), (20, 17, 244)])
def test_temporal_blocking_3d_equals_single_steps(sp, dtype, model, st, shape):
    """3D FP32 / BF16 Allen-Cahn, Gray-Scott and Model C with two steps per launch
    (plane rings, intermediate planes rounded to the storage type), and Model C's
    one-step plane rings, equal single-step launches bit for bit: two tiles in x (one ragged), ragged y tiles,
    z segments, a grid smaller than the two-step halo in every direction, and
    graph replays (45 steps)."""
    outs = []
    configs = [(1, 0), (2, 0), (2, 1)]  # family 1: taller tiles
    if model == 3:
        configs += [(1, 4), (1, 5)]  # Model C: one step in the plane rings
    for spl, fam in configs:
        sim, dt = make(sp, model, shape, st, dtype=dtype, steps_per_launch=spl)
        with sim:
            sim.launch_config = (spl, fam)
            sim.step(1)
            sim.step(44)
            assert sim.launch_config == (spl, fam)
            outs.append([sim.read(f, as_f64=False) for f in range(2 if model in TWO else 1)])
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("shape", [(256, 256), (9, 8), (45, 70)])
@pytest.mark.parametrize("model,st", [(0, 0), (1, 2), (2, 0), (3, 1)])
def test_fp64_fused_steps_small_grids(sp, model, st, shape):
    """2D FP64 with 2 and 4 steps per launch on small grids (the grid a few tiles
    wide, one ragged tile, a grid smaller than the fused halo) equals the oracle
    bit for bit, including graph replays (64 steps)."""
    ref = None
    for cfg in ((2, 0), (4, 0)):
        sim, dt = make(sp, model, shape, st)
        with sim:
            sim.launch_config = cfg
            sim.step(1)
            sim.step(64)
            got = [sim.read(f) for f in range(2 if model in TWO else 1)]
        if ref is None:
            ic = oracle_ic(model, shape, sim.prm)
            if model in TWO:
                ref = O.step(model, st, ic[0], ic[1], dt=dt, prm=oparams(sim.prm), nsteps=65)
            else:
                ref = (O.step(model, st, ic, dt=dt, prm=oparams(sim.prm), nsteps=65),)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), cfg


@pytest.mark.parametrize("model,shape,dtype,st", [(2, (520, 777), 1, 0), (1, (300, 270), 0, 0),
                                                  (1, (1100, 1030), 0, 0), (0, (40, 33, 65), 1, 3),
                                                  (1, (37, 45, 70), 0, 4), (2, (20, 64, 40), 0, 4)])
def test_autotune_keeps_results(sp, model, shape, dtype, st):
    """Autotuning times candidate launch configurations on the live grid; the steps
    it takes are ordinary steps, so the result equals an untuned run bit for bit
    (FP64: equal to the oracle, so every candidate kernel family that ran during
    tuning is checked too).  The chosen configuration is one of the candidates and
    graphs captured for it replay correctly."""
    n = 130
    a, dt = make(sp, model, shape, st, dtype=dtype)
    b, _ = make(sp, model, shape, st, dtype=dtype, flags=sp.FLAG_AUTOTUNE)
    c, _ = make(sp, model, shape, st, dtype=dtype)
    with a, b, c:
        a.step(n)
        b.step(n)  # tunes inside this call
        taken = c.autotune()
        c.step(n - taken)
        assert a.steps_taken == b.steps_taken == c.steps_taken == n
        prm = c.prm
        spl, var = c.launch_config
        assert b.launch_config == c.launch_config  # the second tuning came from the cache
        if len(shape) == 3:
            assert spl == 1 and var in ((0, 1, 2) if (dtype != 0 or st == 4) else (0, 2) if model == 1 else (0,))
        elif dtype == 0 and shape[0] * shape[1] <= 1 << 20:
            assert (spl, var) in ((1, 0), (1, 1), (2, 0), (4, 0))
        elif dtype == 0:
            assert (spl, var) in ((1, 0), (1, 1), (1, 2), (1, 4))
        else:
            assert (spl, var) in ((1, 0), (1, 1), (2, 0), (4, 0))
        for f in range(2 if model in TWO else 1):
            ra = a.read(f, as_f64=False)
            assert np.array_equal(ra, b.read(f, as_f64=False)) and np.array_equal(ra, c.read(f, as_f64=False))
    if dtype == 0:
        ic = oracle_ic(model, shape, prm)
        if model in TWO:
            ru, rv = O.step(model, st, ic[0], ic[1], dt=dt, prm=oparams(prm), nsteps=n)
            assert np.array_equal(ra, rv)
        else:
            assert np.array_equal(ra, O.step(model, st, ic, dt=dt, prm=oparams(prm), nsteps=n))


@pytest.mark.parametrize("shape", [(70, 296), (45, 64), (9, 8), (130, 488)])
@pytest.mark.parametrize("model,st", CASES_2D)
@pytest.mark.parametrize("dtype", [1, 2])
def test_2d_kernel_families_agree(sp, dtype, model, st, shape):
    """2D FP32 / BF16 single steps: the warp-strip kernel (family 0; needs nx a
    multiple of the 16-byte vector) and the shared-memory tile kernel (family 1)
    evaluate the same expressions, so they agree bit for bit.  Shapes: two strips
    plus a ragged one, a grid narrower than one strip, nx equal to one vector,
    and several strips with rows split across warps."""
    outs = []
    for variant in (0, 1):
        sim, dt = make(sp, model, shape, st, dtype=dtype)
        with sim:
            sim.launch_config = (1, variant)
            assert sim.launch_config == (1, variant)
            sim.step(13)
            outs.append([sim.read(f, as_f64=False) for f in range(2 if model in TWO else 1)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    if dtype == 1:
        ic = oracle_ic(model, shape, sim.prm)
        if model in TWO:
            ref = O.step(model, st, ic[0], ic[1], dt=dt, prm=oparams(sim.prm), nsteps=13)[0]
        else:
            ref = O.step(model, st, ic, dt=dt, prm=oparams(sim.prm), nsteps=13)
        assert O.rel_l2(outs[0][0].astype(np.float64), ref) < TOL[1]


@pytest.mark.parametrize("shape", [(70, 300), (45, 64), (9, 8), (130, 520)])
@pytest.mark.parametrize("model,st", CASES_2D)
def test_2d_fp64_families_equal_oracle(sp, model, st, shape):
    """2D FP64: the strip kernel in its three shapes (family 0: 128 threads;
    2: 64 threads; 4: half the rows per batch) and the small-tile kernel
    (family 1) each equal the oracle bit for bit.  Shapes: strips of 128 and 256
    columns with a ragged one, a grid narrower than one strip, a grid smaller
    than the stencil's ring, and rows split over many CTAs."""
    ref = None
    for variant in (0, 1, 2, 4):
        sim, dt = make(sp, model, shape, st)
        with sim:
            sim.launch_config = (1, variant)
            assert sim.launch_config == (1, variant)
            sim.step(11)
            got = sim.read(0)
        if ref is None:
            ic = oracle_ic(model, shape, sim.prm)
            if model in TWO:
                ref = O.step(model, st, ic[0], ic[1], dt=dt, prm=oparams(sim.prm), nsteps=11)[0]
            else:
                ref = O.step(model, st, ic, dt=dt, prm=oparams(sim.prm), nsteps=11)
        assert np.array_equal(got, ref), f"family {variant}"


@pytest.mark.parametrize("shape", [(37, 45, 70), (2, 3, 5), (3, 1, 4), (1, 1, 1), (40, 33, 65), (70, 20, 64)])
@pytest.mark.parametrize("model", [0, 1, 2])
def test_fp64_27point_families_equal_oracle(sp, model, shape):
    """3D FP64 27-point: the kernel that shares the x-pair sums between y
    neighbours (family 0; Cahn-Hilliard in two passes through the mu buffer),
    the accessor-based plane ring (family 1) and z-streaming with plane sums in
    registers (family 2) all equal the oracle bit for bit, through a graph
    replay (33 steps, checked after 9 and 42).  Shapes: ragged tiles, sides
    below the stencil radius, a single point, a long z axis split across
    CTAs."""
    kw = dict(gs_patches=1, gs_patch=1) if model == 2 and min(shape) < 8 else {}
    refs = {}
    for fam in (0, 1, 2):
        sim, dt = make(sp, model, shape, 4, **kw)
        with sim:
            sim.launch_config = (1, fam)
            assert sim.launch_config == (1, fam)
            ic = oracle_ic(model, shape, sim.prm)
            for n in (9, 33):
                sim.step(n)
                total = sim.steps_taken
                if total not in refs:
                    prev = refs.get(9) if total == 42 else None
                    if model in TWO:
                        start = prev if prev is not None else ic
                        refs[total] = O.step(model, 4, start[0], start[1], dt=dt, prm=oparams(sim.prm),
                                             nsteps=n)
                    else:
                        start = prev if prev is not None else ic
                        refs[total] = O.step(model, 4, start, dt=dt, prm=oparams(sim.prm), nsteps=n)
                ref = refs[total]
                if model in TWO:
                    assert np.array_equal(sim.read(0), ref[0]), f"family {fam}, {total} steps"
                    assert np.array_equal(sim.read(1), ref[1]), f"family {fam}, {total} steps"
                else:
                    assert np.array_equal(sim.read(0), ref), f"family {fam}, {total} steps"


@pytest.mark.parametrize("shape", [(37, 45, 70), (2, 3, 5), (3, 1, 4), (1, 1, 1), (40, 33, 65), (70, 20, 64)])
@pytest.mark.parametrize("st", [3, 5])
def test_fp64_cahn_hilliard_two_pass_equals_oracle(sp, st, shape):
    """3D FP64 Cahn-Hilliard, 7- and 13-point: the two passes through the mu
    buffer (family 0) and the fused kernel (family 2) equal the oracle bit for
    bit, through a graph replay (42 steps)."""
    sim0, dt = make(sp, 1, shape, st)
    with sim0:
        ic = oracle_ic(1, shape, sim0.prm)
        ref9 = O.step(1, st, ic, dt=dt, prm=oparams(sim0.prm), nsteps=9)
        ref42 = O.step(1, st, ref9, dt=dt, prm=oparams(sim0.prm), nsteps=33)
    for fam in (0, 2):
        sim, _ = make(sp, 1, shape, st)
        with sim:
            sim.launch_config = (1, fam)
            assert sim.launch_config == (1, fam)
            sim.step(9)
            assert np.array_equal(sim.read(0), ref9), f"family {fam}"
            sim.step(33)
            assert np.array_equal(sim.read(0), ref42), f"family {fam}"


def test_fp64_27point_family_2_models(sp):
    """3D FP64 has a third kernel family only for Allen-Cahn, Cahn-Hilliard and
    Gray-Scott with the 27-point stencil and for Cahn-Hilliard with the 7- and
    13-point stencils (not Model C, not Allen-Cahn or Gray-Scott with those)."""
    for model, st, dtype in ((3, 4, 0), (0, 3, 0), (2, 5, 0), (3, 3, 0)):
        sim, _ = make(sp, model, (8, 8, 8), st, dtype=dtype)
        with sim:
            with pytest.raises(sp.SpError):
                sim.launch_config = (1, 2)


def test_set_launch_config_rejects_unavailable(sp):
    sim, _ = make(sp, 1, (64, 64), 0, dtype=0)
    with sim:
        for bad in ((8, 0), (2, 1), (1, 7), (1, 5)):
            with pytest.raises(sp.SpError):
                sim.launch_config = bad
        for cfg in ((1, 1), (1, 2), (1, 4), (2, 0), (4, 0), (1, 0)):
            sim.launch_config = cfg
            assert sim.launch_config == cfg
    sim, _ = make(sp, 1, (64, 64), 0, dtype=1)
    with sim:
        with pytest.raises(sp.SpError):
            sim.launch_config = (1, 4)  # strip shapes are FP64 only
    sim, _ = make(sp, 1, (20, 24, 28), 3, dtype=0)
    with sim:
        with pytest.raises(sp.SpError):
            sim.launch_config = (1, 1)  # 3D FP64 7-point: families 0 and 2 only


@pytest.mark.parametrize("shape", [(40, 33, 64), (20, 18, 136), (5, 7, 8), (70, 40, 256)])
@pytest.mark.parametrize("model,st", CASES_3D)
@pytest.mark.parametrize("dtype", [1, 2])
def test_3d_kernel_families_agree(sp, dtype, model, st, shape):
    """3D FP32 / BF16: the warp-row kernel (family 0), the cp.async plane-ring
    kernel (family 1; both need nx a multiple of the chunk), the
    register-staged ring kernel (family 2) agree bit for bit.  Shapes: ragged tiles in y and z, several x tiles with a ragged one, a
    grid smaller than one tile in every axis (neighbours wrap), and a long z
    axis split across CTAs."""
    outs = []
    for variant in (0, 1, 2):
        sim, dt = make(sp, model, shape, st, dtype=dtype)
        with sim:
            sim.launch_config = (1, variant)
            sim.step(7)
            outs.append([sim.read(f, as_f64=False) for f in range(2 if model in TWO else 1)])
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert np.array_equal(a, b)
    if dtype == 1:
        ic = oracle_ic(model, shape, sim.prm)
        if model in TWO:
            ref = O.step(model, st, ic[0], ic[1], dt=dt, prm=oparams(sim.prm), nsteps=7)[0]
        else:
            ref = O.step(model, st, ic, dt=dt, prm=oparams(sim.prm), nsteps=7)
        assert O.rel_l2(outs[0][0].astype(np.float64), ref) < TOL[1]


TMA_SHAPES = {1: [(40, 33, 64), (5, 7, 8), (70, 40, 256), (9, 17, 68), (3, 2, 4), (6, 40, 192)],
              2: [(40, 33, 64), (5, 7, 8), (70, 40, 256), (9, 17, 136), (6, 40, 256)]}


@pytest.mark.parametrize("case", range(6))
@pytest.mark.parametrize("model,st", [(m, s) for m in (0, 1, 2) for s in (3, 4, 5)])
@pytest.mark.parametrize("dtype", [1, 2])
def test_3d_tma_family_equals_cp_async_family(sp, dtype, model, st, case):
    """3D FP32 / BF16: the plane ring with tensor-map (TMA) plane loads (family 6)
    equals the cp.async plane ring (family 1) bit for bit, through a graph replay
    (40 steps).  Shapes: ragged tiles in x, y and z, a grid smaller than one tile
    in every axis (the box's out-of-grid chunks are all wrapped copies, several
    periods for nx = 4), several x tiles, and long z axes split across CTAs."""
    shapes = TMA_SHAPES[dtype]
    if case >= len(shapes):
        pytest.skip("fewer BF16 shapes (nx a multiple of 8)")
    shape = shapes[case]
    kw = dict(gs_patches=1, gs_patch=1) if model == 2 and min(shape) < 8 else {}
    outs = []
    for variant in (1, 6):
        sim, dt = make(sp, model, shape, st, dtype=dtype, **kw)
        with sim:
            sim.launch_config = (1, variant)
            assert sim.launch_config == (1, variant)
            sim.step(40)
            outs.append([sim.read(f, as_f64=False) for f in range(2 if model in TWO else 1)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_3d_tma_family_availability(sp):
    """Family 6 needs 3D FP32 / BF16, nx a multiple of 16 bytes of cells, and not
    Model C."""
    for model, shape, st, dtype in ((3, (8, 8, 8), 3, 1), (1, (8, 8, 10), 3, 1), (1, (8, 8, 12), 3, 2),
                                    (1, (8, 8, 8), 3, 0), (1, (64, 64), 0, 1)):
        sim, _ = make(sp, model, shape, st, dtype=dtype)
        with sim:
            with pytest.raises(sp.SpError):
                sim.launch_config = (1, 6)


def test_3d_tma_wait_timeout_reports_and_recovers(sp):
    """A bounded mbarrier wait that gives up (forced with the test hook: no polls)
    ends the kernel with the copies in flight drained and sets the simulation's
    flag: the next read raises SP_ETIMEOUT once, the context stays usable, and a
    later run with the default bound equals the cp.async family bit for bit."""
    shape = (20, 33, 64)
    sim, _ = make(sp, 1, shape, 3, dtype=1)
    with sim:
        sim.launch_config = (1, 6)
        try:
            sp.set_wait_polls(-1)
            sim.step(2)
        finally:
            sp.set_wait_polls(0)
        with pytest.raises(sp.SpError) as ei:
            sim.read(0)
        assert ei.value.code == 6  # SP_ETIMEOUT
        sim.read(0)  # the flag was cleared
    outs = []
    for variant in (6, 1):
        sim, _ = make(sp, 1, shape, 3, dtype=1)
        with sim:
            sim.launch_config = (1, variant)
            sim.step(5)
            outs.append(sim.read(0, as_f64=False))
    assert np.array_equal(outs[0], outs[1])


def test_two_host_threads_step_independent_grids(sp):
    """Two simulations stepped (and autotuned) concurrently from two host threads
    give the same fields as when run one after the other: the launch
    configuration is per simulation and the autotune cache is shared safely."""
    import threading

    cases = [(1, (300, 296), 1, 0), (2, (40, 33, 64), 1, 3)]

    def run(model, shape, dtype, st, out, idx, tune):
        sim, _ = make(sp, model, shape, st, dtype=dtype)
        with sim:
            if tune:
                sim.autotune()
                sim.step(120 - sim.steps_taken)
            else:
                sim.step(120)
            out[idx] = [sim.read(f, as_f64=False) for f in range(2 if model in TWO else 1)]

    seq = [None, None]
    for i, c in enumerate(cases):
        run(*c, seq, i, False)
    par = [None, None]
    ts = [threading.Thread(target=run, args=(*c, par, i, True)) for i, c in enumerate(cases)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=300)
    for a, b in zip(seq, par):
        assert b is not None
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("st,shape", [(0, (70, 301)), (1, (45, 64)), (2, (40, 33)), (3, (20, 18, 36)),
                                      (4, (17, 24, 33)), (5, (20, 18, 36))])
@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_unfused_ablation_equals_fused(sp, dtype, st, shape):
    """Kernel family 3 (Cahn-Hilliard only) is the unfused two-pass ablation: mu
    through a device-memory temporary, then the outer Laplacian.  Same expressions
    in the same order, so it equals the fused kernels bit for bit (40 steps, so
    graph replay is included)."""
    outs = []
    for fam in (None, 3):
        sim, dt = make(sp, 1, shape, st, dtype=dtype)
        with sim:
            if fam is not None:
                sim.launch_config = (1, fam)
                assert sim.launch_config == (1, 3)
            sim.step(40)
            outs.append(sim.read(0, as_f64=False))
    assert np.array_equal(outs[0], outs[1])
    if dtype == 0:
        ic = oracle_ic(1, shape, sim.prm)
        assert np.array_equal(outs[1], O.step(1, st, ic, dt=dt, prm=oparams(sim.prm), nsteps=40))


def test_unfused_ablation_only_for_cahn_hilliard(sp):
    for model in (0, 2):
        sim, _ = make(sp, model, (32, 32), 0)
        with sim:
            with pytest.raises(sp.SpError):
                sim.launch_config = (1, 3)



@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("shape,st", [((64, 96), 0), ((20, 24, 28), 3), ((17, 20, 23), 4)])
def test_model_c_reductions(sp, dtype, shape, st):
    """Model C: SP_MASS is the conserved density's (field 1), conserved over the
    run; SP_FREE_ENERGY adds rho^2/2 - c3 phi^2 rho and matches the oracle's."""
    sim, dt = make(sp, 3, shape, st, dtype=dtype)
    with sim:
        m0 = sim.reduce(sp.MASS)
        sim.step(40)
        u, v = sim.read(0), sim.read(1)
        scale = np.abs(v).sum() + 1.0
        assert abs(sim.reduce(sp.MASS) - O.mass(v)) <= 1e-13 * scale
        assert abs(sim.reduce(sp.MASS) - m0) <= (1e-12 if dtype == 0 else 1e-4) * scale
        assert abs(sim.reduce(sp.SUM_V) - O.kahan_sum(v)) <= 1e-13 * scale
        fe = O.free_energy_c(u, v, c1=sim.prm.c1, c2=sim.prm.c2, c3=sim.prm.c3)
        assert abs(sim.reduce(sp.FREE_ENERGY) - fe) <= 1e-12 * (abs(fe) + np.abs(u).sum() + scale)


def test_model_c_free_energy_decreases_on_gpu(sp):
    """The GPU path of Model C is a gradient flow of the listing's free energy too."""
    sim, _ = make(sp, 3, (96, 128), 0, dt=0.005, ic_amp=0.8, ic_mean=0.2)
    with sim:
        F = [sim.reduce(sp.FREE_ENERGY)]
        for _ in range(30):
            sim.step(2)
            F.append(sim.reduce(sp.FREE_ENERGY))
    assert all(b < a for a, b in zip(F, F[1:])), F


def test_fp64_probe_rate(sp):
    """The FP64 throughput probe returns a plausible sustained rate (Gop/s, one op per
    FMA): below the nominal 2 FP64 ops per clock per SM at the maximum clock and far
    above a serial rate."""
    g = sp.probe_fp64_rate()
    assert 100.0 < g <= 152 * 2 * 2.07 * 1.02
