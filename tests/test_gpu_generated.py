"""Generated cross Laplacians (SP_LAP_GENERATED) on the GPU against the oracle
(oracle.step_gen): the weights are the same FP64 numbers on both sides (the
exact rational solution rounded once), so FP64 steps agree bit for bit."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

DT = {0: 0.02, 1: 0.001, 2: 0.2, 3: 0.01}


@pytest.fixture(scope="module")
def sp():
    import __graft_entry__

    __graft_entry__._load_builder().build()
    import paper_2511_10508_gb300 as sp

    return sp


def make(sp, model, shape, order, dtype=0, **kw):
    base = dict(stencil=sp.LAP_GENERATED, stencil_order=order, dtype=dtype, seed=kw.pop("seed", 91))
    if model == 2:
        base.update(gs_patches=2, gs_patch=min(3, *shape), ic_amp=0.05)
    else:
        base.update(ic_amp=0.4)
    base.update(kw)
    if dtype == 2:  # BF16 storage has no accuracy bound and must be asked for explicitly
        base["flags"] = base.get("flags", 0) | sp.FLAG_BF16_NO_BOUND
    return sp.Simulation(model, shape, dt=DT[model], **base)


def oracle_ic(model, shape, prm):
    if model == 2:
        return O.initial_condition(O.GS, shape, seed=prm.seed, amp=prm.ic_amp, patches=prm.gs_patches,
                                   patch=prm.gs_patch)
    return O.initial_condition(model, shape, seed=prm.seed, mean=prm.ic_mean, amp=prm.ic_amp)


def oprm(p):
    return O.params(c1=p.c1, c2=p.c2, kappa=p.kappa, Du=p.Du, Dv=p.Dv, F=p.F, k=p.k, c3=p.c3)


@pytest.mark.parametrize("shape", [(37, 45), (13, 17, 19), (3, 5), (2, 3, 4)])
@pytest.mark.parametrize("order", [2, 4, 6, 8])
@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_generated_fp64_bitwise(sp, model, order, shape):
    n = 7
    with make(sp, model, shape, order) as s:
        ic = oracle_ic(model, shape, s.prm)
        s.step(n)
        got = [s.read(f) for f in range(s.nfields)]
        p = s.prm
    ref = O.step_gen(model, order, *(ic if model in (2, 3) else (ic,)), dt=DT[model], prm=oprm(p), nsteps=n)
    ref = list(ref) if model in (2, 3) else [ref]
    for g, r in zip(got, ref):
        assert np.array_equal(g, r), np.abs(g - r).max()


@pytest.mark.parametrize("model,order", [(1, 8), (3, 6), (0, 4)])
def test_generated_graph_replay(sp, model, order):
    shape = (48, 64)
    with make(sp, model, shape, order) as s:
        ic = oracle_ic(model, shape, s.prm)
        s.step(40)
        got = [s.read(f) for f in range(s.nfields)]
        p = s.prm
    ref = O.step_gen(model, order, *(ic if model in (2, 3) else (ic,)), dt=DT[model], prm=oprm(p), nsteps=40)
    ref = list(ref) if model in (2, 3) else [ref]
    assert all(np.array_equal(g, r) for g, r in zip(got, ref))


@pytest.mark.parametrize("model,order", [(1, 6), (2, 8)])
def test_generated_fp32(sp, model, order):
    shape = (40, 96)
    with make(sp, model, shape, order, dtype=1) as s:
        start = [s.read(f) for f in range(s.nfields)]
        s.step(10)
        got = [s.read(f) for f in range(s.nfields)]
        p = s.prm
    ref = O.step_gen(model, order, *start, dt=DT[model], prm=oprm(p), nsteps=10)
    ref = list(ref) if model in (2, 3) else [ref]
    for g, r in zip(got, ref):
        assert O.rel_l2(g, r) < 1e-5


@pytest.mark.parametrize("shape", [(70, 300), (45, 64), (9, 8), (33, 258)])
@pytest.mark.parametrize("order", [2, 4, 6, 8])
@pytest.mark.parametrize("model", [0, 1, 2, 3])
@pytest.mark.parametrize("dtype", [1, 2])
def test_generated_2d_tiles_equal_per_point(sp, dtype, model, order, shape):
    """2D FP32 / BF16: the shared-memory tile kernel (family 0, mu of
    Cahn-Hilliard in shared memory) and the per-point kernels (family 1, mu
    through a buffer in device memory) evaluate the same expressions, so they
    agree bit for bit.  Shapes: ragged tiles in x and y, one tile, a grid smaller
    than the halo, and rows that are not whole 16-byte chunks."""
    outs = []
    for fam in (0, 1):
        with make(sp, model, shape, order, dtype=dtype) as s:
            s.launch_config = (1, fam)
            assert s.launch_config == (1, fam)
            s.step(9)
            outs.append([s.read(f, as_f64=False) for f in range(s.nfields)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_generated_not_served(sp):
    with sp.Server(1 << 30) as srv:
        with pytest.raises(sp.SpError):
            srv.submit(1, (64, 64), dt=0.001, nsteps=10, stencil=sp.LAP_GENERATED, stencil_order=4)
