"""Semi-implicit Fourier spectral scheme on the GPU against the numpy oracle
(oracle/spectral.py).  The transforms differ (the library's own mixed-radix FFTs
vs numpy's), so results are compared with bounds: FP64 to 1e-12 of the field
scale after the stated steps, FP32 storage and arithmetic to relative L2 1e-5
against the FP64 oracle started from the same (rounded) field."""
import numpy as np
import pytest

from oracle import spectral as SO

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    import __graft_entry__

    __graft_entry__._load_builder().build()
    import paper_2511_10508_gb300 as sp

    return sp


def sim_of(sp, model, shape, dtype=0, dt=0.1, **kw):
    kw.setdefault("ic_amp", 0.4)
    return sp.Simulation(model, shape, dt=dt, dtype=dtype, scheme=sp.SCHEME_SPECTRAL, seed=31, **kw)


# sides with every radix (8, 4, 2, 3, 5, 7), odd sides (no Nyquist bin), powers of two
# (the radix-8/4/2 kernels), 2D and 3D, an odd number of rows (one row transformed alone)
CASES = [(0, (64, 96)), (1, (64, 96)), (0, (24, 20, 30)), (1, (24, 20, 30)), (1, (63, 45)), (0, (7, 9, 5)),
         (1, (64, 128)), (0, (16, 32, 64)), (1, (8, 16, 4)), (1, (1, 32)), (0, (5, 7, 1)), (1, (35, 56))]


@pytest.mark.parametrize("model,shape", CASES)
def test_spectral_fp64_matches_oracle(sp, model, shape):
    """Even and odd sides (the Nyquist bin only exists for even n), 2D and 3D."""
    dt, n, h = 0.1, 25, 0.9
    with sim_of(sp, model, shape, dt=dt, h=h, c1=0.8, c2=1.1, kappa=1.3) as s:
        u0 = s.read(0)
        s.step(n)
        got = s.read(0)
    ref = SO.step(model, u0, h=h, dt=dt, c1=0.8, c2=1.1, kappa=1.3, nsteps=n)
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("model,shape", CASES[:4])
def test_spectral_fp32_against_fp64_oracle(sp, model, shape):
    dt, n = 0.1, 20
    with sim_of(sp, model, shape, dtype=sp.F32, dt=dt) as s:
        u0 = s.read(0)
        s.step(n)
        got = s.read(0)
    ref = SO.step(model, u0, dt=dt, nsteps=n)
    e = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert e < 1e-5, e


@pytest.mark.parametrize("model,shape,dtype", [(1, (128, 4096), 0), (0, (96, 2048), 0), (1, (64, 8192), 1),
                                               (0, (40, 4096), 1), (1, (64, 64, 64), 0)])
def test_spectral_largest_sides(sp, model, shape, dtype):
    """The longest lines one CTA transforms: 4096 points in FP64 and 8192 in FP32
    (powers of two), 2048 / 4096 otherwise."""
    dt, n = 0.1, 6
    with sim_of(sp, model, shape, dtype=dtype, dt=dt) as s:
        u0 = s.read(0)
        s.step(n)
        got = s.read(0)
    ref = SO.step(model, u0, dt=dt, nsteps=n)
    if dtype == 0:
        assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    else:
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5


@pytest.mark.parametrize("shape,dtype", [((11, 16), 0), ((16, 8192), 0), ((16, 6144), 1), ((22, 4, 4), 1)])
def test_spectral_rejects_unsupported_sides(sp, shape, dtype):
    """Prime factors beyond 7, or lines longer than one CTA transforms: SP_EINVAL."""
    with pytest.raises(sp.SpError) as e:
        sim_of(sp, 1, shape, dtype=dtype)
    assert e.value.code == 1


def test_spectral_cahn_hilliard_conserves_mass_at_large_dt(sp):
    """dt = 0.5 is four times forward Euler's bound (0.125 for the 5-point stencil);
    the semi-implicit step stays bounded and conserves the mean.  (With the cubic
    term explicit the scheme is not unconditionally stable: from this start the
    oracle itself diverges at dt = 1.)"""
    with sim_of(sp, 1, (128, 128), dt=0.5, ic_amp=0.5) as s:
        m0 = s.reduce(sp.MASS)
        s.step(200)
        u = s.read(0)
        m1 = s.reduce(sp.MASS)
    assert np.isfinite(u).all() and np.abs(u).max() < 2.0
    assert abs(m1 - m0) <= 1e-11 * np.abs(u).sum()


def test_spectral_write_refreshes_the_spectrum(sp):
    """sp_write replaces phi; the next step starts from the new field."""
    rng = np.random.default_rng(2)
    new = rng.uniform(-0.3, 0.3, (40, 48))
    with sim_of(sp, 0, (40, 48), dt=0.2) as s:
        s.step(3)
        s.write(0, new)
        s.step(10)
        got = s.read(0)
    ref = SO.step(0, new, dt=0.2, nsteps=10)
    assert np.abs(got - ref).max() <= 1e-12


def test_spectral_rejected_by_the_server(sp):
    with sp.Server(1 << 30) as srv:
        with pytest.raises(sp.SpError):
            srv.submit(1, (64, 64), dt=0.1, nsteps=10, scheme=sp.SCHEME_SPECTRAL)
