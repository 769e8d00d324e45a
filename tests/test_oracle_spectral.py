"""Pins of the semi-implicit Fourier spectral oracle (oracle/spectral.py) against
facts fixed by the mathematics:
  * a single Fourier mode of the linear problem (c2 = 0) is multiplied by exactly
    1 / (1 - dt L(k)) per step, with the continuous symbols of each model;
  * a uniform field follows the closed-form update (phi - dt c2 phi^3) / (1 - dt c1);
  * Cahn-Hilliard conserves the mean (the k = 0 mode is untouched);
  * the Allen-Cahn kink tanh(x / sqrt 2), a stationary solution of the PDE, stays
    put to spectral accuracy (a stencil Laplacian would move it by O(h^2));
  * shift equivariance and the stability bound of the reading.

``SP_ORACLE_SPECTRAL`` may name another copy of the module (the mutant tests use it).
"""
import importlib.util
import math
import os

import numpy as np
import pytest


def _load():
    path = os.environ.get("SP_ORACLE_SPECTRAL")
    if not path:
        from oracle import spectral

        return spectral
    spec = importlib.util.spec_from_file_location("spectral_under_test", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


S = _load()
SHAPES = {2: (12, 16), 3: (10, 12, 14)}


def mode(shape, ks, amp=1.0):
    idx = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")[::-1]  # x, y(, z)
    ph = sum(2 * np.pi * k * i / n for k, i, n in zip(ks, idx, shape[::-1]))
    return amp * np.cos(ph)


@pytest.mark.parametrize("model", [S.AC, S.CH])
@pytest.mark.parametrize("dims", [2, 3])
def test_linear_mode_factor(model, dims):
    """c2 = 0: each step multiplies a mode by 1 / (1 - dt L(k)), L = c1 - k^2 (AC) or
    k^2 (c1 - kappa k^2) (CH), k^2 = sum (2 pi m / (n h))^2."""
    shape = SHAPES[dims]
    h, dt, n = 0.8, 0.3, 12
    c1, kappa = 0.6, 1.4
    ks = (2, 1, 3)[:dims]
    k2 = sum((2 * np.pi * k / (m * h)) ** 2 for k, m in zip(ks, shape[::-1]))
    L = (c1 - k2) if model == S.AC else k2 * (c1 - kappa * k2)
    f = mode(shape, ks, amp=0.4)
    out = S.step(model, f, h=h, dt=dt, c1=c1, c2=0.0, kappa=kappa, nsteps=n)
    np.testing.assert_allclose(out, f / (1 - dt * L) ** n, rtol=0, atol=1e-13)


def test_uniform_allen_cahn_closed_form():
    """A uniform phi0 (only the k = 0 mode) moves to (phi0 - dt c2 phi0^3) / (1 - dt c1)."""
    c1, c2, dt, phi0 = 0.7, 1.3, 0.4, 0.55
    out = S.step(S.AC, np.full(SHAPES[2], phi0), dt=dt, c1=c1, c2=c2, nsteps=1)
    np.testing.assert_allclose(out, (phi0 - dt * c2 * phi0 ** 3) / (1 - dt * c1), rtol=2e-15, atol=0)


@pytest.mark.parametrize("dims", [2, 3])
def test_cahn_hilliard_conserves_mean(dims):
    rng = np.random.default_rng(5)
    u = 0.1 + 0.5 * rng.uniform(-1, 1, SHAPES[dims])
    out = S.step(S.CH, u, dt=0.05, nsteps=100)
    assert abs(out.mean() - u.mean()) < 1e-14
    assert np.abs(out - u).max() > 1e-3  # it did evolve


def test_allen_cahn_kink_is_stationary_to_spectral_accuracy():
    """tanh(x / sqrt 2) solves phi'' + phi - phi^3 = 0.  Two well-separated kinks on
    a periodic line (interaction ~ exp(-sqrt 2 * 64)) with h = 0.25 stay put after
    40 steps of dt = 0.5 to 1e-7; the 5-point stencil would move them by ~1e-3."""
    n, h = 1024, 0.25
    x = (np.arange(n) - n // 2) * h
    L = n * h
    prof = np.tanh((x + L / 4) / np.sqrt(2)) * np.tanh((L / 4 - x) / np.sqrt(2))
    u = np.tile(prof, (4, 1))
    out = S.step(S.AC, u, h=h, dt=0.5, nsteps=40)
    assert np.abs(out - u).max() < 1e-7


@pytest.mark.parametrize("model", [S.AC, S.CH])
def test_shift_equivariance(model):
    rng = np.random.default_rng(9)
    u = rng.uniform(-0.5, 0.5, SHAPES[3])
    shift = (2, -3, 5)
    a = S.step(model, u, dt=0.05, nsteps=3)
    b = S.step(model, np.roll(u, shift, (0, 1, 2)), dt=0.05, nsteps=3)
    np.testing.assert_allclose(np.roll(a, shift, (0, 1, 2)), b, rtol=0, atol=1e-14)


def test_stability_bound():
    assert S.stable(S.AC, 0.99, 1.0, 1.0) and not S.stable(S.AC, 1.0, 1.0, 1.0)
    # Cahn-Hilliard: max_k k^2 (c1 - kappa k^2) = c1^2 / (4 kappa)
    assert S.stable(S.CH, 3.99, 1.0, 1.0) and not S.stable(S.CH, 4.0, 1.0, 1.0)
    k2 = np.linspace(0, 3, 30001)
    assert math.isclose((k2 * (1.0 - k2)).max(), 0.25, rel_tol=1e-6)
