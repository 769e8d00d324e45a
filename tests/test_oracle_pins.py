"""Pins of the FP64 oracle against facts fixed by the mathematics, not by itself.

Each test states what it checks and which mistake in the oracle it would catch:
  * stencil weights   -- exactness on polynomials (Taylor moments) and the O(h^2)
                          isotropy condition (paper, Sec. "Compile-Time Stencil
                          Generation": stencils from polynomial interpolation);
  * Fourier symbols    -- L_h cos(theta.x) = -lambda(theta)/h^2 cos(theta.x) with the
                          closed-form lambda of each stencil;
  * diffusion decay    -- a single Fourier mode decays exactly as (1 - dt D lambda/h^2)^n;
  * linear Cahn-Hilliard mode growth (Eq. model-b with c2 = 0);
  * Allen-Cahn and Cahn-Hilliard relax to tanh(x/sqrt(2)) with the stencil's order;
  * Gray-Scott uniform steady states (u v = F + k, F (1 - u) = (F + k) v);
  * fixed points, mass conservation, shift equivariance;
  * the free energy against a closed form and a summation-by-parts identity;
  * the SplitMix64 generator against published outputs; the noise statistics;
  * Model C (Sec. "Model C", signs from the paper's free-energy listing): exact
    reduction to Allen-Cahn and diffusion when uncoupled, the uniform-state
    update, linear response of both fields to single Fourier modes, density
    conservation, free-energy decrease and its closed form.
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# ----------------------------------------------------------------- helpers


def grid_coords(shape, h):
    """Coordinates x, y (, z) as arrays in numpy order (.., y, x), centred."""
    axes = [(np.arange(n) - n // 2) * h for n in shape]
    mesh = np.meshgrid(*axes, indexing="ij")
    return mesh[::-1]  # x, y(, z)


def symbol(st, thetas):
    """Closed-form lambda(theta) (eigenvalue of -h^2 L_h) of each stencil."""
    c = [math.cos(t) for t in thetas]
    if st == O.S1 or st == O.S4:
        return sum(4 * math.sin(t / 2) ** 2 for t in thetas)
    if st == O.S2:
        cx, cy = c
        return (20 - 8 * cx - 8 * cy - 4 * cx * cy) / 6
    if st == O.S3 or st == O.S6:
        return sum(2.5 - (8 / 3) * math.cos(t) + (1 / 6) * math.cos(2 * t) for t in thetas)
    if st == O.S5:
        cx, cy, cz = c
        return -(-64 / 15 + (14 / 15) * (cx + cy + cz) + (2 / 5) * (cx * cy + cx * cz + cy * cz)
                 + (4 / 15) * cx * cy * cz)
    raise ValueError(st)


def mode_field(shape, ks, amp=1.0):
    """amp * cos(sum_a 2 pi k_a i_a / n_a), numpy order shape, ks in (kx, ky[, kz])."""
    idx = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")[::-1]
    ph = sum(2 * np.pi * k * i / n for k, i, n in zip(ks, idx, shape[::-1]))
    thetas = [2 * np.pi * k / n for k, n in zip(ks, shape[::-1])]
    return amp * np.cos(ph), thetas


SHAPES = {2: (12, 16), 3: (10, 12, 14)}  # numpy order; nx != ny != nz to catch transposes
ALL = [O.S1, O.S2, O.S3, O.S4, O.S5, O.S6]

# ------------------------------------------------------ stencil weights


def monomials(dims, deg):
    out = []
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            if dims == 2:
                out.append((a, b, 0))
            else:
                for c in range(deg + 1 - a - b):
                    out.append((a, b, c))
    return out


@pytest.mark.parametrize("st", ALL)
def test_stencil_exact_on_polynomials(orc, st):
    """L_h reproduces the exact Laplacian of every monomial up to degree order+1.

    A second-order stencil is exact up to cubic polynomials, a fourth-order one up
    to quintics; a wrong weight or offset fails at some monomial."""
    dims = O.STENCIL_DIMS[st]
    r = O.STENCIL_RADIUS[st]
    order = 4 if st in (O.S3, O.S6) else 2
    h = 0.5
    shape = (9, 10) if dims == 2 else (7, 8, 9)
    X = grid_coords(shape, h)
    inner = tuple(slice(r, n - r) for n in shape)
    for (a, b, c) in monomials(dims, order + 1):
        x, y = X[0], X[1]
        z = X[2] if dims == 3 else np.ones_like(x)
        f = x ** a * y ** b * z ** c
        lap = np.zeros_like(f)
        if a >= 2:
            lap += a * (a - 1) * x ** (a - 2) * y ** b * z ** c
        if b >= 2:
            lap += b * (b - 1) * x ** a * y ** (b - 2) * z ** c
        if c >= 2 and dims == 3:
            lap += c * (c - 1) * x ** a * y ** b * z ** (c - 2)
        got = orc.laplacian(st, f, h)
        scale = max(1.0, np.abs(f).max() / h ** 2)
        np.testing.assert_allclose(got[inner], lap[inner], rtol=0, atol=1e-12 * scale,
                                   err_msg=f"monomial {(a, b, c)}")


@pytest.mark.parametrize("st", [O.S1, O.S2, O.S4, O.S5])
def test_second_order_leading_error(orc, st):
    """The O(h^2) error term on x^4 is 2h^2 for every consistent 2nd-order stencil
    (Taylor: h^2/12 d^4/dx^4); the isotropic S2/S5 also have error (2/3)h^2 on x^2 y^2,
    i.e. error (h^2/12) lap^2 f, while the cross S1/S4 have none there."""
    dims = O.STENCIL_DIMS[st]
    h = 0.25
    shape = (5, 5) if dims == 2 else (5, 5, 5)
    X = grid_coords(shape, h)
    ctr = tuple(n // 2 for n in shape)
    x, y = X[0], X[1]
    e_x4 = orc.laplacian(st, x ** 4, h)[ctr] - 0.0
    e_x2y2 = orc.laplacian(st, x ** 2 * y ** 2, h)[ctr] - 0.0
    assert e_x4 == pytest.approx(2 * h * h, rel=1e-12)
    if st in (O.S2, O.S5):
        assert e_x2y2 == pytest.approx(2 * h * h / 3, rel=1e-12)
    else:
        assert abs(e_x2y2) < 1e-14


@pytest.mark.parametrize("st", ALL)
def test_stencil_fourier_symbol(orc, st):
    """L_h cos(theta.x) = -lambda(theta)/h^2 cos(theta.x) for the closed-form symbols."""
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    h = 0.7
    modes = [(1, 0, 0), (0, 1, 0), (2, 3, 1), (5, 1, 2), (6, 6, 5)]
    for ks in modes:
        ks = ks[:dims]
        f, th = mode_field(shape, ks)
        lam = symbol(st, th)
        got = orc.laplacian(st, f, h)
        np.testing.assert_allclose(got, -lam / h ** 2 * f, rtol=0, atol=2e-13 * (1 + lam / h ** 2))


# --------------------------------------------------- linear dynamics pins


@pytest.mark.parametrize("st", ALL)
def test_diffusion_mode_decay(orc, st):
    """Allen-Cahn with c1 = c2 = 0 is pure diffusion: one Fourier mode's amplitude is
    exactly (1 - dt lambda / h^2)^n after n steps."""
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    h, dt, n = 1.0, 0.05, 40
    ks = (3, 2, 1)[:dims]
    f, th = mode_field(shape, ks, amp=0.3)
    lam = symbol(st, th)
    out = orc.step(O.AC, st, f, h=h, dt=dt, prm=O.params(c1=0.0, c2=0.0), nsteps=n)
    expect = (1 - dt * lam / h ** 2) ** n * f
    np.testing.assert_allclose(out, expect, rtol=0, atol=1e-13)


@pytest.mark.parametrize("st", [O.S1, O.S3, O.S5])
def test_gray_scott_diffusion_of_each_field(orc, st):
    """With F = k = 0: v = 0 leaves u to diffuse with Du, u = 0 leaves v to diffuse
    with Dv; each mode decays as (1 - dt D lambda / h^2)^n (catches Du/Dv swaps)."""
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    h, dt, n = 1.0, 0.5, 30
    prm = O.params(Du=0.16, Dv=0.08, F=0.0, k=0.0)
    f, th = mode_field(shape, (1, 2, 1)[:dims], amp=0.25)
    lam = symbol(st, th)
    z = np.zeros(shape)
    u, v = orc.step(O.GS, st, f, z, h=h, dt=dt, prm=prm, nsteps=n)
    np.testing.assert_allclose(u, (1 - dt * 0.16 * lam) ** n * f, atol=1e-13, rtol=0)
    assert np.all(v == 0)
    u, v = orc.step(O.GS, st, z, f, h=h, dt=dt, prm=prm, nsteps=n)
    np.testing.assert_allclose(v, (1 - dt * 0.08 * lam) ** n * f, atol=1e-13, rtol=0)
    assert np.all(u == 0)


@pytest.mark.parametrize("st", ALL)
def test_linear_cahn_hilliard_mode(orc, st):
    """Eq. (model-b) with c2 = 0 is linear: a mode evolves by the exact factor
    (1 + dt (lambda/h^2) (c1 - kappa lambda/h^2))^n (catches sign/kappa/c1 errors and
    an outer Laplacian taken of phi instead of mu)."""
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    h, dt, n = 1.2, 0.01, 50
    c1, kappa = 0.7, 1.3
    ks = (2, 1, 1)[:dims]
    f, th = mode_field(shape, ks, amp=0.2)
    lam = symbol(st, th) / h ** 2
    out = orc.step(O.CH, st, f, h=h, dt=dt, prm=O.params(c1=c1, c2=0.0, kappa=kappa), nsteps=n)
    g = (1 + dt * lam * (c1 - kappa * lam)) ** n
    np.testing.assert_allclose(out, g * f, rtol=0, atol=1e-13)


# ---------------------------------------------------- nonlinear pins


def two_kink_profile(x, L):
    """tanh(x/sqrt2) tanh((L/2-x)/sqrt2) tanh((L-x)/sqrt2): kinks at 0 and L/2 of the
    periodic domain [0, L); the far factors differ from 1 by ~e^{-sqrt2 L/2}."""
    r = math.sqrt(2.0)
    return np.tanh(x / r) * np.tanh((L / 2 - x) / r) * np.tanh((L - x) / r)


@pytest.mark.parametrize("st", [O.S1, O.S3])
def test_allen_cahn_relaxes_to_tanh_interface(orc, st):
    """Eq. (model-a) with c1 = c2 = 1 has the steady interface tanh(x / sqrt 2)
    (it solves phi'' = phi^3 - phi).  A +-1 step with two interfaces (odd about
    each, which pins their positions) relaxes to it; the steady-state error falls
    by ~4 (S1, 2nd order) or ~16 (S3, 4th order) per halving of h."""
    L = 32.0
    errs = []
    for nx in (64, 128, 256):
        h = L / nx
        x = np.arange(nx) * h
        phi0 = np.where(np.arange(nx) < nx // 2, 1.0, -1.0)
        phi0[0] = 0.0
        phi0[nx // 2] = 0.0
        lam_max = {O.S1: 4.0, O.S3: 16.0 / 3.0}[st] / h ** 2
        dt = 0.4 / (lam_max + 2.0)
        n = int(40.0 / dt)
        out = orc.step(O.AC, st, phi0[None, :], h=h, dt=dt, nsteps=n)
        errs.append(np.abs(out[0] - two_kink_profile(x, L)).max())
    want = 4.0 if st == O.S1 else 16.0
    for i in range(2):
        r = errs[i] / errs[i + 1]
        assert want * 0.75 < r < want * 1.3, (errs,)


@pytest.mark.parametrize("st", ALL)
def test_cahn_hilliard_mu_vanishes_on_tanh_interface(orc, st):
    """The chemical potential of Eq. (model-b), mu = c2 phi^3 - c1 phi - kappa lap phi,
    vanishes on phi = tanh(x / sqrt 2) when c1 = c2 = kappa = 1; the discrete mu
    falls as h^2 (2nd-order stencils) or h^4 (4th order).  A wrong sign or a dropped
    term leaves mu = O(1)."""
    L = 32.0
    dims = O.STENCIL_DIMS[st]
    errs = []
    for nx in (64, 128, 256):
        h = L / nx
        x = np.arange(nx) * h
        prof = two_kink_profile(x, L)
        f = np.broadcast_to(prof, (3, nx) if dims == 2 else (2, 3, nx)).copy()
        mu = orc.chemical_potential(st, f, h=h, prm=O.params(c1=1.0, c2=1.0, kappa=1.0))
        errs.append(np.abs(mu).max())
    want = 16.0 if st in (O.S3, O.S6) else 4.0
    assert errs[0] < 0.05
    for i in range(2):
        r = errs[i] / errs[i + 1]
        assert want * 0.8 < r < want * 1.25, (errs,)


@pytest.mark.parametrize("st", [O.S1, O.S3])
def test_cahn_hilliard_tanh_nearly_stationary(orc, st):
    """Stepping Eq. (model-b) from the tanh profile moves it by no more than the
    discretisation error of mu allows (here: < 1e-2 at h = 0.25 after t = 1)."""
    L, nx = 32.0, 128
    h = L / nx
    prof = two_kink_profile(np.arange(nx) * h, L)[None, :]
    lam_max = {O.S1: 4.0, O.S3: 16.0 / 3.0}[st] / h ** 2
    dt = 0.4 / (lam_max * (lam_max + 2.0))
    out = orc.step(O.CH, st, prof, h=h, dt=dt, nsteps=int(1.0 / dt))
    assert np.abs(out - prof).max() < 1e-2
    assert abs(out.sum() - prof.sum()) < 1e-11


def test_allen_cahn_uniform_fixed_points(orc):
    """phi = +-sqrt(c1/c2) and phi = 0 are exact fixed points of Eq. (model-a)."""
    for st in ALL:
        dims = O.STENCIL_DIMS[st]
        for val in (2.0, -2.0, 0.0):
            f = np.full(SHAPES[dims], val)
            out = orc.step(O.AC, st, f, dt=0.05, prm=O.params(c1=2.0, c2=0.5), nsteps=3)
            assert np.array_equal(out, f)


@pytest.mark.parametrize("st", [O.S1, O.S4, O.S5])
def test_gray_scott_uniform_steady_states(orc, st):
    """(u, v) = (1, 0) is an exact fixed point; with F = 0.05, k = 0.04 the uniform
    states with u v = F + k and F (1 - u) = (F + k) v (two roots) are fixed to rounding.
    A sign error in u v^2 or a swap of F and k moves them."""
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    prm = O.params(Du=0.16, Dv=0.08, F=0.05, k=0.04)
    one, zero = np.ones(shape), np.zeros(shape)
    u, v = orc.step(O.GS, st, one, zero, dt=1.0, prm=prm, nsteps=5)
    assert np.array_equal(u, one) and np.array_equal(v, zero)
    F, k = 0.05, 0.04
    disc = math.sqrt(1 - 4 * (F + k) ** 2 / F)
    for sgn in (1, -1):
        vs = F * (1 + sgn * disc) / (2 * (F + k))
        us = 1 - (F + k) * vs / F
        u, v = orc.step(O.GS, st, np.full(shape, us), np.full(shape, vs), dt=1.0, prm=prm, nsteps=1)
        assert np.abs(u - us).max() < 1e-15 and np.abs(v - vs).max() < 1e-15


@pytest.mark.parametrize("st", ALL)
def test_cahn_hilliard_mass_conservation(orc, st):
    """Eq. (model-b) is a divergence: the sum of phi is conserved to rounding."""
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    f = orc.initial_condition(O.CH, shape, seed=11, mean=0.05, amp=0.5)
    out = orc.step(O.CH, st, f, dt=0.002, nsteps=200)
    drift = abs(out.sum() - f.sum()) / (f.size * np.abs(f).max())
    assert drift < 200 * 1e-15


@pytest.mark.parametrize("model,st", [(m, s) for m in (O.AC, O.CH, O.GS, O.MC) for s in ALL])
def test_periodic_shift_equivariance(orc, model, st):
    """Stepping a rolled field equals rolling the stepped field, bit for bit
    (periodic wrap and translation invariance of every term)."""
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    shift = (3, -5, 2)[:dims]
    axes = tuple(range(dims))
    dt = {O.AC: 0.05, O.CH: 0.002, O.GS: 0.5, O.MC: 0.02}[model]
    if model in (O.GS, O.MC):
        kw = dict(patches=2, patch=3) if model == O.GS else {}
        u, v = orc.initial_condition(model, shape, seed=5, amp=0.1, **kw)
        a = orc.step(model, st, u, v, dt=dt, nsteps=3)
        b = orc.step(model, st, np.roll(u, shift, axes), np.roll(v, shift, axes), dt=dt, nsteps=3)
        assert np.array_equal(np.roll(a[0], shift, axes), b[0])
        assert np.array_equal(np.roll(a[1], shift, axes), b[1])
    else:
        f = orc.initial_condition(model, shape, seed=7, amp=0.5)
        a = orc.step(model, st, f, dt=dt, nsteps=3)
        b = orc.step(model, st, np.roll(f, shift, axes), dt=dt, nsteps=3)
        assert np.array_equal(np.roll(a, shift, axes), b)


# --------------------------------------------------------- reductions


def test_compensated_sum_matches_exact(orc):
    """Neumaier summation is within one rounding of the exactly rounded sum (fsum)."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal(100_000) * 10.0 ** rng.integers(-8, 9, 100_000)
    x = np.concatenate([x, [1e16, 1.0, -1e16, 3.0]])
    s = orc.kahan_sum(x)
    exact = math.fsum(x)
    assert abs(s - exact) <= 2 * np.spacing(abs(exact)) + 4 * x.size * 2.0 ** -106 * np.abs(x).sum()


def test_rel_l2_closed_forms(orc):
    """Relative L2 distance ||a - b||_2 / ||b||_2 on cases worked by hand: the
    denominator is the norm of the second argument, both norms are square roots
    of sums of squares, and an all-zero reference gives the absolute norm."""
    # ||(3, -1)|| / ||(0, 5)|| = sqrt(10) / 5
    assert orc.rel_l2([3.0, 4.0], [0.0, 5.0]) == pytest.approx(math.sqrt(10.0) / 5.0, rel=1e-15)
    # the reference decides the scale: ||(1, 0)|| / ||(1, 0)|| = 1 against ||(1, 0)|| / ||(2, 0)|| = 1/2
    assert orc.rel_l2([2.0, 0.0], [1.0, 0.0]) == 1.0
    assert orc.rel_l2([1.0, 0.0], [2.0, 0.0]) == 0.5
    # 3-4-5 triangles: ||(3, 4)|| = 5 over ||(0, 0, 5, 12)|| = 13
    assert orc.rel_l2([3.0, 4.0, 5.0, 12.0], [0.0, 0.0, 5.0, 12.0]) == pytest.approx(5.0 / 13.0, rel=1e-15)
    # all-zero reference: the absolute norm ||a||
    assert orc.rel_l2([3.0, -4.0], [0.0, 0.0]) == 5.0
    assert orc.rel_l2([0.0, 0.0], [0.0, 0.0]) == 0.0
    # identical arrays are at distance 0; a scaled copy (1 + e) b is at |e| for any b
    rng = np.random.default_rng(11)
    b = rng.standard_normal(1001)
    assert orc.rel_l2(b, b) == 0.0
    for e in (0.5, -0.25, 2.0 ** -20):
        assert orc.rel_l2((1.0 + e) * b, b) == pytest.approx(abs(e), rel=1e-12)
    # a single perturbed entry of a constant field: sqrt(d^2 / (n c^2))
    n, c, d = 400, 0.5, 0.03
    a = np.full(n, c)
    a[17] += d
    assert orc.rel_l2(a, np.full(n, c)) == pytest.approx(math.sqrt(d * d / (n * c * c)), rel=1e-13)


def test_mass_is_cell_volume_times_sum(orc):
    f = orc.initial_condition(O.CH, (6, 7, 8), seed=1, mean=0.3, amp=0.2)
    assert orc.mass(f, h=0.5) == pytest.approx(0.125 * math.fsum(f.ravel()), rel=1e-15)


def test_free_energy_closed_form_mode(orc):
    """F_h of phi = A cos(theta x) on an nx x ny grid: the gradient sum is
    A^2 nx ny (1 - cos theta) / h^2, sum phi^2 = A^2 N/2, sum phi^4 = 3 A^4 N / 8."""
    nx, ny, k, A, h = 16, 6, 3, 0.8, 0.5
    f, th = mode_field((ny, nx), (k, 0), amp=A)
    c1, c2 = 1.3, 0.7
    N = nx * ny
    expect = h * h * (0.5 * A * A * N * (1 - math.cos(th[0])) / h ** 2
                      - 0.5 * c1 * A * A * N / 2 + 0.25 * c2 * 3 * A ** 4 * N / 8)
    assert orc.free_energy(f, h=h, c1=c1, c2=c2) == pytest.approx(expect, rel=1e-13)


@pytest.mark.parametrize("dims", [2, 3])
def test_free_energy_summation_by_parts(orc, dims):
    """Under periodic BCs the forward-difference gradient energy equals
    -1/2 h^d sum phi L_h phi with the 5-/7-point stencil (summation by parts)."""
    shape = SHAPES[dims]
    f = orc.initial_condition(O.AC, shape, seed=9, amp=1.0)
    h = 0.8
    st = O.S1 if dims == 2 else O.S4
    grad = orc.free_energy(f, h=h, c1=0.0, c2=0.0)
    sbp = -0.5 * h ** dims * math.fsum((f * orc.laplacian(st, f, h)).ravel())
    assert grad == pytest.approx(sbp, rel=1e-13)


# ------------------------------------------------------- initial condition


def test_splitmix64_published_outputs(orc):
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    assert rows
    for seed, n, out in rows:
        assert orc.splitmix64_nth(int(seed), int(n)) == int(out)
        assert orc.u01(int(seed), int(n)) == (int(out) >> 11) * 2.0 ** -53


def test_noise_initial_condition_statistics(orc):
    """U(mean - amp, mean + amp) noise: bounds, moments and a KS test against uniform."""
    scipy_stats = pytest.importorskip("scipy.stats")
    f = orc.initial_condition(O.AC, (256, 256), seed=0, mean=0.0, amp=0.1)
    assert f.min() >= -0.1 and f.max() < 0.1
    assert abs(f.mean()) < 3 * 0.1 / math.sqrt(3 * f.size)
    assert f.var() == pytest.approx(0.01 / 3, rel=0.02)
    assert scipy_stats.kstest((f.ravel() + 0.1) / 0.2, "uniform").pvalue > 1e-3
    g = orc.initial_condition(O.AC, (256, 256), seed=1, mean=0.0, amp=0.1)
    assert not np.array_equal(f, g)


@pytest.mark.parametrize("dims", [2, 3])
def test_gray_scott_patches(orc, dims):
    """Without noise a single patch is exactly patch^d points at (0.5, 0.25) forming a
    periodically wrapped square/cube; everything else is (1, 0)."""
    shape = (40, 48) if dims == 2 else (12, 14, 16)
    patch = 6
    for seed in range(5):
        u, v = orc.initial_condition(O.GS, shape, seed=seed, amp=0.0, patches=1, patch=patch)
        m = u == 0.5
        assert m.sum() == patch ** dims
        assert np.all(v[m] == 0.25) and np.all(u[~m] == 1.0) and np.all(v[~m] == 0.0)
        for ax in range(dims):
            proj = m.any(axis=tuple(a for a in range(dims) if a != ax))
            assert proj.sum() == patch
            # a contiguous run on the ring: exactly one start
            assert int((proj & ~np.roll(proj, 1)).sum()) == 1
            # centred on the generator's draw c = splitmix64(seed, 2N + a) mod n_a, where
            # a = 0, 1, 2 is the physical axis x, y, z (numpy axis dims-1-a)
            a = dims - 1 - ax
            n_a = shape[ax]
            N = int(np.prod(shape))
            c = orc.splitmix64_nth(seed, 2 * N + a) % n_a
            want = {(c - patch // 2 + j) % n_a for j in range(patch)}
            assert set(np.flatnonzero(proj).tolist()) == want
    u, v = orc.initial_condition(O.GS, shape, seed=3, amp=0.01, patches=8, patch=patch)
    base_u = np.where(np.abs(u - 0.5) < 0.02, 0.5, 1.0)
    assert np.abs(u - base_u).max() <= 0.01
    assert np.abs(v - np.where(base_u == 0.5, 0.25, 0.0)).max() <= 0.01


@pytest.mark.parametrize("model,shape", [(O.CH, (40, 48)), (O.GS, (40, 48)), (O.AC, (12, 14, 16)),
                                         (O.GS, (12, 14, 16)), (O.MC, (40, 48)), (O.MC, (12, 14, 16))])
def test_initial_condition_window_matches_full_grid(orc, model, shape):
    """A window of the initial condition, with periodic wrap, equals the same
    slice of the full-grid initial condition (including Gray-Scott patches)."""
    kw = dict(seed=7, amp=0.05)
    if model == O.GS:
        kw.update(patches=5, patch=6)
    full = orc.initial_condition(model, shape, **kw)
    dims = len(shape)
    for origin in [(0,) * dims, (-3, 5, 11)[:dims], (35, 44, 13)[:dims]]:
        wshape = (9, 7, 5)[:dims]
        win = orc.initial_condition_window(model, shape, origin, wshape, **kw)
        idx = np.ix_(*[(np.arange(w) + o) % n for w, o, n in zip(wshape, origin, shape)])
        if model in (O.GS, O.MC):
            assert np.array_equal(win[0], full[0][idx]) and np.array_equal(win[1], full[1][idx])
        else:
            assert np.array_equal(win, full[idx])


# ------------------------------------------------------------ Model C
#
# F = sum h^d [ 1/2 |D+ phi|^2 - c1/2 phi^2 + c2/4 phi^4 + 1/2 rho^2 - c3 phi^2 rho ]
# dphi/dt = -dF/dphi = lap phi + c1 phi - c2 phi^3 + 2 c3 phi rho
# drho/dt = lap dF/drho = lap (rho - c3 phi^2)

MC_DT = 0.02


@pytest.mark.parametrize("st", ALL)
def test_model_c_uncoupled_reduces_to_allen_cahn_and_diffusion(orc, st):
    """With c3 = 0 the two fields decouple: phi follows Allen-Cahn bit for bit, and a
    Fourier mode of rho decays exactly as (1 - dt lambda / h^2)^n."""
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    h, n = 1.0, 25
    phi = orc.initial_condition(O.AC, shape, seed=13, amp=0.6)
    rho, th = mode_field(shape, (1, 3, 2)[:dims], amp=0.4)
    prm = O.params(c1=0.8, c2=1.2, c3=0.0)
    a, b = orc.step(O.MC, st, phi, rho, h=h, dt=MC_DT, prm=prm, nsteps=n)
    assert np.array_equal(a, orc.step(O.AC, st, phi, h=h, dt=MC_DT, prm=prm, nsteps=n))
    lam = symbol(st, th)
    np.testing.assert_allclose(b, (1 - MC_DT * lam / h ** 2) ** n * rho, rtol=0, atol=1e-13)


@pytest.mark.parametrize("c3", [0.5, 0.3])
def test_model_c_uniform_state_update(orc, c3):
    """Uniform (phi0, rho0): the Laplacians vanish, rho stays exactly, and phi moves by
    dt phi0 (c1 - c2 phi0^2 + 2 c3 rho0) (the coupling's sign and factor 2)."""
    c1, c2, phi0, rho0 = 0.8, 1.1, 0.6, -0.7
    u = np.full(SHAPES[2], phi0)
    v = np.full(SHAPES[2], rho0)
    a, b = orc.step(O.MC, O.S1, u, v, dt=MC_DT, prm=O.params(c1=c1, c2=c2, c3=c3), nsteps=1)
    assert np.all(b == rho0)
    expect = phi0 + MC_DT * phi0 * (c1 - c2 * phi0 ** 2 + 2 * c3 * rho0)
    np.testing.assert_allclose(a, expect, rtol=4e-16, atol=0)


@pytest.mark.parametrize("st", ALL)
def test_model_c_linear_response_of_both_fields(orc, st):
    """About a uniform state (phi0, rho0), a small Fourier mode in phi or in rho
    evolves for one step by the linearised update
        dphi' = dphi + dt [ (-lam + c1 - 3 c2 phi0^2 + 2 c3 rho0) dphi + 2 c3 phi0 drho ]
        drho' = drho + dt [ -lam (drho - 2 c3 phi0 dphi) ]
    (lam = lambda/h^2 of the stencil): fixes the sign and size of every term of both
    equations, including the two couplings."""
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    h, eps = 1.1, 1e-6
    c1, c2, c3, phi0, rho0 = 0.9, 1.3, 0.5, 0.35, 0.25
    prm = O.params(c1=c1, c2=c2, c3=c3)
    mode, th = mode_field(shape, (2, 1, 3)[:dims])
    lam = symbol(st, th) / h ** 2
    base = [np.full(shape, phi0), np.full(shape, rho0)]
    b0 = orc.step(O.MC, st, *base, h=h, dt=MC_DT, prm=prm, nsteps=1)
    a_phi = c1 - 3 * c2 * phi0 ** 2 + 2 * c3 * rho0
    for which in (0, 1):
        pert = [base[0] + (eps * mode if which == 0 else 0), base[1] + (eps * mode if which == 1 else 0)]
        out = orc.step(O.MC, st, *pert, h=h, dt=MC_DT, prm=prm, nsteps=1)
        dphi, drho = (eps, 0.0) if which == 0 else (0.0, eps)
        pred_phi = dphi + MC_DT * ((-lam + a_phi) * dphi + 2 * c3 * phi0 * drho)
        pred_rho = drho + MC_DT * (-lam * (drho - 2 * c3 * phi0 * dphi))
        np.testing.assert_allclose(out[0] - b0[0], pred_phi * mode, rtol=0, atol=1e-3 * eps)
        np.testing.assert_allclose(out[1] - b0[1], pred_rho * mode, rtol=0, atol=1e-3 * eps)


@pytest.mark.parametrize("st", [O.S1, O.S3, O.S4, O.S5])
def test_model_c_conserves_density(orc, st):
    """drho/dt is a Laplacian: the sum of rho is conserved to rounding, the sum of phi
    is not."""
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    u, v = orc.initial_condition(O.MC, shape, seed=17, mean=0.1, amp=0.5)
    a, b = orc.step(O.MC, st, u, v, dt=MC_DT, nsteps=200)
    assert abs(b.sum() - v.sum()) / (v.size * np.abs(v).max()) < 200 * 1e-15
    assert abs(a.sum() - u.sum()) > 1e-3


@pytest.mark.parametrize("st", [O.S1, O.S4])
def test_model_c_free_energy_decreases(orc, st):
    """The dynamics are the gradient flow of the listing's free energy, so for a small
    time step F decreases at every step (the printed equation's signs would not be a
    gradient flow of this F)."""
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    u, v = orc.initial_condition(O.MC, shape, seed=19, mean=0.2, amp=0.8)
    prm = O.params(c1=1.0, c2=1.0, c3=0.5)
    F = [O.free_energy_c(u, v, c1=1.0, c2=1.0, c3=0.5)]
    for _ in range(60):
        u, v = orc.step(O.MC, st, u, v, dt=0.005, prm=prm, nsteps=1)
        F.append(O.free_energy_c(u, v, c1=1.0, c2=1.0, c3=0.5))
    assert all(b < a for a, b in zip(F, F[1:])), F


def test_model_c_free_energy_closed_form(orc):
    """Uniform fields: F = V (-c1/2 phi0^2 + c2/4 phi0^4 + rho0^2/2 - c3 phi0^2 rho0)."""
    shape, h = (6, 8, 10), 0.5
    c1, c2, c3, phi0, rho0 = 0.7, 1.4, 0.45, 0.6, -0.3
    F = O.free_energy_c(np.full(shape, phi0), np.full(shape, rho0), h=h, c1=c1, c2=c2, c3=c3)
    V = np.prod(shape) * h ** 3
    expect = V * (-c1 / 2 * phi0 ** 2 + c2 / 4 * phi0 ** 4 + rho0 ** 2 / 2 - c3 * phi0 ** 2 * rho0)
    assert math.isclose(F, expect, rel_tol=1e-13)


def test_model_c_initial_condition_streams(orc):
    """Model C's two fields are uniform noise from generator streams i (phi) and N + i
    (rho), independent of each other."""
    shape = (9, 11)
    u, v = orc.initial_condition(O.MC, shape, seed=21, mean=0.1, amp=0.4)
    N = u.size
    for i in (0, 5, N - 1):
        assert u.ravel()[i] == 0.1 + 0.4 * (2 * O.u01(21, i) - 1)
        assert v.ravel()[i] == 0.1 + 0.4 * (2 * O.u01(21, N + i) - 1)


# ------------------------------------------------------------ Model H
#
# mu = -lap m - c1 m + c2 m^3;  dm/dt = lap mu - c3 div(m j);  dj/dt = lap j - c3 m grad mu
# (signs of the paper's EQUATION_OF listing); grad / div by central differences of
# the stencil's order: radius 1 (f(+1) - f(-1)) / 2h, radius 2 (8 (f(+1) - f(-1)) -
# (f(+2) - f(-2))) / 12h.

MH_DT = 0.004  # inside the forward-Euler bound of every stencil for these coefficients


def diff_symbol(st, theta):
    """D cos(theta x) = -s sin(theta x) and D sin(theta x) = s cos(theta x), unscaled."""
    if O.STENCIL_RADIUS[st] == 1:
        return 2 * math.sin(theta)
    return 16 * math.sin(theta) - 2 * math.sin(2 * theta)


def grad_scale(st, h):
    return 1 / (2 * h) if O.STENCIL_RADIUS[st] == 1 else 1 / (12 * h)


def sin_field(shape, ks, amp=1.0):
    idx = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")[::-1]
    ph = sum(2 * np.pi * k * i / n for k, i, n in zip(ks, idx, shape[::-1]))
    return amp * np.sin(ph)


@pytest.mark.parametrize("st", ALL)
def test_model_h_uncoupled(orc, st):
    """c3 = 0: m follows Cahn-Hilliard (to rounding: the scaling of the outer
    Laplacian is folded differently) and each component of j diffuses, a mode
    decaying exactly as (1 - dt lambda / h^2)^n."""
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    h, n = 1.0, 20
    m = orc.initial_condition(O.CH, shape, seed=23, amp=0.4)
    js = []
    for a in range(dims):
        f, th = mode_field(shape, tuple((a + 1, 2, 1)[:dims]), amp=0.3)
        js.append(f)
    prm = O.params(c1=0.9, c2=1.1, c3=0.0)
    mo, jo = O.step_h(st, m, js, h=h, dt=MH_DT, prm=prm, nsteps=n)
    ref = orc.step(O.CH, st, m, h=h, dt=MH_DT, prm=prm, nsteps=n)
    np.testing.assert_allclose(mo, ref, rtol=0, atol=1e-13)
    for a in range(dims):
        _, th = mode_field(shape, tuple((a + 1, 2, 1)[:dims]))
        lam = symbol(st, th)
        np.testing.assert_allclose(jo[a], (1 - MH_DT * lam / h ** 2) ** n * js[a], rtol=0, atol=1e-13)


@pytest.mark.parametrize("st", ALL)
def test_model_h_current_from_a_density_mode(orc, st):
    """m = m0 + eps cos(theta.x), j = 0: one step gives
    j_a = dt c3 g m0 dmu s_a sin(theta.x)  (from -c3 m grad mu), with
    dmu = eps (3 c2 m0^2 - c1 + kappa lambda/h^2), s_a the difference symbol, g its
    scale; m moves by -dt (lambda/h^2) dmu cos(theta.x) (the outer Laplacian)."""
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    h, eps, m0 = 0.9, 1e-6, 0.4
    c1, c2, kappa, c3 = 0.8, 1.2, 1.0, 0.7
    ks = (2, 1, 3)[:dims]
    f, th = mode_field(shape, ks)
    lam = symbol(st, th) / h ** 2
    dmu = eps * (3 * c2 * m0 ** 2 - c1 + kappa * lam)
    prm = O.params(c1=c1, c2=c2, kappa=kappa, c3=c3)
    m = m0 + eps * f
    mo, jo = O.step_h(st, m, [np.zeros(shape)] * dims, h=h, dt=MH_DT, prm=prm, nsteps=1)
    s = sin_field(shape, ks)
    g = grad_scale(st, h)
    for a in range(dims):
        pred = MH_DT * c3 * g * m0 * dmu * diff_symbol(st, th[a]) * s
        np.testing.assert_allclose(jo[a], pred, rtol=0, atol=1e-3 * eps * MH_DT)
    # second-order terms (dt lambda 3 c2 m0 eps^2 ~ 1e-13) stay far below the first-order ones (~6e-8)
    np.testing.assert_allclose(mo - m0, (eps - MH_DT * lam * dmu) * f, rtol=0, atol=1e-6 * eps)


@pytest.mark.parametrize("st", ALL)
def test_model_h_density_from_a_current_mode(orc, st):
    """m = m0, j_x = eps sin(theta.x): one step moves m by
    -dt c3 g m0 eps s_x cos(theta.x)  (from -c3 div(m j)) and j_x diffuses."""
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    h, eps, m0 = 1.1, 1e-6, 0.35
    c3 = 0.6
    ks = (1, 2, 1)[:dims]
    f, th = mode_field(shape, ks)
    s = sin_field(shape, ks)
    lam = symbol(st, th) / h ** 2
    js = [eps * s] + [np.zeros(shape)] * (dims - 1)
    mo, jo = O.step_h(st, np.full(shape, m0), js, h=h, dt=MH_DT, prm=O.params(c3=c3), nsteps=1)
    g = grad_scale(st, h)
    np.testing.assert_allclose(mo - m0, -MH_DT * c3 * g * m0 * eps * diff_symbol(st, th[0]) * f, rtol=0,
                               atol=1e-9 * eps)
    np.testing.assert_allclose(jo[0], (1 - MH_DT * lam) * eps * s, rtol=0, atol=1e-9 * eps)
    for a in range(1, dims):
        assert np.abs(jo[a]).max() == 0.0


@pytest.mark.parametrize("st", [O.S1, O.S3, O.S4])
def test_model_h_conserves_m(orc, st):
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    m, js = O.initial_condition_h(shape, seed=29, mean=0.1, amp=0.5)
    mo, jo = O.step_h(st, m, js, dt=MH_DT, prm=O.params(c3=1.0), nsteps=100)
    assert abs(mo.sum() - m.sum()) / (m.size * np.abs(m).max()) < 100 * 1e-15
    assert abs(jo[0].sum() - js[0].sum()) > 1e-6  # j is not conserved


@pytest.mark.parametrize("st", [O.S1, O.S4])
def test_model_h_free_energy_decreases(orc, st):
    """With the listing's signs the couplings cancel in dF/dt, so F = Landau(m) +
    |j|^2/2 decreases at every small step."""
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    m, js = O.initial_condition_h(shape, seed=31, mean=0.1, amp=0.6)
    prm = O.params(c3=1.5)
    F = [O.free_energy_h(m, js)]
    for _ in range(40):
        m, js = O.step_h(st, m, js, dt=0.002, prm=prm, nsteps=1)
        F.append(O.free_energy_h(m, js))
    assert all(b < a for a, b in zip(F, F[1:])), F


@pytest.mark.parametrize("st", [O.S2, O.S5, O.S6])
def test_model_h_shift_equivariance(orc, st):
    dims = O.STENCIL_DIMS[st]
    shape = SHAPES[dims]
    axes = tuple(range(dims))
    shift = (3, -5, 2)[:dims]
    m, js = O.initial_condition_h(shape, seed=37, amp=0.3)
    prm = O.params(c3=0.8)
    a = O.step_h(st, m, js, dt=MH_DT, prm=prm, nsteps=3)
    b = O.step_h(st, np.roll(m, shift, axes), [np.roll(c, shift, axes) for c in js], dt=MH_DT, prm=prm, nsteps=3)
    assert np.array_equal(np.roll(a[0], shift, axes), b[0])
    for x, y in zip(a[1], b[1]):
        assert np.array_equal(np.roll(x, shift, axes), y)


def test_model_h_initial_condition_streams(orc):
    shape = (5, 6, 7)
    m, js = O.initial_condition_h(shape, seed=41, mean=0.2, amp=0.3)
    N = m.size
    for i in (0, 17, N - 1):
        assert m.ravel()[i] == 0.2 + 0.3 * (2 * O.u01(41, i) - 1)
        for a in range(3):
            assert js[a].ravel()[i] == 0.3 * (2 * O.u01(41, (a + 1) * N + i) - 1)
