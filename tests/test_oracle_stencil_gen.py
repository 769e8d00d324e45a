"""Pins of the generated stencils (oracle/stencil_gen.py) and of the oracle's
steps with them (oracle.step_gen):
  * the weights equal the published central second-derivative coefficients
    (Fornberg, Math. Comp. 51 (1988), Table 1) for orders 2, 4, 6, 8;
  * the stencil is exact on polynomials up to degree order + 1 and converges
    at its order on a smooth periodic field;
  * order 4 in 2D equals this library's 4th-order 9-point cross S3 (same
    weights over 12), and the Fourier symbol of the generated cross stencil
    gives the exact decay of a diffusion mode;
  * the generated Allen-Cahn / Cahn-Hilliard / Gray-Scott / Model C steps reduce
    to the fixed-stencil steps where the stencils coincide (order 2).
``SP_ORACLE_STENCIL_GEN`` may name another copy of the module (mutant tests)."""
import importlib.util
import math
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O


def _load():
    path = os.environ.get("SP_ORACLE_STENCIL_GEN")
    if not path:
        from oracle import stencil_gen

        return stencil_gen
    spec = importlib.util.spec_from_file_location("stencil_gen_under_test", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


G = _load()

PUBLISHED = {  # w_0, w_1, ..., w_r of the central second derivative
    2: [Fr(-2), Fr(1)],
    4: [Fr(-5, 2), Fr(4, 3), Fr(-1, 12)],
    6: [Fr(-49, 18), Fr(3, 2), Fr(-3, 20), Fr(1, 90)],
    8: [Fr(-205, 72), Fr(8, 5), Fr(-1, 5), Fr(8, 315), Fr(-1, 560)],
}


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_weights_equal_published_coefficients(order):
    assert G.second_derivative_weights(order) == PUBLISHED[order]


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_exact_on_polynomials(order):
    w = G.second_derivative_weights(order)
    r = order // 2
    for k in range(order + 2):
        lhs = w[0] * (1 if k == 0 else 0) + sum(wj * (j ** k + (-j) ** k) for j, wj in enumerate(w[1:], start=1))
        assert lhs == (2 if k == 2 else 0), (order, k)


@pytest.mark.parametrize("order", [2, 4, 6])
def test_convergence_order(order):
    """Error of the 1D second derivative of sin(2 pi x) on [0, 1) falls as h^order."""
    w = [float(x) for x in G.second_derivative_weights(order)]
    errs = []
    for n in (32, 64):
        h = 1.0 / n
        x = np.arange(n) * h
        f = np.sin(2 * np.pi * x)
        d2 = w[0] * f + sum(wj * (np.roll(f, -j) + np.roll(f, j)) for j, wj in enumerate(w[1:], start=1))
        d2 /= h * h
        errs.append(np.abs(d2 + (2 * np.pi) ** 2 * f).max())
    rate = math.log2(errs[0] / errs[1])
    assert abs(rate - order) < 0.2, rate


def test_order_4_in_2d_is_the_library_s3_stencil():
    """The 2D cross of order 4 has kernel weights (2 w_0, w_1, w_2) = (-60, 16, -1)/12,
    the integer weights of S3 over its denominator 12."""
    wk = G.kernel_weights(4, 2)
    assert wk == [-60 / 12, 16 / 12, -1 / 12]


@pytest.mark.parametrize("order,dims", [(2, 2), (4, 3), (6, 2), (8, 3)])
def test_diffusion_mode_decay_with_generated_stencil(order, dims):
    """Allen-Cahn with c1 = c2 = 0: a Fourier mode decays by (1 - dt lambda / h^2)^n,
    lambda = -sum_axes (w_0 + 2 sum_j w_j cos(j theta_a))."""
    shape = (12, 16) if dims == 2 else (10, 12, 14)
    ks = (3, 2, 1)[:dims]
    idx = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")[::-1]
    th = [2 * np.pi * k / n for k, n in zip(ks, shape[::-1])]
    f = 0.3 * np.cos(sum(t * i for t, i in zip(th, idx)))
    w = [float(x) for x in G.second_derivative_weights(order)]
    lam = -sum(w[0] + 2 * sum(wj * math.cos(j * t) for j, wj in enumerate(w[1:], start=1)) for t in th)
    h, dt, n = 1.0, 0.02, 30
    out = O.step_gen(O.AC, order, f, h=h, dt=dt, prm=O.params(c1=0.0, c2=0.0), nsteps=n)
    np.testing.assert_allclose(out, (1 - dt * lam / h ** 2) ** n * f, rtol=0, atol=1e-13)


@pytest.mark.parametrize("order,dims", [(2, 2), (4, 2), (6, 3), (8, 3)])
def test_lambda_max(order, dims):
    w = [float(x) for x in G.second_derivative_weights(order)]
    lam_pi = -dims * (w[0] + 2 * sum(wj * (-1) ** j for j, wj in enumerate(w[1:], start=1)))
    assert math.isclose(G.lambda_max(order, dims), lam_pi, rel_tol=1e-15)
    assert G.lambda_max(2, 2) == 8.0 and G.lambda_max(2, 3) == 12.0


@pytest.mark.parametrize("model", [O.AC, O.CH, O.GS, O.MC])
def test_order_2_steps_equal_the_fixed_5_and_7_point_steps(model):
    """Order 2 is the 5-point (2D) / 7-point (3D) stencil with the same evaluation
    order (the pair sums, then fma with the centre), so the steps agree bit for bit."""
    for shape, st in [((12, 16), O.S1), ((8, 10, 12), O.S4)]:
        dt = {O.AC: 0.05, O.CH: 0.002, O.GS: 0.5, O.MC: 0.02}[model]
        if model == O.GS:
            u, v = O.initial_condition(O.GS, shape, seed=3, amp=0.1, patches=2, patch=3)
        elif model == O.MC:
            u, v = O.initial_condition(O.MC, shape, seed=3, amp=0.3)
        else:
            u, v = O.initial_condition(model, shape, seed=3, amp=0.4), None
        args = (u,) if v is None else (u, v)
        a = O.step_gen(model, 2, *args, dt=dt, nsteps=4)
        b = O.step(model, st, *args, dt=dt, nsteps=4)
        if v is None:
            assert np.array_equal(a, b)
        else:
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
