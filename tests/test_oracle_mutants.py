"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (on the CPU; the
GPU path is not involved), compiles it to a temporary library and runs the pin
suite against it through ``SP_ORACLE_LIB``.  The suite must fail on every mutant.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sp_oracle.c")

MUTANTS = {
    "S1 centre weight": ("return fma(-4.0, P(0, 0, 0), C);", "return fma(-3.0, P(0, 0, 0), C);"),
    "S2 denominator": ("case OR_S2: return 6;", "case OR_S2: return 5;"),
    "S3 outer ring sign": ("return fma(-60.0, P(0, 0, 0), fma(16.0, F1, -F2));",
                           "return fma(-60.0, P(0, 0, 0), fma(16.0, F1, F2));"),
    "S5 corner weight": ("fma(3.0, E, K)", "fma(3.0, E, 2.0 * K)"),
    "S5 dropped edge plane": ("double E = D0 + (Cm + Cp);", "double E = D0 + (Cm + Cm);"),
    "S6 z ring": ("(P(0, 0, -2) + P(0, 0, 2))", "(P(0, 0, -2) + P(0, 0, 1))"),
    "y offset read from x table": ("int64_t yy = g->w[1][(dy + OR_MAXR)", "int64_t yy = g->w[1][(dx + OR_MAXR)"),
    "Allen-Cahn reaction sign": ("fma(-c2, p * p, c1)", "fma(c2, p * p, c1)"),
    "Allen-Cahn dropped c1": ("fma(-c2, p * p, c1)", "fma(-c2, p * p, 0.0)"),
    "Cahn-Hilliard kappa sign": ("-(kq * S));", "(kq * S));"),
    "Cahn-Hilliard c2 sign": ("fma(pi, fma(c2, pi * pi, -c1)", "fma(pi, fma(-c2, pi * pi, -c1)"),
    "Cahn-Hilliard outer Laplacian of phi": ("fma(dq, stencil_sum(st, mu, &g", "fma(dq, stencil_sum(st, uc, &g"),
    "Gray-Scott uv^2 sign in v": ("fma(dvq, stencil_sum(st, vc, &g, x, y, z), uvv)",
                                  "fma(dvq, stencil_sum(st, vc, &g, x, y, z), -uvv)"),
    "Gray-Scott F and k swapped": ("const double F = prm[P_F], Fk", "const double F = prm[P_K], Fk"),
    "Gray-Scott Du for Dv": ("dvq = prm[P_DV] / q_h2", "dvq = prm[P_DU] / q_h2"),
    "Gray-Scott v read from u": ("const double a = uc[i], b = vc[i];", "const double a = uc[i], b = uc[i];"),
    "free energy quartic": ("0.25 * c2 * p2 * p2", "0.5 * c2 * p2 * p2"),
    "free energy y gradient along x": ("const double gy = (f[(z * ny + (y + 1) % ny) * nx + x] - p) / h;",
                                       "const double gy = (f[(z * ny + y) * nx + (x + 1) % nx] - p) / h;"),
    "3D cell volume": ("dims == 3 ? (h * h) * h : h * h", "h * h"),
    "sum drops compensation": ("return s + c;", "return s;"),
    "one-sided noise": ("u[i] = mean + amp * (2.0 * or_u01(seed, (uint64_t)i) - 1.0);",
                        "u[i] = mean + amp * or_u01(seed, (uint64_t)i);"),
    "splitmix increment": ("(n + 1u) * UINT64_C(0x9E3779B97F4A7C15)", "n * UINT64_C(0x9E3779B97F4A7C15)"),
    "patch corner": ("int64_t l = (c - patch / 2) % nn[a];", "int64_t l = (c - patch) % nn[a];"),
    "Model C printed coupling sign in phi": ("fma(c3x2, r, c1)", "fma(-c3x2, r, c1)"),
    "Model C coupling without factor 2": ("c3x2 = 2.0 * prm[P_C3]", "c3x2 = prm[P_C3]"),
    "Model C printed sign in rho": ("mu[i] = fma(-c3, uc[i] * uc[i], vc[i]);",
                                    "mu[i] = fma(c3, uc[i] * uc[i], vc[i]);"),
    "Model C density Laplacian of rho only": ("vn[i] = fma(dq, stencil_sum(st, mu, &g, x, y, z), r);",
                                              "vn[i] = fma(dq, stencil_sum(st, vc, &g, x, y, z), r);"),
    "Model C free-energy coupling sign": ("+ 0.5 * r * r - c3 * p2 * r", "+ 0.5 * r * r + c3 * p2 * r"),
    "generated stencil accumulation sign": ("acc = (jj == g->gen_r) ? g->gen_w[jj] * pj : fma(g->gen_w[jj], pj, acc);",
                                            "acc = (jj == g->gen_r) ? g->gen_w[jj] * pj : fma(g->gen_w[jj], pj, -acc);"),
    "generated stencil without z pairs": ("if (g->gen_dims == 3) pj = pj + (P(0, 0, jj) + P(0, 0, -jj));",
                                          "if (g->gen_dims == 4) pj = pj + (P(0, 0, jj) + P(0, 0, -jj));"),
    "Model H printed coupling sign in j": ("-(c3g * (mc[i] * gm)))", "(c3g * (mc[i] * gm)))"),
    "Model H divergence sign": ("fma(sL, stencil_sum(st, mu, &g, x, y, z), -(c3g * div))",
                                "fma(sL, stencil_sum(st, mu, &g, x, y, z), (c3g * div))"),
    "Model H gradient of m instead of mu": ("const double gm = central_diff(radius, a, mu, &g, x, y, z);",
                                            "const double gm = central_diff(radius, a, mc, &g, x, y, z);"),
    "Model H 4th-order difference weight": ("return fma(8.0, d1, -d2);", "return fma(6.0, d1, -d2);"),
    "Model H gradient scale": ("1.0 / (2.0 * h) : 1.0 / (12.0 * h)", "1.0 / h : 1.0 / (12.0 * h)"),
    "Model H flux of j only": ("mj[(size_t)a * n + i] = mc[i] * jcur[a][i];", "mj[(size_t)a * n + i] = jcur[a][i];"),
    "Model H current noise stream": ("or_u01(seed, (uint64_t)((a + 1) * N + i))", "or_u01(seed, (uint64_t)(a * N + i))"),
    "relative L2 without the square root": ("return den > 0 ? sqrt(num / den) : sqrt(num);",
                                            "return den > 0 ? num / den : num;"),
    "relative L2 normalised by the first argument": ("r[i] = b[i] * b[i];", "r[i] = a[i] * a[i];"),
    "relative L2 of absolute differences": ("d[i] = (a[i] - b[i]) * (a[i] - b[i]);",
                                            "d[i] = fabs(a[i] - b[i]);"),
    "Model C density noise stream": ("            v[i] = mean + amp * (2.0 * or_u01(seed, (uint64_t)(N + i)) - 1.0);",
                                     "            v[i] = mean + amp * (2.0 * or_u01(seed, (uint64_t)i) - 1.0);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mut = src.replace(old, new)
    csrc = tmp_path / "mutant.c"
    csrc.write_text(mut)
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", str(so), str(csrc), "-lm"])
    env = dict(os.environ, SP_ORACLE_LIB=str(so), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_stencil_gen.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutant {name!r}:\n{r.stdout[-2000:]}"
