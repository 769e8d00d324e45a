"""The spectral oracle's pins must catch plausible mistakes: each case plants one
mistake in a copy of oracle/spectral.py (CPU only) and runs the pin suite against
it through ``SP_ORACLE_SPECTRAL``; the suite must fail."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "spectral.py")

MUTANTS = {
    "stencil symbol instead of |k|^2": ("return sum(k * k for k in mesh)",
                                        "return sum((2.0 / h * np.sin(k * h / 2.0)) ** 2 for k in mesh)"),
    "missing 2 pi on the full axes": ("k = 2.0 * np.pi * np.fft.fftfreq(n, d=h)", "k = np.fft.fftfreq(n, d=h)"),
    "Allen-Cahn Laplacian sign": ("return c1 - k2", "return c1 + k2"),
    "Cahn-Hilliard kappa sign": ("return k2 * (c1 - kappa * k2)", "return k2 * (c1 + kappa * k2)"),
    "Cahn-Hilliard nonlinear term without Laplacian": ("nh = -k2 * np.fft.rfftn(c2 * cube, axes=axes)",
                                                       "nh = np.fft.rfftn(c2 * cube, axes=axes)"),
    "explicit part subtracted": ("uh = (uh + dt * nh) / denom", "uh = (uh - dt * nh) / denom"),
    "Allen-Cahn cubic sign": ("nh = np.fft.rfftn(-c2 * cube, axes=axes)", "nh = np.fft.rfftn(c2 * cube, axes=axes)"),
    "stability bound": ("dt * c1 * c1 / (4.0 * kappa) < 1.0", "dt * c1 * c1 / (2.0 * kappa) < 1.0"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_spectral_pins_reject_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    mut = tmp_path / "spectral_mutant.py"
    mut.write_text(src.replace(old, new))
    env = dict(os.environ, SP_ORACLE_SPECTRAL=str(mut))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_spectral.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0, f"pins did not catch mutant {name!r}:\n{r.stdout[-2000:]}"
