"""The stencil generator's pins must catch plausible mistakes: each case plants
one in a copy of oracle/stencil_gen.py and runs tests/test_oracle_stencil_gen.py
against it through ``SP_ORACLE_STENCIL_GEN``; the suite must fail."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "stencil_gen.py")

MUTANTS = {
    "centre weight without the factor 2": ("return [-2 * sum(w)] + w", "return [-sum(w)] + w"),
    "odd powers in the system": ("[Fraction(j ** (2 * m)) for j", "[Fraction(j ** (2 * m - 1)) for j"),
    "right-hand side on the wrong row": ("Fraction(1 if m == 1 else 0)", "Fraction(1 if m == 2 else 0)"),
    "kernel centre not times d": ("return [float(dims * w[0])]", "return [float(w[0])]"),
    "lambda_max at theta = 0": ("(-1) ** j for j, wj", "1 ** j for j, wj"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_stencil_gen_pins_reject_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    mut = tmp_path / "stencil_gen_mutant.py"
    mut.write_text(src.replace(old, new))
    env = dict(os.environ, SP_ORACLE_STENCIL_GEN=str(mut))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_stencil_gen.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0, f"pins did not catch mutant {name!r}:\n{r.stdout[-2000:]}"
