"""The pins' own test: the oracle built with each planted mistake
(oracle.c, ORC_MUTANT = 1..16: flipped warp direction, swapped
interpolation weights, a dropped mean product in Eq. 3, the sample instead
of the population variance, a factor 2 in Eqs. 9-10, border neighbours
included, ties to the largest d, a flipped parabola offset, a sign slip in
the L-R check, in post-processing, Y from u, the target volume's direction,
the gradient's weight term, the least-squares slope, the roll sign, and an
off-by-one search window) must fail at least one pin test."""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_grad.py", "tests/test_oracle_fit.py",
        "tests/test_oracle_restricted.py"]
MUTANTS = list(range(1, 17))


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("mutants")


@pytest.mark.parametrize("k", MUTANTS)
def test_planted_mistake_fails_a_pin(k, mutant_dir):
    lib = oracle.build(out=str(mutant_dir / f"liboracle_m{k}.so"), mutant=k)
    env = dict(os.environ, ORC_LIB=lib, OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *PINS], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"mutant {k} passed every pin:\n{r.stdout[-2000:]}"
