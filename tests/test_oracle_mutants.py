"""The oracle's pins catch planted mistakes.

Each mutant is the oracle compiled with one deliberate mistake (the step
marked PLANTED(k) in ``oracle/gsta_oracle.c``): a dropped term, a sign flip,
a transposed operand, a missing Jacobian entry, a wrong constant or cut-off,
a wrong tie order, a skipped freeze test. The oracle's CPU pins
(``tests/test_oracle_*.py`` and the finite-difference checks in
``tests/test_fd_local.py``) run against each mutant in a child process and
must fail; against the oracle itself they pass (the rest of this suite).
"""
import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    1: "dilation not added to the 2-D covariance",
    2: "Jacobian entry -fx x / z^2 dropped",
    3: "world-to-camera rotation transposed",
    4: "SH normalisation without (l - m)! / (l + m)!",
    5: "compositing weight takes the transmittance after the splat",
    6: "sign of dL/dmean2d x flipped",
    7: "background dropped from the colour behind a splat (backward)",
    8: "SSIM constant C2 = 0.02^2",
    9: "Adam second-moment bias correction dropped",
    10: "freeze on either gradient norm instead of both",
    11: "transmittance cut-off 1e-3",
    12: "Adam updates frozen Gaussians",
    13: "equal sort keys in descending index order",
    14: "alpha cap 0.99 dropped",
    15: "view-dependent colour's gradient with respect to the mean dropped",
    16: "quaternion normalisation's projection dropped (backward)",
    17: "factor 2 of the projected-covariance gradient dropped",
    18: "clamped screen coordinates still pass gradient",
    19: "positional gradient norm in pixels instead of (W/2, H/2) units",
}


def _pins(k: int) -> subprocess.CompletedProcess:
    files = sorted(f for f in glob.glob(os.path.join(ROOT, "tests", "test_oracle_*.py"))
                   if not f.endswith("test_oracle_mutants.py"))
    files.append(os.path.join(ROOT, "tests", "test_fd_local.py"))
    env = dict(os.environ, GSTA_ORACLE_PLANT=str(k))
    return subprocess.run([sys.executable, "-m", "pytest", *files, "-x", "-q", "-p", "no:cacheprovider",
                           "-m", "not gpu"], env=env, cwd=ROOT, capture_output=True, text=True, timeout=900)


@pytest.fixture(scope="module")
def outcomes():
    import oracle

    for k in MUTANTS:
        oracle.build(plant=k)
    with ThreadPoolExecutor(4) as ex:
        return dict(zip(MUTANTS, ex.map(_pins, MUTANTS)))


@pytest.mark.parametrize("k", sorted(MUTANTS))
def test_pins_fail_on_planted_mistake(outcomes, k):
    p = outcomes[k]
    tail = p.stdout[-2000:] + p.stderr[-500:]
    assert p.returncode == 1 and " failed" in p.stdout, f"mutant {k} ({MUTANTS[k]}) survived or crashed:\n{tail}"
