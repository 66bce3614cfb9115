"""The oracle's pins catch planted mistakes.

Each mutant is the oracle with one deliberate mistake: the step marked
PLANTED(k) in ``oracle/gsta_oracle.c`` (compiled in with -DORACLE_PLANT=k)
or ``planted(k)`` in the oracle's Python modules (switched on by the
environment variable GSTA_ORACLE_PLANT=k) -- a dropped term, a sign flip, a
transposed operand, a missing Jacobian entry, a wrong constant or cut-off,
a wrong tie order, a skipped freeze test, a wrong schedule or selection. The oracle's CPU pins
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
    20: "predictor: first hidden layer without its ReLU",
    21: "predictor: second ReLU's derivative dropped in the gradient",
    22: "predictor: bfloat16 by truncation instead of round-to-nearest-even",
    23: "predictor history: one view per visible window instead of the visible count",
    24: "predictor feature 8: opacity logit instead of the opacity",
    25: "predicted freezing clears an existing freeze",
    26: "predictor Adam: first-moment bias correction dropped",
    27: "densification clones the large candidates and splits the small",
    28: "split children offset without the Gaussian's rotation",
    29: "a split original is kept beside its children",
    30: "opacity reset leaves the opacity's Adam moments",
    31: "Eq. 5 thresholds without the [0.5, 1.5] clamp",
    32: "Eq. 7 early stop on the most recent PSNR change alone",
    33: "no waiting period after a freeze-map reset",
    34: "significance score without the opacity factor",
    35: "significance pruning removes the highest scores",
    36: "plateau schedule decays without patience",
    37: "mingrad score takes the smaller of the two ratios",
    38: "Gaussians not seen in the window are eligible for freezing",
    39: "downscaled camera's principal point without the half-pixel shift",
    40: "area average footprint shifted by half a source pixel",
    41: "blur kernel exp(-r^2 / sigma^2)",
    42: "absolute-value opacity: gradient without the sign of the parameter",
    43: "dL/dconic off-diagonal term halved",
    44: "tile membership cut-off at alpha 1/128 instead of 1/255",
    45: "volume mask threshold sigmoid(m) > 0.1 instead of 0.01",
    46: "batched step: the scene's gradient is its last view's, not the sum",
    47: "batched step: Adam's bias correction one step ahead of the scene's counter",
    48: "xyz rate without the vanilla exponential decay",
}


def _pins(k: int) -> subprocess.CompletedProcess:
    files = sorted(f for f in glob.glob(os.path.join(ROOT, "tests", "test_oracle_*.py"))
                   if not f.endswith("test_oracle_mutants.py"))
    files.append(os.path.join(ROOT, "tests", "test_fd_local.py"))
    env = dict(os.environ, GSTA_ORACLE_PLANT=str(k), OMP_NUM_THREADS="1")  # the children run side by side
    return subprocess.run([sys.executable, "-m", "pytest", *files, "-x", "-q", "-p", "no:cacheprovider",
                           "-m", "not gpu"], env=env, cwd=ROOT, capture_output=True, text=True, timeout=900)


@pytest.fixture(scope="module")
def outcomes():
    import oracle

    oracle.build()  # the unplanted library; each child compiles its own planted copy
    with ThreadPoolExecutor(max(2, min(8, os.cpu_count() or 2))) as ex:
        return dict(zip(MUTANTS, ex.map(_pins, MUTANTS)))


@pytest.mark.parametrize("k", sorted(MUTANTS))
def test_pins_fail_on_planted_mistake(outcomes, k):
    p = outcomes[k]
    tail = p.stdout[-2000:] + p.stderr[-500:]
    assert p.returncode == 1 and " failed" in p.stdout, f"mutant {k} ({MUTANTS[k]}) survived or crashed:\n{tail}"
