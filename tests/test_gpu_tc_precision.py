"""T_c of each precision path from the Binder-cumulant crossing (Eq. 2's
magnetisation, U4 = 1 - <M^4> / (3 <M^2>^2)), against the FP64 path.

sc L = 8 and 16, periodic, J = 1, K = 0, T = 1.38 .. 1.50 in steps of 0.04,
6 replicas per point, 2000 equilibration sweeps and 8 blocks of 1000 sweeps;
FP32 runs batched, FP64 and FP16 lattice by lattice.  The crossing of the
two sizes, with a jackknife error, must agree between FP32 / FP16 and FP64
within 3 sigma of the difference, and lie within max(3 sigma, 0.03) of the
sc Heisenberg T_c = 1.443 J (small sizes shift the crossing a little).  The
FP64 path is pinned to the oracle element by element in the parity tests.
"""
import math

import pytest

from paper_2106_11286_gb300 import scan

pytestmark = pytest.mark.gpu

SIZES = (8, 16)
TEMPS = (1.38, 1.42, 1.46, 1.50)


@pytest.fixture(scope="module")
def crossings():
    out = {}
    for precision in ("fp64", "fp32", "fp16"):
        sc = scan.run_scan(SIZES, TEMPS, n_equil=2000, n_blocks=8, block_sweeps=1000, replicas=6,
                           precision=precision, seed=91)
        out[precision] = scan.binder_crossing(sc, 0, 1)
    return out


def test_fp64_crossing_near_tc(crossings):
    tc, err = crossings["fp64"]
    assert math.isfinite(tc) and math.isfinite(err)
    assert abs(tc - 1.443) < max(3 * err, 0.03), (tc, err)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_reduced_precision_tc_within_three_sigma_of_fp64(crossings, precision):
    t64, e64 = crossings["fp64"]
    tp, ep = crossings[precision]
    assert math.isfinite(tp)
    assert abs(tp - t64) < 3 * math.hypot(e64, ep), (precision, tp, ep, t64, e64)
