"""The paper's M(T) curve and critical exponent, at a test-sized lattice.

sc 32^3 and 64^3 periodic, J = 1, K = 0.01 (the paper's anisotropy), e = z,
ordered start, T = 1.20 .. 1.46, 2 replicas per point in one persistent FP32
batch, 3000 equilibration sweeps and 10 blocks of 500.  T_c is the Binder
crossing of the two sizes; beta is the paper's fit, least squares of
log <|M|> on log(T_c - T) over the points T <= 1.40, with a jackknife error
that includes T_c's.
* T_c: within [1.440, 1.460].  The isotropic model's literature value is
  1.443 (the paper quotes 1.445 for K = 0.01); a small easy-axis anisotropy
  raises it (128^3 / 64^3 measured 1.4508 +- 0.0005).
* beta: within max(3 sigma, 0.045) of the 3D Heisenberg exponent 0.369.
  The fit over this range gives an effective exponent: the corrections to
  scaling lower it by about 0.035 here (128^3 measured 0.333 +- 0.002 and
  256^3 the same within 0.002), so the asymptotic value is reached only
  closer to T_c.  Mean-field (0.5) and 2D (0.125) values are far outside.
"""
import pytest

from paper_2106_11286_gb300 import scan

pytestmark = pytest.mark.gpu

TEMPS = (1.20, 1.25, 1.30, 1.34, 1.37, 1.40, 1.42, 1.43, 1.44, 1.45, 1.46)


@pytest.fixture(scope="module")
def curve():
    return scan.run_scan((32, 64), TEMPS, n_equil=3000, n_blocks=10, block_sweeps=500, replicas=2, K=0.01, seed=55,
                         init="aligned")


def test_curie_temperature_from_the_crossing(curve):
    tc, err = scan.binder_crossing(curve, 0, 1)
    assert 1.440 <= tc <= 1.460, (tc, err)


def test_beta_from_the_power_law_fit(curve):
    fit = [j for j, T in enumerate(TEMPS) if T <= 1.40]
    beta, err, tc = scan.beta_fit(curve, 1, fit, tc_sizes=(0, 1))
    assert err > 0
    assert abs(beta - 0.369) < max(3 * err, 0.045), (beta, err, tc)


def test_magnetisation_falls_towards_tc(curve):
    m = [curve.absM[(1, j)].mean() for j in range(len(TEMPS))]
    assert all(a > b for a, b in zip(m, m[1:]))
    assert m[0] > 0.5 and m[-1] < 0.15
