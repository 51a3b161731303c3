"""Thermodynamics of the reduced-precision paths at a lattice of the size
class of the benchmark workloads: FP32 and FP16 against FP64 within 3 sigma.

sc 64^3 periodic (262,144 spins), J = 1, K = 0.1, e = z, T = 1.0 (the
parameters of the 464^3 precision workload), 16 independent seeds per
precision.  Each chain starts ordered along e (so it equilibrates below T_c
without coarsening), runs 200 unmeasured and 500 measured sweeps; the
per-seed means of <E>/N, <|M|> and <|M.e|> are independent, so their spread
gives the standard error.  The FP64 path is pinned element by element to the
oracle elsewhere; here it is the reference.  Chains are bit-reproducible, so
the outcome is fixed for these seeds.
"""
import math

import numpy as np
import pytest

from paper_2106_11286_gb300 import hs

pytestmark = pytest.mark.gpu

L = 64
N = L ** 3
SEEDS = range(300, 316)


def run(precision, seed):
    with hs.Lattice("sc", dims=(L, L, L), J=1.0, K=0.1, e=(0, 0, 1), precision=precision, seed=seed) as lat:
        lat.init(hs.HS_INIT_ALIGNED)
        lat.sweep(1.0, 200)
        lat.accumulate(True)
        lat.reset_accumulator()
        lat.sweep(1.0, 500)
        mom, cnt = lat.read_accumulator()
    return np.array([mom[hs.MOMENTS.index("sum_E")] / cnt / N, mom[hs.MOMENTS.index("sum_absM")] / cnt,
                     mom[hs.MOMENTS.index("sum_absMe")] / cnt])


@pytest.fixture(scope="module")
def results():
    return {p: np.array([run(p, s) for s in SEEDS]) for p in ("fp64", "fp32", "fp16")}


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_within_three_sigma_of_fp64(results, precision):
    ref, got = results["fp64"], results[precision]
    n = len(SEEDS)
    for k, name in enumerate(("E/N", "|M|", "|M.e|")):
        diff = got[:, k].mean() - ref[:, k].mean()
        sigma = math.sqrt(got[:, k].var(ddof=1) / n + ref[:, k].var(ddof=1) / n)
        assert sigma > 0
        assert abs(diff) < 3 * sigma, (precision, name, diff, sigma)


def test_the_chains_are_ordered_and_distinct(results):
    # below T_c with K > 0: |M| near its ordered value, every seed its own chain
    assert 0.5 < results["fp64"][:, 1].mean() < 1.0
    for p in results:
        assert len(np.unique(results[p][:, 0])) == len(SEEDS)
