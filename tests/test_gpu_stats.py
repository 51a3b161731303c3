"""Thermodynamics of the reduced-precision paths against the FP64 path.

sc 16^3 periodic, J = 1, K = 0.1, e = z, T = 1.0, random start, 1000
equilibration + 1000 measured sweeps per seed (the small workload).  Each
precision runs 12 independent seeds; the per-seed means are independent, so
their spread gives the standard error.  FP32 and FP16 (binary16 storage,
renormalised trial) must agree with FP64 on <E>/N, <|M|> and <|M_z|> within
3 sigma of the difference.  The FP64 path itself is pinned element by element
to the oracle elsewhere; here the oracle's role is played by that path.
"""
import math

import numpy as np
import pytest

from paper_2106_11286_gb300 import hs

pytestmark = pytest.mark.gpu

DIMS = (16, 16, 16)
N = 16 ** 3


def run(precision, seed):
    with hs.Lattice("sc", dims=DIMS, J=1.0, K=0.1, e=(0, 0, 1), precision=precision, seed=seed) as lat:
        lat.init()
        lat.sweep(1.0, 1000)
        lat.accumulate(True)
        lat.reset_accumulator()
        lat.sweep(1.0, 1000)
        mom, cnt = lat.read_accumulator()
        spins = lat.get_spins()
    return np.array([mom[hs.MOMENTS.index("sum_E")] / cnt / N, mom[hs.MOMENTS.index("sum_absM")] / cnt,
                     mom[hs.MOMENTS.index("sum_absMe")] / cnt]), spins


@pytest.fixture(scope="module")
def results():
    out = {}
    for precision in ("fp64", "fp32", "fp16"):
        vals, norms = [], []
        for seed in range(100, 112):
            v, S = run(precision, seed)
            vals.append(v)
            norms.append(np.abs(np.linalg.norm(S, axis=1) - 1).max())
        out[precision] = (np.array(vals), max(norms))
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_within_three_sigma_of_fp64(results, precision):
    ref, _ = results["fp64"]
    got, _ = results[precision]
    for k, name in enumerate(("E/N", "|M|", "|M_z|")):
        a, b = got[:, k], ref[:, k]
        diff = a.mean() - b.mean()
        sigma = math.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b))
        assert abs(diff) < 3 * sigma, (precision, name, a.mean(), b.mean(), sigma)


def test_spin_norm_error_per_precision(results):
    # |S| = 1 is kept by every update: FP64 to rounding, FP32 to the hardware
    # sine/cosine error, FP16 to one binary16 step
    assert results["fp64"][1] < 1e-14
    assert results["fp32"][1] < 3e-6
    assert results["fp16"][1] < 1.5e-3
