"""Finite-size pin of the oracle near the sc Heisenberg critical point (K = 0).

The Binder cumulant U4 = 1 - <M^4> / (3 <M^2>^2) of Eq. 2's magnetisation is
size independent at T_c: below it U4 grows with L, above it U4 falls with L.
The paper quotes T_C / J = 1.445 for the sc lattice (Fig. 3 discussion); the
high-resolution literature value is 1.443.  On L = 4, 6, 8 the ordering of
U4 must flip between T = 1.35 and 1.55, which brackets the crossing around
T_c.  (Locating the crossing to better than a few hundredths needs far more
sweeps than the oracle affords; the GPU batched run does that.)
"""
import numpy as np


def binder(orc, L, T, n_equil, n_meas, seed):
    g = orc.lattice("sc", (L, L, L))
    S = orc.init_spins(g, seed=seed)
    m2 = np.empty(n_meas)
    for s in range(n_equil + n_meas):
        orc.sweep(g, S, J=1.0, K=0.0, e=(0, 0, 1), beta=1.0 / T, seed=seed, sweep_index=s)
        if s >= n_equil:
            m = S.sum(0) / g.n
            m2[s - n_equil] = m @ m
    return 1.0 - (m2 ** 2).mean() / (3.0 * m2.mean() ** 2)


def test_binder_ordering_flips_across_tc(orc):
    lo = [binder(orc, L, 1.35, 1000, 6000, 700 + L) for L in (4, 6, 8)]
    hi = [binder(orc, L, 1.55, 1000, 6000, 800 + L) for L in (4, 6, 8)]
    assert lo[0] < lo[1] < lo[2]
    assert hi[0] > hi[1] > hi[2]
