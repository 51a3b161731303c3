"""Pins of the oracle's Metropolis sweep and measurement against physics.

Each check is fixed by the mathematics, not by the oracle itself:

* sphere sampling moments (<S_a> = 0, <S_a^2> = 1/3, |S| = 1, z and phi uniform);
* ground state E = -N (J z / 2 + K) (periodic) or -J n_bonds - K N (open), Eq. 1
  with each bond once;
* |S_i| = 1 kept by every update, and the sum of accepted dH equals the change
  of the fully recomputed energy (Metropolis step (iii) against Eq. 1);
* beta = 0: every move accepted, <E> = -K N / 3, <M^2> = 1/N,
  <M^4> = (N^2 + 2N(N-1)/3) / N^4 (Eq. 2 with independent uniform spins);
* beta -> infinity from the ground state: nothing is accepted;
* one spin with anisotropy only: <(S.e)^2> by 1-D quadrature;
* dimers: <S1.S2> = L(beta J) (Langevin function) for K = 0, and a 2-D
  quadrature (azimuth integrated with Bessel functions) for K != 0;
* open chain, K = 0: <E> = -(N-1) J L(beta J);
* M -> 1 as T -> 0 and M ~ N^-1/2 at high T.

Sensitivity: some checks are re-run on a deliberately wrong model (sign of J
flipped, anisotropy dropped) and must then fail, so a dropped term or a wrong
sign in the oracle could not pass them.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special, stats

from paper_2106_11286_gb300 import inputs


def langevin(x):
    return 1.0 / math.tanh(x) - 1.0 / x


def run_chain(orc, g, S, n_sweeps, *, J, K, e, beta, seed, mode=0, start=0, observe=None):
    out = []
    for s in range(start, start + n_sweeps):
        orc.sweep(g, S, J=J, K=K, e=e, beta=beta, seed=seed, sweep_index=s, mode=mode)
        if observe is not None:
            out.append(observe(S))
    return out


# ---------------------------------------------------------------- sampling
@pytest.mark.parametrize("mode", [0, 1])
def test_trial_and_init_sphere_moments(orc, mode):
    n = 200000
    g = orc.csr_graph(*inputs.isolated_sites(n))
    S0 = orc.init_spins(g, seed=11)
    # beta = 0 accepts every move, so the state after one sweep is the raw
    # trial orientations of the chosen random-number schedule
    S1 = S0.copy()
    acc, _, _ = orc.sweep(g, S1, J=1.0, K=0.3, e=(0, 0, 1), beta=0.0, seed=11, sweep_index=5, mode=mode)
    assert acc == n
    for S in (S0, S1):
        nrm = np.linalg.norm(S, axis=1)
        assert np.abs(nrm - 1).max() < (1e-15 if mode == 0 else 1e-15)
        m = S.mean(0)
        assert (np.abs(m) < 5 / math.sqrt(3 * n)).all()
        sq = (S ** 2).mean(0)
        assert (np.abs(sq - 1 / 3) < 5 * math.sqrt(4 / 45 / n)).all()
        assert abs((S[:, 0] * S[:, 1]).mean()) < 5 * math.sqrt(1 / 15 / n)
        assert stats.kstest(S[:, 2], "uniform", args=(-1, 2)).pvalue > 1e-4
        phi = np.arctan2(S[:, 1], S[:, 0])
        assert stats.kstest(phi, "uniform", args=(-math.pi, 2 * math.pi)).pvalue > 1e-4
    assert not np.array_equal(S0, S1)


def test_fp16_mode_stores_binary16_values(orc):
    g = orc.csr_graph(*inputs.isolated_sites(5000))
    S = orc.init_spins(g, seed=2)
    orc.sweep(g, S, J=1.0, K=0.0, e=(0, 0, 1), beta=0.0, seed=2, sweep_index=0, mode=2)
    assert np.array_equal(S.astype(np.float16).astype(np.float64), S)
    assert np.abs(np.linalg.norm(S, axis=1) - 1).max() < 2e-3


def test_init_reproducible_and_replica_dependent(orc):
    g = orc.lattice("sc", (4, 4, 4))
    a = orc.init_spins(g, seed=1, replica=0)
    b = orc.init_spins(g, seed=1, replica=0)
    c = orc.init_spins(g, seed=1, replica=1)
    d = orc.init_spins(g, seed=2, replica=0)
    assert np.array_equal(a, b)
    assert not np.allclose(a, c) and not np.allclose(a, d)


# ---------------------------------------------------------------- energy
@pytest.mark.parametrize("kind,dims", [("sc", (4, 6, 8)), ("bcc", (3, 4, 5)), ("fcc", (3, 3, 4))])
def test_ground_state_energy_periodic(orc, kind, dims):
    J, K = 1.3, 0.2
    e = np.array([1.0, 2.0, 2.0]) / 3.0
    g = orc.lattice(kind, dims, periodic=True)
    S = inputs.aligned_spins(g.n, e)
    E = orc.energy(g, S, J=J, K=K, e=e)
    assert E == pytest.approx(-g.n * (J * g.z / 2 + K), rel=1e-13)
    S[::2] *= -1  # anti-aligned half: anisotropy unchanged (quadratic in S.e)
    E2 = orc.energy(g, S, J=0.0, K=K, e=e)
    assert E2 == pytest.approx(-g.n * K, rel=1e-13)


def test_ground_state_energy_open_and_masked(orc):
    J, K = 1.0, 0.1
    row_ptr, col, mask = inputs.bcc_nanoparticle(radius=3.2, box=8, vacancy_fraction=0.1, seed=5)
    g = orc.csr_graph(row_ptr, col, mask)
    n_bonds = sum(1 for i in range(g.n) if mask[i] for j in col[row_ptr[i]:row_ptr[i + 1]]
                  if mask[j] and j > i)
    S = inputs.aligned_spins(g.n, (0, 0, 1))
    assert orc.energy(g, S, J=J, K=K, e=(0, 0, 1)) == pytest.approx(-J * n_bonds - K * int(mask.sum()), rel=1e-13)


def test_energy_brute_force_small(orc):
    """Eq. 1 summed over all ordered pairs at nearest-neighbour distance / 2."""
    g = orc.lattice("bcc", (3, 3, 3), periodic=True)
    S = inputs.random_unit_spins(g.n, 4)
    J, K, e = 0.7, -0.3, np.array([0.0, 0.6, 0.8])
    E_pairs = 0.0
    for i in range(g.n):
        for j in g.col[g.row_ptr[i]:g.row_ptr[i + 1]]:
            E_pairs += -J * S[i] @ S[j] / 2
    E_pairs += -K * ((S @ e) ** 2).sum()
    assert orc.energy(g, S, J=J, K=K, e=e) == pytest.approx(E_pairs, rel=1e-12)


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("mode", [0, 1])
def test_norm_kept_and_incremental_energy(orc, mode):
    J, K, e = 1.0, 0.1, (0, 0, 1)
    g = orc.lattice("sc", (8, 8, 8))
    S = orc.init_spins(g, seed=1)
    for s in range(20):
        E0 = orc.energy(g, S, J=J, K=K, e=e)
        acc, sdh, _ = orc.sweep(g, S, J=J, K=K, e=e, beta=1.0, seed=1, sweep_index=s, mode=mode)
        E1 = orc.energy(g, S, J=J, K=K, e=e)
        assert 0 < acc < g.n
        assert E1 - E0 == pytest.approx(sdh, abs=1e-9 * g.n)
        assert np.abs(np.linalg.norm(S, axis=1) - 1).max() < 1e-15


def test_beta_infinite_from_ground_state_rejects_everything(orc):
    g = orc.lattice("fcc", (3, 3, 3))
    e = (0.0, 0.0, 1.0)
    S = inputs.aligned_spins(g.n, e)
    S[1::3] *= -1.0  # not the ground state of J, but of K alone
    for s in range(5):
        acc, _, _ = orc.sweep(g, S, J=0.0, K=1.0, e=e, beta=1e12, seed=9, sweep_index=s)
        assert acc == 0
    S = inputs.aligned_spins(g.n, e)
    E0 = orc.energy(g, S, J=1.0, K=0.2, e=e)
    for s in range(5):
        acc, _, _ = orc.sweep(g, S, J=1.0, K=0.2, e=e, beta=1e12, seed=9, sweep_index=s)
        assert acc == 0
    assert orc.energy(g, S, J=1.0, K=0.2, e=e) == E0


def test_energy_never_rises_at_zero_temperature(orc):
    g = orc.lattice("sc", (6, 6, 6))
    S = orc.init_spins(g, seed=3)
    E = orc.energy(g, S, J=1.0, K=0.1, e=(0, 0, 1))
    for s in range(30):
        _, sdh, _ = orc.sweep(g, S, J=1.0, K=0.1, e=(0, 0, 1), beta=1e15, seed=3, sweep_index=s)
        E1 = orc.energy(g, S, J=1.0, K=0.1, e=(0, 0, 1))
        assert sdh <= 0 and E1 <= E + 1e-9
        E = E1


# ---------------------------------------------------------------- beta = 0
def test_infinite_temperature_moments(orc):
    K = 0.4
    g = orc.lattice("sc", (4, 4, 4))
    N = g.n
    S = orc.init_spins(g, seed=5)
    Es, M2s, M4s = [], [], []
    for s in range(4000):
        acc, _, _ = orc.sweep(g, S, J=1.0, K=K, e=(0, 0, 1), beta=0.0, seed=5, sweep_index=s)
        assert acc == N
        m = orc.measure(g, S, J=1.0, K=K, e=(0, 0, 1))
        Es.append(m["E"]); M2s.append(m["M2"]); M4s.append(m["M4"])
    # every sweep redraws every spin: samples are independent
    n = len(Es)
    for vals, want in ((Es, -K * N / 3), (M2s, 1 / N), (M4s, (N ** 2 + 2 * N * (N - 1) / 3) / N ** 4)):
        v = np.array(vals)
        assert abs(v.mean() - want) < 5 * v.std() / math.sqrt(n), (v.mean(), want)
    U4 = 1 - np.mean(M4s) / (3 * np.mean(M2s) ** 2)
    assert abs(U4 - (1 - (1 + 2 * (N - 1) / (3 * N)) / 3)) < 0.02


# ---------------------------------------------------------------- closed forms
def _independent_average(samples):
    """samples[t, k]: sweep t, independent system k.  Mean and its error."""
    per_system = samples.mean(0)
    return per_system.mean(), per_system.std(ddof=1) / math.sqrt(len(per_system))


@pytest.mark.parametrize("beta,K", [(1.0, 0.5), (3.0, -0.7)])
def test_single_spin_anisotropy_quadrature(orc, beta, K):
    n = 4000
    g = orc.csr_graph(*inputs.isolated_sites(n))
    e = np.array([1.0, 1.0, 1.0]) / math.sqrt(3)
    S = orc.init_spins(g, seed=21)
    run_chain(orc, g, S, 20, J=1.0, K=K, e=e, beta=beta, seed=21)
    obs = run_chain(orc, g, S, 200, J=1.0, K=K, e=e, beta=beta, seed=21, start=20,
                    observe=lambda S: (S @ e) ** 2)
    mean, err = _independent_average(np.array(obs))
    num = integrate.quad(lambda x: x * x * math.exp(beta * K * x * x), -1, 1)[0]
    den = integrate.quad(lambda x: math.exp(beta * K * x * x), -1, 1)[0]
    assert abs(mean - num / den) < 5 * err


def dimer_dot(S):
    return np.einsum("ij,ij->i", S[0::2], S[1::2])


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("beta", [0.5, 2.0])
def test_dimer_langevin(orc, beta, mode):
    npairs = 5000
    g = orc.csr_graph(*inputs.dimers(npairs))
    assert g.n_colours == 2
    S = orc.init_spins(g, seed=31)
    run_chain(orc, g, S, 20, J=1.0, K=0.0, e=(0, 0, 1), beta=beta, seed=31, mode=mode)
    obs = np.array(run_chain(orc, g, S, 200, J=1.0, K=0.0, e=(0, 0, 1), beta=beta, seed=31, start=20,
                             mode=mode, observe=dimer_dot))
    mean, err = _independent_average(obs)
    assert abs(mean - langevin(beta)) < 5 * err
    # whole distribution of x = S1.S2: density proportional to exp(beta x) on [-1, 1]
    x = obs[-1]

    def cdf(t):
        return (np.exp(beta * t) - math.exp(-beta)) / (math.exp(beta) - math.exp(-beta))
    assert stats.kstest(x, cdf).pvalue > 1e-4
    # sensitivity: the antiferromagnetic sign would give -L(beta J)
    assert abs(mean - (-langevin(beta))) > 20 * err


def dimer_quadrature(beta, J, K):
    """<S1.S2> and <(S.e)^2> of a dimer with e = z: quadrature over the two
    polar cosines a, b; the azimuth difference is integrated exactly,
    int exp(x cos p) dp = 2 pi I0(x), int cos p exp(x cos p) dp = 2 pi I1(x)."""
    def w(a, b):
        s = math.sqrt(max(0.0, (1 - a * a) * (1 - b * b)))
        return math.exp(beta * J * a * b + beta * K * (a * a + b * b)), s
    def f_z(a, b):
        wt, s = w(a, b)
        return wt * special.i0(beta * J * s)
    def f_dot(a, b):
        wt, s = w(a, b)
        return wt * (a * b * special.i0(beta * J * s) + s * special.i1(beta * J * s))
    def f_a2(a, b):
        return a * a * f_z(a, b)
    Z = integrate.dblquad(f_z, -1, 1, -1, 1, epsabs=1e-11)[0]
    dot = integrate.dblquad(f_dot, -1, 1, -1, 1, epsabs=1e-11)[0] / Z
    a2 = integrate.dblquad(f_a2, -1, 1, -1, 1, epsabs=1e-11)[0] / Z
    return dot, a2


def test_dimer_with_anisotropy_quadrature(orc):
    beta, J, K = 1.5, 1.0, 0.8
    npairs = 5000
    g = orc.csr_graph(*inputs.dimers(npairs))
    S = orc.init_spins(g, seed=41)
    e = (0, 0, 1)
    run_chain(orc, g, S, 30, J=J, K=K, e=e, beta=beta, seed=41)
    obs = run_chain(orc, g, S, 250, J=J, K=K, e=e, beta=beta, seed=41, start=30,
                    observe=lambda S: (dimer_dot(S), S[:, 2] ** 2))
    dots = np.array([o[0] for o in obs])
    a2s = np.array([o[1] for o in obs])
    want_dot, want_a2 = dimer_quadrature(beta, J, K)
    m, err = _independent_average(dots)
    assert abs(m - want_dot) < 5 * err
    m2, err2 = _independent_average(a2s)
    assert abs(m2 - want_a2) < 5 * err2
    # sensitivity: dropping the anisotropy term moves <(S.e)^2> away from 1/3 ...
    assert abs(want_a2 - 1 / 3) > 20 * err2
    # ... and the K = 0 quadrature reproduces the Langevin function
    assert dimer_quadrature(beta, J, 0.0)[0] == pytest.approx(langevin(beta * J), rel=1e-7)


def test_open_chain_energy(orc):
    n, beta, J = 64, 1.2, 1.0
    chains = 40
    # many independent chains in one graph: block-diagonal CSR
    rp, cl = inputs.open_chain(n)
    row_ptr = np.concatenate([[0]] + [rp[1:] + k * rp[-1] for k in range(chains)]).astype(np.int64)
    col = np.concatenate([cl + k * n for k in range(chains)]).astype(np.int32)
    g = orc.csr_graph(row_ptr, col)
    assert g.n_colours == 2
    S = orc.init_spins(g, seed=51)
    run_chain(orc, g, S, 50, J=J, K=0.0, e=(0, 0, 1), beta=beta, seed=51)

    def chain_E(S):
        d = np.einsum("ij,ij->i", S[:-1], S[1:]).reshape(-1)
        keep = np.ones(len(d), dtype=bool)
        keep[n - 1::n] = False  # pairs that straddle two chains
        return -J * d[keep].reshape(chains, n - 1).sum(1)
    obs = np.array(run_chain(orc, g, S, 400, J=J, K=0.0, e=(0, 0, 1), beta=beta, seed=51, start=50,
                             observe=chain_E))
    E_full = [orc.energy(g, S, J=J, K=0.0, e=(0, 0, 1))]
    assert E_full[0] == pytest.approx(obs[-1].sum(), rel=1e-12)
    mean, err = _independent_average(obs)
    assert abs(mean - (-(n - 1) * J * langevin(beta * J))) < 5 * err


def test_low_and_high_temperature_limits(orc):
    g = orc.lattice("sc", (6, 6, 6))
    e = (0, 0, 1)
    S = inputs.aligned_spins(g.n, e)
    obs = run_chain(orc, g, S, 100, J=1.0, K=0.1, e=e, beta=20.0, seed=61,
                    observe=lambda S: orc.measure(g, S, J=1.0, K=0.1, e=e)["absM"])
    assert np.mean(obs[20:]) > 0.97
    S = orc.init_spins(g, seed=61)
    obs = run_chain(orc, g, S, 300, J=1.0, K=0.1, e=e, beta=0.05, seed=61,
                    observe=lambda S: orc.measure(g, S, J=1.0, K=0.1, e=e)["M2"])
    # high T: M^2 of order 1/N (weakly enhanced by the residual coupling)
    assert np.mean(obs[50:]) < 2.0 / g.n


@pytest.mark.parametrize("kind,dims", [("sc", (8, 6, 4)), ("fcc", (3, 3, 2))])
def test_fp32_schedule_gives_every_site_its_own_numbers(orc, kind, dims):
    """The FP32 schedule shares a Philox block between two sites of a colour
    (rank >> 1, halves rank & 1): no two sites may receive the same trial."""
    g = orc.lattice(kind, dims)
    S = orc.init_spins(g, seed=4)
    acc, _, _ = orc.sweep(g, S, J=1.0, K=0.0, e=(0, 0, 1), beta=0.0, seed=4, sweep_index=2, mode=1)
    assert acc == g.n
    assert len(np.unique(S, axis=0)) == g.n
    # and a second sweep draws fresh numbers
    S2 = S.copy()
    orc.sweep(g, S2, J=1.0, K=0.0, e=(0, 0, 1), beta=0.0, seed=4, sweep_index=3, mode=1)
    assert not np.any(np.all(S2 == S, axis=1))
