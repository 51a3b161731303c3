"""Pins of the oracle's on-site anisotropy tensor term -sum_i S_i^T A S_i
(the effective shape anisotropy the paper offers in place of dipolar
coupling, read as a general symmetric tensor), against what the
mathematics fixes rather than against the oracle itself:

* A = K' e e^T is the uniaxial term: the chain and the energy equal those of
  K + K' without a tensor (up to rounding, so decisions only in the band);
* A = lambda I is a constant for unit spins: the chain is unchanged and E
  shifts by exactly -lambda N;
* ground states: all spins along an eigenvector of A with eigenvalue mu give
  E = -N (J z / 2 + mu), the largest mu is the minimum, and perturbations
  raise E;
* one isolated spin samples exp(beta S^T A S) on the sphere: its averages
  match a two-dimensional quadrature, for a tensor with large off-diagonal
  entries (a dropped factor 2 or a transposed index would show);
* the sum of accepted dH equals the full-recompute energy change.
"""
import math

import numpy as np
import pytest

from paper_2106_11286_gb300 import inputs


def _rotation(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    return q * np.sign(np.diag(r))


def _tensor(eigs, seed):
    R = _rotation(seed)
    A = R @ np.diag(eigs) @ R.T
    return (A + A.T) / 2, R


def _six(A):
    return np.array([A[0, 0], A[1, 1], A[2, 2], A[0, 1], A[0, 2], A[1, 2]])


def test_uniaxial_tensor_is_the_K_term(orc):
    g = orc.lattice("sc", (8, 6, 4))
    e = np.array([0.3, -0.4, 0.866])
    e = e / np.linalg.norm(e)
    K0, K1 = 0.2, 0.35
    S_a = inputs.random_unit_spins(g.n, 3)
    S_b = S_a.copy()
    band_a = np.zeros(g.n, dtype=np.uint8)
    band_b = np.zeros(g.n, dtype=np.uint8)
    for s in range(6):
        orc.sweep(g, S_a, J=1.0, K=K0 + K1, e=e, beta=0.9, seed=4, sweep_index=s, band=1e-9, band_site=band_a)
        orc.sweep(g, S_b, J=1.0, K=K0, e=e, beta=0.9, seed=4, sweep_index=s, band=1e-9, band_site=band_b,
                  A=K1 * np.outer(e, e))
    assert band_a.sum() == 0 and band_b.sum() == 0
    np.testing.assert_allclose(S_b, S_a, atol=1e-14, rtol=0)
    Ea = orc.energy(g, S_a, J=1.0, K=K0 + K1, e=e)
    Eb = orc.energy(g, S_a, J=1.0, K=K0, e=e, A=K1 * np.outer(e, e))
    assert Eb == pytest.approx(Ea, rel=1e-13)


def test_isotropic_tensor_is_a_constant(orc):
    g = orc.lattice("bcc", (4, 4, 3))
    lam = 0.7
    S_a = inputs.random_unit_spins(g.n, 8)
    S_b = S_a.copy()
    for s in range(5):
        orc.sweep(g, S_a, J=1.0, K=0.1, e=(0, 0, 1), beta=1.1, seed=2, sweep_index=s, band=1e-9)
        orc.sweep(g, S_b, J=1.0, K=0.1, e=(0, 0, 1), beta=1.1, seed=2, sweep_index=s, band=1e-9,
                  A=lam * np.eye(3))
    np.testing.assert_allclose(S_b, S_a, atol=1e-14, rtol=0)
    E0 = orc.energy(g, S_a, J=1.0, K=0.1, e=(0, 0, 1))
    E1 = orc.energy(g, S_a, J=1.0, K=0.1, e=(0, 0, 1), A=lam * np.eye(3))
    assert E1 - E0 == pytest.approx(-lam * g.n, rel=1e-12)


@pytest.mark.parametrize("kind,dims,z", [("sc", (6, 4, 4), 6), ("bcc", (3, 3, 3), 8), ("fcc", (2, 2, 2), 12)])
def test_tensor_ground_states(orc, kind, dims, z):
    eigs = np.array([0.3, -0.1, 0.7])
    A, R = _tensor(eigs, 5)
    g = orc.lattice(kind, dims)
    J = 1.0
    for k, mu in enumerate(eigs):
        S = np.tile(R[:, k], (g.n, 1))
        assert orc.energy(g, S, J=J, K=0.0, e=(0, 0, 1), A=A) == pytest.approx(-g.n * (J * z / 2 + mu), rel=1e-12)
    # the largest eigenvalue's axis is the minimum: random tilts raise E
    S0 = np.tile(R[:, 2], (g.n, 1))
    E0 = orc.energy(g, S0, J=J, K=0.0, e=(0, 0, 1), A=A)
    rng = np.random.default_rng(1)
    for _ in range(20):
        S = S0 + 0.05 * rng.normal(size=S0.shape)
        S /= np.linalg.norm(S, axis=1)[:, None]
        assert orc.energy(g, S, J=J, K=0.0, e=(0, 0, 1), A=A) > E0


def _sphere_average(beta, A, fns, n_z=160, n_phi=320):
    """<f> under exp(beta S^T A S) on the unit sphere: Gauss-Legendre in z,
    the trapezoid rule (exact for trigonometric polynomials) in phi."""
    z, wz = np.polynomial.legendre.leggauss(n_z)
    phi = 2 * np.pi * np.arange(n_phi) / n_phi
    Z, P = np.meshgrid(z, phi, indexing="ij")
    r = np.sqrt(1 - Z * Z)
    S = np.stack([r * np.cos(P), r * np.sin(P), Z], axis=-1)
    q = np.einsum("...a,ab,...b->...", S, A, S)
    w = np.exp(beta * q) * wz[:, None]
    return [float((f(S) * w).sum() / w.sum()) for f in fns]


@pytest.mark.parametrize("beta", [1.5, 4.0])
def test_single_spin_tensor_quadrature(orc, beta):
    A = np.array([[0.1, 0.6, -0.2],
                  [0.6, -0.3, 0.4],
                  [-0.2, 0.4, 0.2]])
    n = 4000
    g = orc.csr_graph(*inputs.isolated_sites(n))
    S = orc.init_spins(g, seed=31)
    fns = [lambda S: S[..., 0] * S[..., 1], lambda S: S[..., 1] * S[..., 2],
           lambda S: np.einsum("...a,ab,...b->...", S, A, S)]
    for s in range(20):
        orc.sweep(g, S, J=1.0, K=0.0, e=(0, 0, 1), beta=beta, seed=31, sweep_index=s, A=A)
    obs = []
    for s in range(20, 220):
        orc.sweep(g, S, J=1.0, K=0.0, e=(0, 0, 1), beta=beta, seed=31, sweep_index=s, A=A)
        obs.append([f(S) for f in fns])
    obs = np.array(obs)  # (sweeps, observable, site)
    want = _sphere_average(beta, A, fns)
    for k in range(len(fns)):
        per_site = obs[:, k, :].mean(0)
        mean, err = per_site.mean(), per_site.std(ddof=1) / math.sqrt(n)
        assert abs(mean - want[k]) < 5 * err, (k, mean, want[k], err)
    # the quadrature itself: beta -> 0 gives the sphere average tr(A)/3
    assert _sphere_average(1e-9, A, fns[2:])[0] == pytest.approx(np.trace(A) / 3, abs=1e-8)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_incremental_energy_with_tensor(orc, mode):
    A, _ = _tensor(np.array([0.4, -0.2, 0.1]), 9)
    g = orc.lattice("sc", (6, 6, 6))
    S = inputs.random_unit_spins(g.n, 12)
    if mode == 2:
        S = S.astype(np.float16).astype(np.float64)
    for s in range(8):
        E0 = orc.energy(g, S, J=1.0, K=0.05, e=(0, 0, 1), A=A)
        acc, sdh, _ = orc.sweep(g, S, J=1.0, K=0.05, e=(0, 0, 1), beta=1.0, seed=5, sweep_index=s, mode=mode,
                                A=A)
        E1 = orc.energy(g, S, J=1.0, K=0.05, e=(0, 0, 1), A=A)
        assert 0 < acc < g.n
        assert E1 - E0 == pytest.approx(sdh, abs=1e-10 * g.n)


def test_tensor_site_updates_reproduce_the_sweep(orc):
    """The single-site form takes the same tensor term as the sweep."""
    A, _ = _tensor(np.array([0.5, 0.0, -0.3]), 2)
    g = orc.lattice("sc", (6, 4, 4))
    S0 = inputs.random_unit_spins(g.n, 7)
    want = S0.copy()
    orc.sweep(g, want, J=1.0, K=0.1, e=(0, 0, 1), beta=0.8, seed=3, sweep_index=2, A=A)
    got = S0.copy()
    for c in range(g.n_colours):
        sites = np.nonzero(g.colour == c)[0]
        h = np.zeros((len(sites), 3))
        for t, i in enumerate(sites):
            for j in g.col[g.row_ptr[i]:g.row_ptr[i + 1]]:
                h[t] += got[j]
        sub = got[sites].copy()
        orc.sites_update(sites, np.arange(len(sites)), np.full(len(sites), c), h, sub, J=1.0, K=0.1, e=(0, 0, 1),
                         beta=0.8, seed=3, sweep_index=2, A=A)
        got[sites] = sub
    assert np.array_equal(got, want)
