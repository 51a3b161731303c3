"""The scan module's statistics on synthetic samples with known answers
(no GPU): jackknife errors, Binder cumulant limits, curve crossing, and the
log-log slope that gives beta/nu at T_c."""
import numpy as np
import pytest

from paper_2106_11286_gb300 import scan


def test_jackknife_of_the_mean_is_the_standard_error():
    x = np.random.default_rng(1).normal(3.0, 2.0, 400)
    val, err = scan.jackknife(lambda m: m, x)
    assert val == pytest.approx(x.mean())
    assert err == pytest.approx(x.std(ddof=1) / np.sqrt(len(x)), rel=1e-12)


def test_jackknife_of_a_ratio_matches_the_delta_method():
    rng = np.random.default_rng(2)
    a, b = rng.normal(4.0, 0.5, 4000), rng.normal(2.0, 0.3, 4000)
    val, err = scan.jackknife(lambda p, q: p / q, a, b)
    delta = np.sqrt((0.5 / 2.0) ** 2 + (4.0 * 0.3 / 4.0) ** 2) / np.sqrt(len(a))
    assert val == pytest.approx(2.0, abs=4 * delta)
    assert err == pytest.approx(delta, rel=0.1)


def test_binder_limits():
    # ordered phase: |M| fixed, <M^4> = <M^2>^2 -> U4 = 2/3
    assert scan.binder(0.25, 0.0625) == pytest.approx(2.0 / 3.0)
    # disordered phase: M an isotropic 3-component Gaussian, <|M|^4> / <|M|^2>^2 = 15 / 9
    M = np.random.default_rng(3).normal(size=(400000, 3))
    r2 = (M ** 2).sum(1)
    assert scan.moment_ratio(r2.mean(), (r2 ** 2).mean()) == pytest.approx(5.0 / 3.0, rel=0.01)
    assert scan.binder(r2.mean(), (r2 ** 2).mean()) == pytest.approx(4.0 / 9.0, abs=0.005)


def test_crossing_of_two_lines():
    T = np.linspace(1.0, 2.0, 11)
    u1 = 0.6 - 0.2 * (T - 1.37)
    u2 = 0.6 - 0.5 * (T - 1.37)
    assert scan.crossing(T, u1, u2) == pytest.approx(1.37, abs=1e-12)
    assert np.isnan(scan.crossing(T, u1, u1 + 1.0))


def test_log_slope_recovers_a_power_law():
    L = np.array([16, 24, 32, 48, 64])
    assert scan.log_slope(L, 0.8 * L ** -0.518) == pytest.approx(-0.518, abs=1e-12)


def test_power_law_fit_below_tc():
    T = np.array([1.0, 1.1, 1.2, 1.3, 1.4, 1.5, 1.6])
    M = np.where(T < 1.445, 1.3 * np.clip(1.445 - T, 1e-9, None) ** 0.364, 0.01)
    assert scan.power_law_exponent(T, M, 1.445) == pytest.approx(0.364, abs=1e-12)


def test_binder_crossing_of_synthetic_curves():
    """Two sizes whose U4(T) are straight lines crossing at T = 1.445; M4 is
    built from U4 with M2 fixed, samples scattered symmetrically around the
    means so the jackknife error is finite and the estimate exact."""
    temps = (1.40, 1.43, 1.46, 1.49)
    sc = scan.Scan(sizes=(8, 16), temps=temps, replicas=1, block_sweeps=1)
    rng = np.random.default_rng(0)
    for i, slope in enumerate((-1.0, -3.0)):
        for j, T in enumerate(temps):
            u = 0.60 + slope * (T - 1.445)
            m2 = 0.1
            m4 = (1 - u) * 3 * m2 * m2
            d = rng.normal(size=10) * 1e-4
            d = np.concatenate([d, -d])
            sc.M2[(i, j)] = np.full(20, m2)
            sc.M4[(i, j)] = m4 * (1 + d)
    tc, err = scan.binder_crossing(sc, 0, 1)
    assert tc == pytest.approx(1.445, abs=1e-9)
    assert 0 < err < 1e-3


def test_beta_fit_recovers_a_planted_exponent():
    """beta_fit on synthetic block means of <|M|> = B (T_c - T)^beta with a
    planted beta and T_c, noise-free and with noise; the T_c of the crossing
    branch comes from planted Binder cumulants that cross at T_c."""
    import numpy as np

    from paper_2106_11286_gb300 import scan
    rng = np.random.default_rng(5)
    temps = (1.0, 1.1, 1.2, 1.3, 1.4, 1.45, 1.5, 1.55)
    tc, beta = 1.47, 0.36
    s = scan.Scan((8, 16), temps, 1, 100)
    for i, L in enumerate((8, 16)):
        for j, T in enumerate(temps):
            m = 0.9 * max(tc - T, 1e-3) ** beta
            s.absM[(i, j)] = m * (1 + 1e-4 * rng.standard_normal(12))
            # U4 = 1 - m4 / (3 m2^2), linear in T with a slope growing with L, so
            # the two sizes cross exactly at tc (linear interpolation is exact)
            u = 0.6 + 0.01 * L * (tc - T)
            m2 = np.full(12, 0.5)
            s.M2[(i, j)] = m2
            s.M4[(i, j)] = 3 * (1 - u) * m2 ** 2
    fit = [j for j, T in enumerate(temps) if T <= 1.4]
    b, err, t = scan.beta_fit(s, 1, fit, tc=tc)
    assert b == pytest.approx(beta, abs=5e-4) and err < 1e-3
    b2, err2, t2 = scan.beta_fit(s, 1, fit, tc_sizes=(0, 1))
    assert t2 == pytest.approx(tc, abs=1e-12)
    assert b2 == pytest.approx(beta, abs=5e-4)
