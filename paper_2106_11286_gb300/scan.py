"""Temperature scans with the batched persistent kernel: magnetisation curves,
Binder cumulants and finite-size-scaling estimates (arXiv 2106.11286, Eq. 2
and the M(T) curves with their critical exponent and Curie temperature).

Every (size, temperature, replica) lattice of a scan is one member of a
single hs_batch; the batch equilibrates, then measures in blocks, and each
block's mean of |M|, M^2, M^4 and E/N (from the members' FP64 accumulators)
is one sample.  Statistical errors come from a jackknife over the samples
(blocks of all replicas of a point), so they account for autocorrelation
shorter than a block.

Analysis only combines measured means: no physics constant is built in.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import hs


@dataclass
class Scan:
    sizes: tuple
    temps: tuple
    replicas: int
    block_sweeps: int
    # [size index][temperature index] -> (samples,) array of block means
    absM: dict = field(default_factory=dict)
    M2: dict = field(default_factory=dict)
    M4: dict = field(default_factory=dict)
    E: dict = field(default_factory=dict)

    def samples(self, name: str, i: int, j: int) -> np.ndarray:
        return getattr(self, name)[(i, j)]


def run_scan(sizes, temps, *, n_equil: int, n_blocks: int, block_sweeps: int, replicas: int = 1, J: float = 1.0,
             K: float = 0.0, e=(0.0, 0.0, 1.0), precision: str = "fp32", seed: int = 2024, stream=None,
             init: str = "random") -> Scan:
    """Advance every (L, T, replica) sc lattice (L^3, periodic) and collect
    block means.  The lattices advance together in one hs_batch (one
    precision; L divisible by 8, or by 4 in FP64), else one after the other
    with hs_sweep, block by block: the same chains either way.  init = "random" starts from
    independent uniform spins, "aligned" from every spin along e (the ordered
    state, which reaches equilibrium below T_c without coarsening).  Returns a
    Scan whose sample arrays have n_blocks * replicas entries per (L, T)."""
    if init not in ("random", "aligned"):
        raise ValueError("init must be 'random' or 'aligned'")
    sizes, temps = tuple(int(L) for L in sizes), tuple(float(T) for T in temps)
    members, betas, where = [], [], []
    for i, L in enumerate(sizes):
        for j, T in enumerate(temps):
            for r in range(replicas):
                members.append(hs.Lattice("sc", dims=(L, L, L), J=J, K=K, e=e, precision=precision, seed=seed,
                                          replica=len(members), stream=stream))
                betas.append(1.0 / T)
                where.append((i, j))
    out = Scan(sizes, temps, replicas, block_sweeps)
    for key in set(where):
        for name in ("absM", "M2", "M4", "E"):
            getattr(out, name)[key] = []
    batch = None
    try:
        for m in members:
            m.init(hs.HS_INIT_RANDOM if init == "random" else hs.HS_INIT_ALIGNED)
        if all(L % (4 if precision == "fp64" else 8) == 0 for L in sizes):   # the batch's row rule
            batch = hs.hs_batch_create([m.h for m in members])
            if n_equil:
                hs.hs_batch_run(batch, betas, 0, n_equil)
        else:
            for m, b in zip(members, betas):
                m.sweep(b, n_equil)
                m.accumulate(True)
        for _ in range(n_blocks):
            for m in members:
                m.reset_accumulator()
            if batch is not None:
                hs.hs_batch_run(batch, betas, block_sweeps, 0)
            else:
                for m, b in zip(members, betas):
                    m.sweep(b, block_sweeps)
            for m, key in zip(members, where):
                mom, cnt = m.read_accumulator()
                n_sites = m.info.n_present
                out.absM[key].append(mom[hs.MOMENTS.index("sum_absM")] / cnt)
                out.M2[key].append(mom[hs.MOMENTS.index("sum_M2")] / cnt)
                out.M4[key].append(mom[hs.MOMENTS.index("sum_M4")] / cnt)
                out.E[key].append(mom[hs.MOMENTS.index("sum_E")] / cnt / n_sites)
    finally:
        if batch is not None:
            hs.hs_batch_destroy(batch)
        for m in members:
            m.close()
    for name in ("absM", "M2", "M4", "E"):
        d = getattr(out, name)
        for key in d:
            d[key] = np.asarray(d[key], dtype=np.float64)
    return out


# ------------------------------------------------------------------ statistics
def jackknife(estimator, *columns):
    """Delete-one jackknife of estimator(*means) over aligned sample columns.
    Returns (estimate from all samples, standard error)."""
    cols = [np.asarray(c, dtype=np.float64) for c in columns]
    n = len(cols[0])
    full = estimator(*(c.mean() for c in cols))
    if n < 2:
        return float(full), float("nan")
    tot = [c.sum() for c in cols]
    reps = np.array([estimator(*((t - c[k]) / (n - 1) for t, c in zip(tot, cols))) for k in range(n)])
    return float(full), float(np.sqrt((n - 1) / n * np.sum((reps - reps.mean()) ** 2)))


def binder(m2: float, m4: float) -> float:
    """U4 = 1 - <M^4> / (3 <M^2>^2)."""
    return 1.0 - m4 / (3.0 * m2 * m2)


def moment_ratio(m2: float, m4: float) -> float:
    """<M^4> / <M^2>^2 (the quantity U4 rescales)."""
    return m4 / (m2 * m2)


def crossing(temps, u_small, u_large) -> float:
    """Temperature where u_large - u_small changes sign from positive to
    non-positive (linear interpolation between scan points); nan if none."""
    t = np.asarray(temps, dtype=np.float64)
    d = np.asarray(u_large, dtype=np.float64) - np.asarray(u_small, dtype=np.float64)
    idx = np.nonzero((d[:-1] > 0) & (d[1:] <= 0))[0]
    if len(idx) == 0:
        return float("nan")
    k = idx[0]
    return float(t[k] + (t[k + 1] - t[k]) * d[k] / (d[k] - d[k + 1]))


def binder_crossing(scan: Scan, i_small: int, i_large: int):
    """T_c estimate from the crossing of the Binder cumulants U4(T) of sizes
    i_small and i_large (linear interpolation between scan temperatures),
    with a delete-one jackknife error over aligned samples of every (L, T)."""
    nT = len(scan.temps)
    keys = [(i, j) for i in (i_small, i_large) for j in range(nT)]
    n = min(len(scan.M2[k]) for k in keys)
    cols = []
    for k in keys:
        cols += [scan.M2[k][:n], scan.M4[k][:n]]

    def estimate(*means):
        u = [binder(means[2 * q], means[2 * q + 1]) for q in range(len(keys))]
        return crossing(scan.temps, u[:nT], u[nT:])

    return jackknife(estimate, *cols)


def log_slope(x, y) -> float:
    """Least-squares slope of log y against log x."""
    lx, ly = np.log(np.asarray(x, dtype=np.float64)), np.log(np.asarray(y, dtype=np.float64))
    A = np.vstack([lx, np.ones_like(lx)]).T
    return float(np.linalg.lstsq(A, ly, rcond=None)[0][0])


def power_law_exponent(temps, M, Tc: float) -> float:
    """The fit the paper applies to its M(T) curves: beta from
    M ~ (Tc - T)^beta, least squares of log M on log(Tc - T) over the scan
    points below Tc."""
    t = np.asarray(temps, dtype=np.float64)
    m = np.asarray(M, dtype=np.float64)
    below = t < Tc
    return log_slope(Tc - t[below], m[below])


def beta_fit(scan: Scan, i_fit: int, temps_idx, tc=None, tc_sizes=None):
    """The paper's fit of its M(T) curves: beta from <|M|> ~ (T_c - T)^beta,
    least squares of log <|M|> on log(T_c - T) over the temperatures
    temps_idx (all below T_c) of size i_fit.  T_c is either given (tc) or
    taken from the Binder-cumulant crossing of the sizes tc_sizes = (i_small,
    i_large) within the same estimate, so its error enters beta's.  Returns
    (beta, error, T_c) with a delete-one jackknife over aligned samples."""
    temps_idx = list(temps_idx)
    nT = len(scan.temps)
    cols = [scan.absM[(i_fit, j)] for j in temps_idx]
    keys = []
    if tc is None:
        if tc_sizes is None:
            raise ValueError("give tc or tc_sizes")
        keys = [(i, j) for i in tc_sizes for j in range(nT)]
        for k in keys:
            cols += [scan.M2[k], scan.M4[k]]
    n = min(len(c) for c in cols)
    cols = [c[:n] for c in cols]
    t_fit = np.asarray([scan.temps[j] for j in temps_idx])
    nf = len(temps_idx)

    def t_c(means):
        if tc is not None:
            return float(tc)
        u = [binder(means[nf + 2 * q], means[nf + 2 * q + 1]) for q in range(len(keys))]
        return crossing(scan.temps, u[:nT], u[nT:])

    def estimate(*means):
        T_c = t_c(means)
        if not np.isfinite(T_c) or np.any(t_fit >= T_c):
            return float("nan")
        return log_slope(T_c - t_fit, np.asarray(means[:nf]))

    b, err = jackknife(estimate, *cols)
    T_c, _ = jackknife(lambda *m: t_c(m), *cols)
    return b, err, T_c


def fss_exponent(scan: Scan, j: int, sizes_idx=None):
    """-d log<|M|> / d log L at temperature index j (at T_c this is beta/nu),
    with a jackknife error over aligned samples of all sizes."""
    idx = list(range(len(scan.sizes))) if sizes_idx is None else list(sizes_idx)
    Ls = [scan.sizes[i] for i in idx]
    cols = [scan.absM[(i, j)] for i in idx]
    n = min(len(c) for c in cols)
    cols = [c[:n] for c in cols]
    return jackknife(lambda *m: -log_slope(Ls, m), *cols)
