"""Shared helpers of the GPU-vs-oracle parity tests (no method arithmetic)."""
import numpy as np

from paper_2106_11286_gb300 import hs


def oracle_graph(orc, kind, dims=None, periodic=True, row_ptr=None, col=None, mask=None):
    if kind == "csr":
        return orc.csr_graph(row_ptr, col, mask)
    return orc.lattice(kind, dims, periodic, mask)


def make_gpu(kind, dims=None, periodic=True, row_ptr=None, col=None, mask=None, *, J, K, e, precision, seed,
             replica=0, A=None):
    if kind == "csr":
        return hs.Lattice("csr", row_ptr=row_ptr, col_idx=col, site_mask=mask, J=J, K=K, e=e,
                          precision=precision, seed=seed, replica=replica, A=A)
    return hs.Lattice(kind, dims=dims, periodic=periodic, site_mask=mask, J=J, K=K, e=e, precision=precision,
                      seed=seed, replica=replica, A=A)


def storage_round(S, precision):
    if precision == "fp32":
        return S.astype(np.float32).astype(np.float64)
    if precision == "fp16":
        return S.astype(np.float16).astype(np.float64)
    return S.copy()


def lower_colour_neighbours(g, i):
    nb = g.col[g.row_ptr[i]:g.row_ptr[i + 1]]
    return [int(j) for j in nb if g.colour[j] < g.colour[i] and (g.mask is None or g.mask[j])]


def check_sweep_parity(g, S_prev, S_gpu, S_orc, band_site, tol):
    """Accept decisions equal except where the oracle flagged the band (or a
    lower-colour neighbour's decision differed); accepted spins within tol;
    rejected spins bit-equal to the previous state.  Returns #mismatches."""
    present = np.ones(g.n, dtype=bool) if g.mask is None else g.mask.astype(bool)
    acc_gpu = np.any(S_gpu != S_prev, axis=1) & present
    acc_orc = np.any(S_orc != S_prev, axis=1) & present
    mismatch = acc_gpu != acc_orc
    bad = []
    order = np.argsort(g.colour, kind="stable")
    for i in order[mismatch[order]]:
        if band_site[i]:
            continue
        if any(mismatch[j] for j in lower_colour_neighbours(g, i)):
            continue
        bad.append(int(i))
    assert not bad, f"accept decisions differ outside the band at sites {bad[:10]}"
    both = acc_gpu & acc_orc & ~mismatch
    if both.any():
        err = np.abs(S_gpu[both] - S_orc[both]).max()
        assert err <= tol, f"accepted spins differ by {err}"
    rej = ~acc_gpu & ~acc_orc & present
    assert np.array_equal(S_gpu[rej], S_prev[rej])
    if g.mask is not None:
        assert (S_gpu[~present] == 0).all()
    return int(mismatch.sum())
