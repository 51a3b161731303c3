"""The allocation-free sweep entry point against the handle-based path.

hs_sweep_sc_fp32_noalloc exists for callers that cannot allocate device
memory themselves (their framework's allocator or a fixed budget owns it, or
cudaMalloc's implicit device-wide synchronisation is not acceptable in their
loop).  They pass their own device buffers for the spins and the results; the
reduction scratch lives in a static device array inside the library.  Two
calls in a row must reproduce what a lattice handle computes from the same
state with the same seed: identical spins, moments within the FP32 tolerance
the other tests use (the per-thread FP32 partial sums may group differently).
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2106_11286_gb300 import hs

pytestmark = pytest.mark.gpu


def to_planes(S, dims):
    """Natural-order (n, 3) spins -> the stencil layout: planes [colour][xyz][z][y][x/2]."""
    Lx, Ly, Lz = dims
    S = S.reshape(Lz, Ly, Lx, 3)
    z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    colour = (x + y + z) & 1
    planes = np.zeros((2, 3, Lz, Ly, Lx // 2))
    for c in (0, 1):
        m = colour == c
        for q in range(3):
            planes[c, q, z[m], y[m], x[m] // 2] = S[z[m], y[m], x[m], q]
    return planes


def from_planes(planes, dims):
    Lx, Ly, Lz = dims
    planes = planes.reshape(2, 3, Lz, Ly, Lx // 2)
    z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    colour = (x + y + z) & 1
    S = np.zeros((Lz, Ly, Lx, 3))
    for q in range(3):
        S[..., q] = planes[colour, q, z, y, x // 2]
    return S.reshape(-1, 3)


def test_noalloc_two_calls_match_the_handle_path():
    torch = pytest.importorskip("torch")
    dims = (32, 16, 12)
    beta, seed, replica = 0.9, 7, 3
    params = dict(J=1.0, K=0.1, e=(0.0, 0.0, 1.0))
    n = dims[0] * dims[1] * dims[2]
    with hs.Lattice("sc", dims=dims, precision="fp32", seed=seed, replica=replica, **params) as lat:
        lat.init()
        S0 = lat.get_spins()
        lat.accumulate(True)
        lat.sweep(beta, 5)
        S5 = lat.get_spins()
        m5, c5 = lat.read_accumulator()
        acc5 = lat.measure()["accept_rate"] * 5 * n
        lat.reset_accumulator()
        lat.sweep(beta, 4)
        S9 = lat.get_spins()
        m9, c9 = lat.read_accumulator()
        acc9 = lat.measure()["accept_rate"] * 4 * n
    planes = torch.tensor(to_planes(S0, dims), dtype=torch.float32, device="cuda").reshape(-1)
    out = torch.full((hs.HS_N_MOMENTS + 2,), -1.0, dtype=torch.float64, device="cuda")

    hs.hs_sweep_sc_fp32_noalloc(planes, dims, beta, 5, out, seed=seed, replica=replica, first_sweep=0, **params)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(from_planes(planes.cpu().numpy(), dims), S5)
    np.testing.assert_allclose(got[:hs.HS_N_MOMENTS], m5, rtol=2e-6)
    assert got[hs.HS_N_MOMENTS] == c5 == 5
    assert got[hs.HS_N_MOMENTS + 1] == pytest.approx(acc5, abs=0.5)

    # second call continues the chain; the scratch still holds the first
    # call's contents and must not leak into the result
    hs.hs_sweep_sc_fp32_noalloc(planes, dims, beta, 4, out, seed=seed, replica=replica, first_sweep=5, **params)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(from_planes(planes.cpu().numpy(), dims), S9)
    np.testing.assert_allclose(got[:hs.HS_N_MOMENTS], m9, rtol=2e-6)
    assert got[hs.HS_N_MOMENTS] == c9 == 4
    assert got[hs.HS_N_MOMENTS + 1] == pytest.approx(acc9, abs=0.5)


def test_noalloc_rejects_bad_sizes():
    torch = pytest.importorskip("torch")
    planes = torch.zeros(6 * 4 * 4 * 2, dtype=torch.float32, device="cuda")
    out = torch.zeros(hs.HS_N_MOMENTS + 2, dtype=torch.float64, device="cuda")
    with pytest.raises(hs.HSError) as ei:
        hs.hs_sweep_sc_fp32_noalloc(planes, (5, 4, 4), 1.0, 1, out)
    assert ei.value.code == -1 and "even" in str(ei.value)
    with pytest.raises(hs.HSError):
        hs.hs_sweep_sc_fp32_noalloc(planes, (4, 4, 4), -1.0, 1, out)
