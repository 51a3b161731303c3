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


def _handle_reference(dims, beta, seed, replica, params):
    """The handle path from its seeded start: spins, moments, sweep count and
    accepted moves after 5 sweeps, then after 4 more (accumulator reset)."""
    n = dims[0] * dims[1] * dims[2]
    with hs.Lattice("sc", dims=dims, precision="fp32", seed=seed, replica=replica, **params) as lat:
        lat.init()
        S0 = lat.get_spins()
        lat.accumulate(True)
        out = []
        for k in (5, 4):
            lat.reset_accumulator()
            lat.sweep(beta, k)
            m, c = lat.read_accumulator()
            out.append((lat.get_spins(), m, c, lat.measure()["accept_rate"] * k * n))
    return S0, out


# (32, 16, 12): Lx/2 = 16, vector width 4, split prefetch;
# (12, 4, 4): Lx/2 = 6, width 2; (10, 8, 6): Lx/2 = 5, width 1
@pytest.mark.parametrize("dims", [(32, 16, 12), (12, 4, 4), (10, 8, 6)])
def test_noalloc_two_calls_match_the_handle_path(dims):
    torch = pytest.importorskip("torch")
    beta, seed, replica = 0.9, 7, 3
    params = dict(J=1.0, K=0.1, e=(0.0, 0.0, 1.0))
    S0, ref = _handle_reference(dims, beta, seed, replica, params)
    planes = torch.tensor(to_planes(S0, dims), dtype=torch.float32, device="cuda").reshape(-1)
    out = torch.full((hs.HS_N_MOMENTS + 2,), -1.0, dtype=torch.float64, device="cuda")

    first = 0
    for call, (k, (S_want, m_want, c_want, acc_want)) in enumerate(zip((5, 4), ref)):
        if call == 1:
            # the defining property: the second call (the module and the
            # scratch address are set up by now) takes no device memory
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            stats0 = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
        # the second call continues the chain; the scratch still holds the
        # first call's contents, which must not leak into the result
        hs.hs_sweep_sc_fp32_noalloc(planes, dims, beta, k, out, seed=seed, replica=replica, first_sweep=first,
                                    **params)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free0
            assert (torch.cuda.memory_allocated(), torch.cuda.memory_reserved()) == stats0
        first += k
        got = out.cpu().numpy()
        assert np.array_equal(from_planes(planes.cpu().numpy(), dims), S_want)
        np.testing.assert_allclose(got[:hs.HS_N_MOMENTS], m_want, rtol=2e-6)
        assert got[hs.HS_N_MOMENTS] == c_want == k
        assert got[hs.HS_N_MOMENTS + 1] == pytest.approx(acc_want, abs=0.5)


def test_noalloc_rejects_misaligned_and_mismatched_buffers():
    torch = pytest.importorskip("torch")
    dims = (32, 16, 12)   # vector width 4: planes must start on 16 bytes
    want = 6 * 12 * 16 * 16
    buf = torch.zeros(want + 4, dtype=torch.float32, device="cuda")
    out = torch.full((hs.HS_N_MOMENTS + 2,), -1.0, dtype=torch.float64, device="cuda")
    planes = buf[1:want + 1]          # contiguous view, 4 bytes past the boundary
    with pytest.raises(hs.HSError) as ei:
        hs.hs_sweep_sc_fp32_noalloc(planes, dims, 1.0, 1, out)
    assert ei.value.code == -1 and "aligned" in str(ei.value)
    torch.cuda.synchronize()
    assert (out.cpu() == -1.0).all() and (buf.cpu() == 0).all()   # nothing was launched
    # the binding refuses wrong dtype, size or a short result buffer before the call
    with pytest.raises(ValueError):
        hs.hs_sweep_sc_fp32_noalloc(buf[:want].half(), dims, 1.0, 1, out)
    with pytest.raises(ValueError):
        hs.hs_sweep_sc_fp32_noalloc(buf[:want - 4], dims, 1.0, 1, out)
    with pytest.raises(ValueError):
        hs.hs_sweep_sc_fp32_noalloc(buf[:want], dims, 1.0, 1, out[:hs.HS_N_MOMENTS])
    with pytest.raises(ValueError):
        hs.hs_sweep_sc_fp32_noalloc(buf[:want], dims, 1.0, 1, out.float())


def test_noalloc_rejects_bad_sizes():
    torch = pytest.importorskip("torch")
    planes = torch.zeros(6 * 4 * 4 * 2, dtype=torch.float32, device="cuda")
    out = torch.zeros(hs.HS_N_MOMENTS + 2, dtype=torch.float64, device="cuda")
    with pytest.raises(hs.HSError) as ei:
        hs.hs_sweep_sc_fp32_noalloc(planes, (5, 4, 4), 1.0, 1, out)
    assert ei.value.code == -1 and "even" in str(ei.value)
    with pytest.raises(hs.HSError):
        hs.hs_sweep_sc_fp32_noalloc(planes, (4, 4, 4), -1.0, 1, out)
