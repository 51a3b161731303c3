"""hs_set_spins_async, the pipelined upload of a whole state, against the
synchronous hs_set_spins.

* FP64 and FP32 host input store the same values as hs_set_spins of those
  values, for every precision and for the plane (sc) and neighbour-table
  (CSR, masked) layouts.
* Stream order: sweeps queued before an upload see the old state, sweeps
  queued after it the new one; a run with uploads queued behind running
  sweeps reproduces the same sequence done synchronously, bit for bit, with
  the same fused sums.
* Three uploads queued back to back (the third reusing the first buffer
  while the first conversion may still be waiting) leave the last state.
* Bad arguments are refused before anything is queued.
"""
import numpy as np
import pytest

from helpers import storage_round
from paper_2106_11286_gb300 import hs, inputs

pytestmark = pytest.mark.gpu

PARAMS = dict(J=1.0, K=0.2, e=(0.0, 0.0, 1.0))


def _lattice(kind, precision, seed=3):
    if kind == "sc":
        return hs.Lattice("sc", dims=(32, 16, 12), precision=precision, seed=seed, **PARAMS)
    rp, col, mask = inputs.bcc_nanoparticle(radius=5.0, box=12, vacancy_fraction=0.05, seed=4)
    return hs.Lattice("csr", row_ptr=rp, col_idx=col, site_mask=mask, precision=precision, seed=seed, **PARAMS)


def _n_sites(lat):
    return hs.hs_get_info(lat.h).n_sites


@pytest.mark.parametrize("kind", ["sc", "csr"])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_async_upload_stores_what_set_spins_stores(kind, precision, dtype):
    torch = pytest.importorskip("torch")
    with _lattice(kind, precision) as lat:
        n = _n_sites(lat)
        S = inputs.random_unit_spins(n, 11).astype(dtype)
        lat.set_spins(S.astype(np.float64))
        want = lat.get_spins()
        lat.init()                                   # another state in between
        host = torch.from_numpy(S.reshape(-1).copy()).pin_memory()
        lat.set_spins_async(host)
        got = lat.get_spins()                        # synchronous: the upload is done
        assert np.array_equal(got, want)
        # pageable numpy input as well
        lat.init()
        lat.set_spins_async(S.reshape(-1))
        assert np.array_equal(lat.get_spins(), want)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_uploads_queued_behind_sweeps_keep_stream_order(precision):
    torch = pytest.importorskip("torch")
    beta = 0.8
    with _lattice("sc", precision) as lat:
        n = _n_sites(lat)
        states = [storage_round(inputs.random_unit_spins(n, 20 + k), precision) for k in range(3)]
        # synchronous reference: state k, then k + 2 sweeps, sums read after each
        lat.accumulate(True)
        lat.set_sweep_counter(5)
        want = []
        for k, S in enumerate(states):
            lat.set_spins(S)
            lat.reset_accumulator()
            lat.sweep(beta, k + 2)
            want.append((lat.get_spins(), lat.read_accumulator()))
        # pipelined: the next upload is queued while the current sweeps run
        hosts = [torch.from_numpy(S.astype(np.float32 if precision != "fp64" else np.float64).reshape(-1)
                                  .copy()).pin_memory() for S in states]
        lat.set_sweep_counter(5)
        lat.set_spins_async(hosts[0])
        for k in range(3):
            lat.reset_accumulator()
            lat.sweep(beta, k + 2)
            if k + 1 < 3:
                lat.set_spins_async(hosts[k + 1])
            moments, count = lat.read_accumulator()
            S_want, (m_want, c_want) = want[k]
            assert count == c_want == k + 2
            assert np.array_equal(moments, m_want)
            if k + 1 == 3:
                assert np.array_equal(lat.get_spins(), S_want)


def test_three_uploads_in_flight_leave_the_last_state():
    torch = pytest.importorskip("torch")
    with _lattice("sc", "fp32") as lat:
        n = _n_sites(lat)
        states = [inputs.random_unit_spins(n, 40 + k).astype(np.float32) for k in range(3)]
        hosts = [torch.from_numpy(S.reshape(-1).copy()).pin_memory() for S in states]
        lat.sweep(0.5, 40)                  # work on the stream ahead of the uploads
        for h in hosts:
            lat.set_spins_async(h)
        assert np.array_equal(lat.get_spins(), states[2].astype(np.float64))


def test_async_upload_rejects_bad_arguments():
    with _lattice("sc", "fp32") as lat:
        n = _n_sites(lat)
        with pytest.raises(ValueError):
            lat.set_spins_async(np.zeros(3 * n, dtype=np.float16))
        with pytest.raises(ValueError):
            lat.set_spins_async(np.zeros(3 * n - 3, dtype=np.float32))
        with pytest.raises(ValueError):
            lat.set_spins_async(np.zeros((3 * n, 2), dtype=np.float32)[:, 0])
        buf = np.zeros(3 * n, dtype=np.float32)
        assert hs.load().hs_set_spins_async(lat.h, buf.ctypes.data, hs.HS_FP16) == -1
        assert hs.load().hs_set_spins_async(lat.h, None, hs.HS_FP32) == -1
