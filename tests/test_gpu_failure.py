"""Failure detection without a GPU fault.

Every device-side wait of the library (the staged kernel's mbarrier waits,
the batched kernel's grid barrier, the wavefront kernel's dependency and
mbarrier waits) is bounded.  The test hooks make one wait run out -- bytes
that never arrive, a CTA that never arrives, a unit never counted -- and the host
must then read HS_E_TIMEOUT from the next synchronising call, with the CUDA
context still usable (the same lattice keeps working afterwards).
"""
import time

import numpy as np
import pytest

from paper_2106_11286_gb300 import hs

pytestmark = pytest.mark.gpu


def test_staged_wait_timeout_is_reported_and_recoverable():
    with hs.Lattice("sc", dims=(16, 16, 8), K=0.1, precision="fp32", seed=1) as lat:
        lat.set_launch(kernel="staged")
        lat.init()
        hs.hs_lattice_inject_timeout(lat.h, True)
        t0 = time.time()
        lat.sweep(1.0, 1)
        with pytest.raises(hs.HSError) as ei:
            lat.measure()
        assert ei.value.code == -5 and time.time() - t0 < 30
        # the flag is cleared and the context is usable: a clean sweep works
        lat.init()
        lat.sweep(1.0, 2)
        m = lat.measure()
        assert np.isfinite(m["E"]) and m["n_sites"] == 16 * 16 * 8


def test_wave_dependency_timeout_is_reported_and_recoverable():
    """The wavefront kernel: CTA 0 does not count its first finished unit, so
    the units that need that plane (and, in turn, the rest) wait until their
    bounded waits run out; the kernel returns and the error is reported."""
    with hs.Lattice("sc", dims=(16, 16, 16), K=0.1, precision="fp32", seed=1) as lat:
        lat.set_launch(kernel="wave")
        lat.init()
        hs.hs_lattice_inject_timeout(lat.h, True)
        t0 = time.time()
        lat.sweep(1.0, 3)
        with pytest.raises(hs.HSError) as ei:
            lat.measure()
        assert ei.value.code == -5 and time.time() - t0 < 30
        lat.init()
        lat.sweep(1.0, 2)
        m = lat.measure()
        assert np.isfinite(m["E"]) and m["n_sites"] == 16 ** 3
    with hs.Lattice("sc", dims=(16, 16, 16), K=0.1, precision="fp32", seed=1) as a, \
            hs.Lattice("sc", dims=(16, 16, 16), K=0.1, precision="fp32", seed=1) as b:
        a.set_launch(kernel="wave")
        for lat in (a, b):
            lat.init()
            lat.sweep(1.0, 4)
        assert np.array_equal(a.get_spins(), b.get_spins())


def test_batch_barrier_timeout_is_reported_and_recoverable():
    lats = [hs.Lattice("sc", dims=(16, 16, 16), K=0.0, precision="fp32", seed=2, replica=r) for r in range(3)]
    try:
        for m in lats:
            m.init()
        b = hs.hs_batch_create([m.h for m in lats])
        try:
            hs.hs_batch_inject_timeout(b, True)
            t0 = time.time()
            hs.hs_batch_run(b, [0.7, 0.7, 0.7], 4, 0)
            for m in lats:
                with pytest.raises(hs.HSError) as ei:
                    m.read_accumulator()
                assert ei.value.code == -5
            assert time.time() - t0 < 60
            # recovered: the next run completes and reports normally
            for m in lats:
                m.init()
                m.reset_accumulator()
            hs.hs_batch_run(b, [0.7, 0.7, 0.7], 3, 0)
            for m in lats:
                mom, cnt = m.read_accumulator()
                assert cnt == 3 and np.isfinite(mom).all()
        finally:
            hs.hs_batch_destroy(b)
    finally:
        for m in lats:
            m.close()
