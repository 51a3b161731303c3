"""Failure detection without a GPU fault.

The one device-side wait of the library, the batched kernel's grid barrier
between colour passes, is bounded.  The test hook makes it run out -- one CTA
never arrives -- and the host must then read HS_E_TIMEOUT from the next
synchronising call on every member, with the CUDA context still usable (the
same batch keeps working afterwards).
"""
import time

import numpy as np
import pytest

from paper_2106_11286_gb300 import hs

pytestmark = pytest.mark.gpu


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
