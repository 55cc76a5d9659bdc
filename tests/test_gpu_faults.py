"""Failure detection on the GPU without a GPU fault: the device-side bounded
wait gives up, reports BATS_ERR_TIMEOUT through the handle's error word, and
the context and handle stay usable (the stage kernel's bulk-copy waits use the
same wait)."""
import time

import numpy as np
import pytest

from paper_2501_06717_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2501_06717_gb300 import bats
    bats.lib()
    return bats


def test_bounded_wait_reports_a_timeout_and_the_handle_recovers(B):
    q = W.blast()
    with B.Solver(q, precision=B.BATS_MIXED) as s:
        s.set_state(0, q.U0)
        t0 = time.time()
        with pytest.raises(B.BatsError) as e:
            B.bats_debug_wait_timeout(s.h)
        waited = time.time() - t0
        assert e.value.code == B.BATS_ERR_TIMEOUT, str(e.value)
        assert 0.5 < waited < 60, waited
        # the next step runs normally and gives the result of a fresh handle
        s.step(3, 0.8)
        U = s.get_state(0)
    with B.Solver(q, precision=B.BATS_MIXED) as s:
        s.set_state(0, q.U0)
        s.step(3, 0.8)
        assert np.array_equal(U, s.get_state(0))
