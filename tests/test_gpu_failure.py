"""Failure detection on the GPU without a GPU fault.

Every wait of the iteration kernels for a bulk copy is bounded by elapsed time; on expiry the kernel sets the
handle's error word, waits (bounded) for the copies its CTA issued, and exits; the later kernels of the
iteration return without work and hbugks_iterate reports HBUGKS_TIMEOUT with the state of the last completed
iteration.  The test hook makes the micro update report its first wait as expired right after that wait has
completed, so the whole path runs while every copy completes normally.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_03479_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    from paper_2605_03479_gb300 import build, hbugks
    build.build()
    return hbugks


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 2e-5)])
def test_expired_wait_is_reported_and_the_next_call_recovers(hb, precision, tol):
    c = I.make_case("to", 7, 10, kn=0.1, st=1.0, nh=2, pr=2 / 3, drive="thermal", amp=0.3, ncell_y=6,
                    precision=precision)
    W0, h0, b0 = I.initial_state(c, seed=5)
    s = hb.Solver(c)
    s.set_state(0, W0, h0, b0)
    start = s.get_state(0)                       # the set state as stored (FP32-split rounds it)
    s.test_expire_wait()
    rc, its, res = s.iterate(5)
    assert rc == hb.TIMEOUT, hb.status_string(rc)
    assert s.iteration_count(0) == 0
    for a, b in zip(s.get_state(0), start):      # the failed iteration left the state as it was
        assert np.array_equal(a, b)
    rc, its, res = s.iterate(3)                  # hook and error word cleared: three normal iterations
    assert rc == hb.OK and its[0] == 3
    got = s.get_state(0)
    P = O.Problem(c)
    W, h, b = W0.copy(), h0.copy(), b0.copy()
    O.iterate(P, W, h, b, 3)
    for g, o, i in zip(got, (W, h, b), (W0, h0, b0)):
        err = np.max(np.abs(g - o))
        assert err <= tol * np.max(np.abs(o - i)) + 2e-7 * precision * np.max(np.abs(o)) + 1e-13 * np.max(np.abs(o))
    s.destroy()


def test_expired_wait_in_enqueued_iterations_is_reported_by_the_next_iterate(hb):
    c = I.make_case("tq", 6, 8, kn=0.2, st=1.0, nh=1, pr=2 / 3, drive="shear", amp=0.02, precision=1)
    s = hb.Solver(c)
    s.test_expire_wait()
    s.enqueue_iterations(20)                     # no host check inside: the error word waits for the next call
    rc, its, res = s.iterate(4)
    assert rc == hb.TIMEOUT
    assert s.iteration_count(0) == 0
    rc, its, res = s.iterate(4)
    assert rc == hb.OK and s.iteration_count(0) == 4
    s.destroy()
