"""The device-side pseudo-time loop (a CUDA graph whose conditional while node repeats one iteration and a
loop test) against the host-polled graphs of 16 iterations: the same kernels, bitwise the same states, the same
stopping rule (iteration budget, convergence of every case, divergence)."""
import numpy as np
import pytest

from paper_2605_03479_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    from paper_2605_03479_gb300 import build, hbugks
    build.build()
    return hbugks


def _batch(precision):
    return [I.make_case("l0", 6, 8, kn=0.1, st=1.0, nh=1, pr=2 / 3, drive="shear", precision=precision),
            I.make_case("l1", 9, 10, kn=1.0, st=0.3, nh=2, pr=2 / 3, drive="thermal", amp=0.4, ncell_y=5,
                        precision=precision)]


@pytest.mark.parametrize("precision", [0, 1])
def test_device_loop_equals_host_loop(hb, precision):
    out = []
    for mode in (0, 1):
        cases = _batch(precision)
        s = hb.Solver(cases)
        s.set_loop_mode(mode)
        for k, c in enumerate(cases):
            s.set_state(k, *I.initial_state(c, seed=20 + k))
        rc, its, res = s.iterate(37)                 # not a multiple of the host loop's 16
        s.enqueue_iterations(5)
        rc2, its2, res2 = s.iterate(3)
        out.append((rc, its.tolist(), res, rc2, its2.tolist(), res2, [s.get_state(k) for k in range(len(cases))],
                    [s.iteration_count(k) for k in range(len(cases))]))
        s.destroy()
    a, b = out
    assert a[0] == b[0] == hb.OK and a[1] == b[1] == [37, 37] and a[4] == b[4] == [3, 3]
    assert a[7] == b[7] == [45, 45]
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[5], b[5])
    for sa, sb in zip(a[6], b[6]):
        for x, y in zip(sa, sb):
            assert np.array_equal(x, y)


def test_device_loop_stops_when_every_case_converged(hb):
    cases = [I.make_case("c0", 6, 8, kn=0.5, st=1.0, nh=1, drive="shear"),
             I.make_case("c1", 5, 8, kn=1.0, st=1.0, nh=1, drive="shear", amp=0.02)]
    s = hb.Solver(cases)
    rc, its, res = s.iterate(100000, tol_rho=1e-9)
    assert rc == hb.OK
    assert np.all(res[:, 0] <= 1e-9) and np.all(its >= 10) and np.all(its < 100000)
    assert [s.iteration_count(k) for k in range(2)] == its.tolist()    # each stopped at its own iteration
    # a further call re-checks convergence after one iteration of each case
    rc, its2, _ = s.iterate(100, tol_rho=1e-9)
    assert rc == hb.OK and its2.tolist() == [1, 1]
