"""GPU at the benchmark sizes, in the launch configuration the bench times (autotuned tiles, captured graphs).

* Thermal cavity 64x64 cells, 48x48 velocities, N_T = 7: one iteration from a seeded state, every element of
  W, h, b against the FP64 oracle (FP64: 1e-10 of the change + 1e-13 of the magnitude; FP32-split: 2e-5 of the
  change + 2e-7 of the magnitude, as in test_gpu_parity.py).
* Thermal cavity 128x128 cells, 64x64 velocities, N_T = 11 (about 6 GB of FP32-split state): the oracle needs
  minutes per iteration there, so properties that hold at any size are checked instead:
  - a resting gas with resting walls at T0 is a fixed point (also pinned on the oracle);
  - the cavity heated from the bottom wall is mirror-symmetric about x = 1/2 and every velocity grid used is
    symmetric, so rho, rho V, rho E are even and rho U is odd under i -> nx - 1 - i, on every level;
  - the FP32-split and FP64 paths agree on W after the same iterations.
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


def _close(got, ref, init, rel_change, rel_mag):
    tol = rel_change * np.max(np.abs(ref - init)) + rel_mag * np.max(np.abs(ref))
    err = np.max(np.abs(got - ref))
    assert err <= tol, (err, tol)


@pytest.fixture(scope="module")
def thermal64_oracle_step():
    case = I.config3(precision=0)
    init = I.initial_state(case, seed=5, amp=0.01)
    P = O.Problem(case)
    W, h, b = (a.copy() for a in init)
    O.iterate(P, W, h, b, 1)
    return init, (W, h, b)


@pytest.mark.parametrize("precision,rc,rm", [(0, 1e-10, 1e-13), (1, 2e-5, 2e-7)])
def test_thermal64_v48_nh3_one_iteration_matches_oracle(hb, thermal64_oracle_step, precision, rc, rm):
    init, ref = thermal64_oracle_step
    case = I.config3(precision=precision)
    s = hb.Solver(case)
    s.set_state(0, *init)
    s.iterate(1)
    got = s.get_state(0)
    s.destroy()
    _close(got[0], ref[0], init[0], rc, 1e-9 if precision else rm)
    _close(got[1], ref[1], init[1], rc, rm)
    _close(got[2], ref[2], init[2], rc, rm)


@pytest.mark.parametrize("precision", [0, 1])
def test_thermal128_v64_nh5_rest_is_a_fixed_point(hb, precision):
    # the sizes of the large cavity; the velocity grid spans +-6.5 so that its midpoint rule reproduces the
    # Maxwellian's moments to round-off (on +-4 the truncated tails leave a 1e-12 imbalance)
    c = I.make_case("rest128", 128, 64, kn=0.05, st=5.0, nh=5, pr=2 / 3, drive="rest", half_width=6.5,
                    precision=precision)
    s = hb.Solver(c)
    W0 = s.get_W(0)
    rc, its, res = s.iterate(3)
    W = s.get_W(0)
    s.destroy()
    tol = 1e-14 if precision == 0 else 1e-7
    assert np.max(res) < tol
    assert np.max(np.abs(W - W0)) < tol


def _mirror(W, nx, ny):
    """W[level][cell][4] mirrored about x = 1/2: cells i -> nx - 1 - i, rho U -> -rho U."""
    M = W.reshape(W.shape[0], ny, nx, 4)[:, :, ::-1, :].copy()
    M[..., 1] *= -1.0
    return M.reshape(W.shape)


@pytest.fixture(scope="module")
def thermal128_both(hb):
    out = {}
    for precision in (0, 1):
        c = I.config5(precision=precision)
        s = hb.Solver(c)
        W0 = s.get_W(0)
        s.iterate(4)
        out[precision] = (W0, s.get_W(0), c)
        s.destroy()
    return out


@pytest.mark.parametrize("precision,rc,rm", [(0, 1e-10, 1e-14), (1, 1e-4, 1e-7)])
def test_thermal128_v64_nh5_is_mirror_symmetric(thermal128_both, precision, rc, rm):
    W0, W, c = thermal128_both[precision]
    assert np.max(np.abs(W - W0)) > 1e-6           # the heated wall has moved the gas
    _close(W, _mirror(W, c.nx, c.ny), W0, rc, rm)


def test_thermal128_v64_nh5_fp32_split_tracks_fp64(thermal128_both):
    W0, W64, _ = thermal128_both[0]
    _, W32, _ = thermal128_both[1]
    _close(W32, W64, W0, 1e-4, 1e-7)
