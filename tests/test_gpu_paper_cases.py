"""The paper's high-frequency limit (Sec 3.1.2) on the GPU: the oscillating lid at St 30, Kn 0.1, Gauss-Hermite
velocities, wall-refined mesh, spectral source at the new iterate.  Next to the lid the gas is collisionless, so
the lid-averaged first harmonics tend to U~ = 1/2 and tau~ = 1/sqrt(pi) (Eqs. nondim_U, nondim_tau).  The GPU
run must reproduce the oracle's harmonics and, like it, land within 2 % of both limits."""
import math

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


def _lid_case(precision):
    c = I.make_case("lid", 4, 16, kn=0.1, st=30.0, nh=1, pr=2 / 3, drive="shear", amp=0.0015, ncell_y=12,
                    vgrid="gauss_hermite", precision=precision)
    c.ynodes = I.wall_refined_nodes(12, 0.001)
    c.spectral_implicit = 1
    return c


def _lid_average(c, H1):
    """lid-averaged first harmonics of U and tau_xy (cell-width weighted over the row under the lid), relative
    to the lid's own first harmonic U_a / 2 (and p0 U_a / 2 for the stress, p0 = 1/2)"""
    dx = np.diff(c.xnodes)
    top = slice((c.ny - 1) * c.nx, c.ny * c.nx)
    U1 = np.sum(H1[1, top] * dx) / c.xnodes[-1]
    T1 = np.sum(H1[4, top] * dx) / c.xnodes[-1]
    lid1 = 0.0015 / 2
    return U1 / lid1, T1 / (0.5 * lid1)


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 2e-5)])
def test_collisionless_limits_of_the_oscillating_lid_on_gpu(hb, precision, tol):
    iters = 400
    c = _lid_case(precision)
    P = O.Problem(c)
    W, h, b = I.initial_state(c)
    O.iterate(P, W, h, b, iters)
    Ho = O.harmonics(np.stack([O.fields(P, h, b, n) for n in range(c.nt)]))[1]
    s = hb.Solver(c)
    s.iterate(iters)
    Hg = s.harmonic(0, 1)
    s.destroy()
    for f in (1, 4):                                       # U, tau_xy per cell
        assert np.max(np.abs(Hg[f] - Ho[f])) <= tol * np.max(np.abs(Ho[f])), f
    Ug, Tg = _lid_average(c, Hg)
    Uo, To = _lid_average(c, Ho)
    assert abs(Ug - Uo) <= tol * abs(Uo) and abs(Tg - To) <= tol * abs(To)
    assert abs(abs(Ug) - 0.5) < 0.02 * 0.5, Ug
    assert abs(abs(Tg) - 1 / math.sqrt(math.pi)) < 0.02 / math.sqrt(math.pi), Tg
    assert -0.15 < np.angle(Ug) < 0.0 and 0.0 < np.angle(-Tg / Ug) < 0.15
