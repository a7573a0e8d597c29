"""The paper's own cavity workloads (Sec 3.1.1, 3.2, 3.3) as seeded inputs, and the oracle on them.

* The wall-refined mesh: both wall cells exactly ds_min wide, symmetric about the cavity centre, monotone,
  for the 45-, 90- and 180-column cavities of aspect 0.5, 1 and 2.
* The Gauss-Hermite velocity grid: its discrete moments of the rest Maxwellian equal the closed forms
  Gamma(k + 1/2) to round-off up to the rule's exact degree, and the rest state is then a fixed point of the
  oracle's iteration without widening the grid.
* The Reynolds-number input of the continuum limit reaches the oracle's reference viscosity as U_mean / Re.
* Mirror symmetry (x -> A - x, U_a -> -U_a) of the oracle on an aspect-0.5, wall-refined, Gauss-Hermite
  cavity: exact, iteration by iteration, so the aspect and the quadrature enter every face the same way.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_03479_gb300 import inputs as I


@pytest.mark.parametrize("n,length", [(45, 0.5), (90, 1.0), (180, 2.0), (12, 1.0)])
def test_wall_refined_mesh(n, length):
    x = I.wall_refined_nodes(n, 0.001, length)
    d = np.diff(x)
    assert x[0] == 0.0 and x[-1] == length
    assert np.all(d > 0)
    assert abs(d[0] - 0.001) < 1e-12 and abs(d[-1] - 0.001) < 1e-12
    np.testing.assert_allclose(x + x[::-1], length, rtol=0, atol=1e-14)
    assert np.max(d) > length / n                 # coarser than uniform in the middle
    with pytest.raises(ValueError):
        I.wall_refined_nodes(n, 1.01 * length / n, length)


@pytest.mark.parametrize("n", [8, 16, 28])
def test_gauss_hermite_grid_moments(n):
    u, w = I.gauss_hermite_grid(n)
    np.testing.assert_allclose(u, -u[::-1], rtol=0, atol=1e-13)
    g = w * np.exp(-u * u)
    for k in range(min(n, 12)):                   # degree 2k <= 2n - 1
        exact = math.gamma(k + 0.5)
        assert abs(np.sum(g * u ** (2 * k)) - exact) < 1e-12 * exact, k
        assert abs(np.sum(g * u ** (2 * k + 1))) < 1e-12 * exact


def test_rest_is_a_fixed_point_on_a_gauss_hermite_grid():
    """Gauss-Hermite nodes integrate the rest Maxwellian's moments exactly, so no widened grid is needed for
    the rest state to stay put (on the +-4 midpoint grid the truncated tails leave a 1e-12 imbalance)."""
    c = I.make_case("rest_gh", 5, 16, kn=0.1, st=2.0, nh=2, pr=2 / 3, drive="rest", vgrid="gauss_hermite",
                    ds_min=0.02, ncell_y=4, aspect=0.5)
    P = O.Problem(c)
    W, h, b = I.initial_state(c)
    W0, h0 = W.copy(), h.copy()
    res = O.iterate(P, W, h, b, 3)
    assert np.max(res) < 1e-14
    assert np.max(np.abs(W - W0)) < 1e-14
    assert np.max(np.abs(h - h0)) < 1e-14 * np.max(h0)


@pytest.mark.parametrize("re", [100.0, 1000.0])
def test_reynolds_input_gives_the_viscosity_of_eq_def_re(re):
    c = I.continuum_case(re)
    assert abs(O.mu0_from_kn(c.kn, c.w_vss, c.alpha_vss) - 0.15 / re) < 1e-14 * (0.15 / re)
    assert c.nu == c.nv == 16 and c.walls[I.TOP][0] == 0.15 and c.walls[I.TOP][3] == 0.0015


def test_paper_workload_shapes():
    for A, nx in ((0.5, 45), (1.0, 90), (2.0, 180)):
        c = I.paper_shear_case(0.1, 30.0, A)
        assert (c.nx, c.ny, c.nu, c.nv) == (nx, 90, 28, 28)
        assert c.xnodes[-1] == A and c.umax == np.max(np.abs(c.u)) > 4.0
        assert c.walls[I.TOP][3] == 0.0015 and c.pr == 2 / 3
    c = I.paper_shear_case(1.0, 1.0)
    assert (c.nu, c.umax) == (64, 4.0)
    t = I.paper_thermal_case(0.1)
    assert (t.nx, t.nu, t.nt) == (90, 64, 5) and t.walls[I.TOP][7] == 0.3 and t.walls[I.BOTTOM][8] == 0.0


def _mirror_x(case, W, h, b):
    nt, nx, ny, nu, nv = case.nt, case.nx, case.ny, case.nu, case.nv
    W = W.reshape(nt, ny, nx, 4)[:, :, ::-1, :].copy()
    W[..., 1] *= -1.0
    h = h.reshape(nt, ny, nx, nv, nu)[:, :, ::-1, :, ::-1]
    b = b.reshape(nt, ny, nx, nv, nu)[:, :, ::-1, :, ::-1]
    return (np.ascontiguousarray(W.reshape(nt, -1, 4)), np.ascontiguousarray(h.reshape(nt, nx * ny, -1)),
            np.ascontiguousarray(b.reshape(nt, nx * ny, -1)))


def test_mirror_symmetry_of_an_aspect_half_gauss_hermite_cavity():
    def case(amp):
        return I.make_case("mirror_A0.5", 5, 12, kn=0.1, st=3.0, nh=1, pr=2 / 3, drive="shear", amp=amp,
                           ncell_y=6, aspect=0.5, ds_min=0.01, vgrid="gauss_hermite")
    cA, cB = case(0.02), case(-0.02)
    WA, hA, bA = I.initial_state(cA, seed=13)
    WB, hB, bB = _mirror_x(cA, WA, hA, bA)
    O.iterate(O.Problem(cA), WA, hA, bA, 8)
    O.iterate(O.Problem(cB), WB, hB, bB, 8)
    Wm, hm, bm = _mirror_x(cA, WA, hA, bA)
    np.testing.assert_allclose(WB, Wm, rtol=0, atol=1e-13)
    np.testing.assert_allclose(hB, hm, rtol=0, atol=1e-13 * hA.max())
    np.testing.assert_allclose(bB, bm, rtol=0, atol=1e-13 * bA.max())


def test_batch48_case_table_is_the_committed_one():
    """The 48-case batch is drawn, not stored; the committed table (tests/golden/batch48_cases.txt, written by
    tests/golden/write_batch48_cases.py) fixes the draw, so a change in numpy's PCG64 stream or in the draw
    order shows here."""
    import importlib.util
    import os
    gold = os.path.join(os.path.dirname(__file__), "golden")
    spec = importlib.util.spec_from_file_location("write_batch48_cases", os.path.join(gold, "write_batch48_cases.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(os.path.join(gold, "batch48_cases.txt")) as f:
        committed = f.read().splitlines()
    assert mod.table_lines() == committed
    cases = I.config4_cases()
    assert len(cases) == 48 and len({c.name for c in cases}) == 48
    for c in cases:
        assert 32 <= c.nx <= 96 and c.nx % 8 == 0 and c.nu in (24, 32, 40, 48) and 1 <= c.n_harmonics <= 3
        assert 0.01 <= c.kn <= 10 and 0.1 <= c.st <= 10
