"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same seeded inputs.

Tolerances:
  * FP64 path: every element of W, h, b within 1e-10 relative, measured against the size of the change the
    iterations made (|gpu - oracle| <= 1e-10 max|oracle - initial| + 1e-13 max|oracle|).  Both sides are FP64
    and differ only in summation order and the delta-form algebra (observed about 1e-14).
  * FP32-split path: h, b, W within 2e-5 of the change plus 2e-7 of the magnitude after a few iterations: the
    per-velocity arithmetic is FP32 on delta = h - H_ref, rounding 6e-8 relative to delta, accumulated over
    a few iterations and the flux stencil; macroscopic fields per harmonic within 1e-5 relative at
    convergence (test_gpu_convergence.py).
Edge cases: ragged tiles, a single cell, a one-cell column or row, N_H = 0 and the largest N_H = 7, odd
velocity grids with zero nodes, the harmonic-mean face step; and the paper's own workload ingredients:
Gauss-Hermite grids, wall-refined meshes, aspect ratios 0.5 and 2, a lid with a mean velocity.
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


def run_both(hb, case, niter, seed=3, amp=0.01):
    W0, h0, b0 = I.initial_state(case, seed=seed, amp=amp)
    s = hb.Solver(case)
    s.set_state(0, W0, h0, b0)
    rc, its, res_g = s.iterate(niter)
    Wg, hg, bg = s.get_state(0)
    P = O.Problem(case)
    W, h, b = W0.copy(), h0.copy(), b0.copy()
    res_o = O.iterate(P, W, h, b, niter)
    s.destroy()
    return (W0, h0, b0), (Wg, hg, bg), (W, h, b), res_g, res_o


def close(got, ref, init, rel_change, rel_mag):
    tol = rel_change * np.max(np.abs(ref - init)) + rel_mag * np.max(np.abs(ref))
    err = np.max(np.abs(got - ref))
    assert err <= tol, (err, tol, np.max(np.abs(ref - init)))
    return err


CASES_FP64 = [
    # (name, case factory, iterations) -- sizes span several velocity blocks with a ragged tail
    ("shear_bgk_9x7_v10", lambda: I.make_case("a", 9, 10, kn=0.1, st=1.0, nh=1, pr=1.0, drive="shear",
                                               ncell_y=7), 10),
    ("shear_shakhov_stretched", lambda: I.make_case("b", 8, 12, kn=0.05, st=2.0, nh=1, pr=2 / 3,
                                                    stretched_ratio=1.1, drive="shear", amp=0.02), 10),
    ("thermal_nh2_kn1", lambda: I.make_case("c", 7, 8, kn=1.0, st=0.5, nh=2, pr=2 / 3, drive="thermal",
                                            amp=0.5, nvel_y=10), 6),
    ("thermal_nh3_kn001", lambda: I.make_case("d", 6, 8, kn=0.01, st=3.0, nh=3, pr=2 / 3, drive="thermal",
                                              amp=0.3), 5),
    ("nh0_steady_lid", lambda: I.make_case("e", 6, 9, kn=0.3, st=1.0, nh=0, pr=2 / 3, drive="shear"), 8),
    ("one_cell_row", lambda: I.make_case("f", 5, 8, kn=0.2, st=1.0, nh=1, pr=2 / 3, drive="shear",
                                         ncell_y=1), 6),
    ("harmonic_face_step", lambda: _with(I.make_case("g", 6, 8, kn=0.1, st=1.0, nh=1, pr=2 / 3,
                                                     stretched_ratio=1.1, drive="shear"), face_step=1), 6),
    # odd grids: the nodes u = 0 and v = 0 (ties at every face, parallel to every wall) are stored in two sign
    # classes with half weight each, (0, 0) in four with a quarter
    ("zero_velocity_nodes", lambda: I.make_case("z", 7, 9, kn=0.2, st=1.0, nh=1, pr=2 / 3, drive="thermal",
                                                amp=0.3, nvel_y=11, ncell_y=6), 6),
    ("max_levels_nh7", lambda: I.make_case("m", 5, 8, kn=0.1, st=2.0, nh=7, pr=2 / 3, drive="thermal",
                                           amp=0.3, ncell_y=4), 4),
    ("single_cell", lambda: I.make_case("s", 1, 10, kn=0.5, st=1.0, nh=2, pr=2 / 3, drive="shear", amp=0.05), 6),
    ("one_cell_column", lambda: I.make_case("k", 1, 8, kn=0.2, st=1.0, nh=1, pr=2 / 3, drive="thermal",
                                            amp=0.3, ncell_y=5), 6),
]


# the paper's own workload ingredients (Sec 3): Gauss-Hermite velocities with nodes past +-4, wall-refined
# meshes, aspect ratios 0.5 and 2, a lid with a mean velocity (continuum limit), the heated top wall
CASES_PAPER = [
    ("paper_gauss_hermite_aspect_half", lambda: I.make_case("p", 5, 12, kn=0.1, st=3.0, nh=1, pr=2 / 3,
                                                            drive="shear", amp=0.02, ncell_y=9, aspect=0.5,
                                                            ds_min=0.01, vgrid="gauss_hermite"), 6),
    ("paper_continuum_lid_aspect_two", lambda: I.make_case("q", 10, 16, kn=I.kn_from_reynolds(100.0, 0.15),
                                                           st=1.0, nh=1, pr=2 / 3, drive="shear", amp=0.0015,
                                                           lid_mean=0.15, ncell_y=5, aspect=2.0, ds_min=0.02), 6),
    ("paper_thermal_top_gauss_hermite", lambda: I.make_case("r", 6, 14, kn=0.05, st=2.0, nh=2, pr=2 / 3,
                                                            drive="thermal_top", amp=0.3, ds_min=0.02,
                                                            vgrid="gauss_hermite"), 5),
]


def _with(case, **kw):
    for k, v in kw.items():
        setattr(case, k, v)
    return case


@pytest.mark.parametrize("name,factory,niter", CASES_FP64 + CASES_PAPER, ids=[c[0] for c in CASES_FP64 + CASES_PAPER])
def test_fp64_matches_oracle(hb, name, factory, niter):
    case = factory()
    init, g, o, res_g, res_o = run_both(hb, case, niter)
    for k in range(3):
        close(g[k], o[k], init[k], 1e-10, 1e-13)
    np.testing.assert_allclose(res_g[0], res_o[-1], rtol=1e-8, atol=1e-16)


def test_fp64_config1_size_matches_oracle(hb):
    """Shear cavity at the full size of the first benchmark configuration (32x32, 24x24, N_H = 1)."""
    case = I.config1()
    init, g, o, res_g, res_o = run_both(hb, case, 3, seed=1)
    for k in range(3):
        close(g[k], o[k], init[k], 1e-10, 1e-13)


@pytest.mark.parametrize("name,factory,niter", CASES_FP64[:4] + CASES_PAPER,
                         ids=[c[0] for c in CASES_FP64[:4] + CASES_PAPER])
def test_fp32_split_matches_oracle(hb, name, factory, niter):
    case = factory()
    case.precision = 1
    init, g, o, res_g, res_o = run_both(hb, case, niter)
    close(g[0], o[0], init[0], 2e-5, 2e-9)
    close(g[1], o[1], init[1], 2e-5, 2e-7)
    close(g[2], o[2], init[2], 2e-5, 2e-7)


@pytest.mark.parametrize("precision", [0, 1])
def test_rest_state_is_a_fixed_point_on_gpu(hb, precision):
    c = I.make_case("rest", 7, 32, kn=0.05, st=4.0, nh=2, pr=2 / 3, drive="rest", half_width=6.5,
                    stretched_ratio=1.1, precision=precision)
    s = hb.Solver(c)
    W0, h0, b0 = s.get_state(0)
    rc, its, res = s.iterate(5)
    W, h, b = s.get_state(0)
    tol = 1e-14 if precision == 0 else 1e-7
    assert np.max(res) < tol
    assert np.max(np.abs(W - W0)) < tol
    assert np.max(np.abs(h - h0)) < tol * np.max(h0)


def test_batch_equals_single_cases(hb):
    """Uneven cases in one handle give bitwise the results of each case run alone."""
    cases = [I.make_case("b0", 6, 8, kn=0.1, st=1.0, nh=1, pr=2 / 3, drive="shear"),
             I.make_case("b1", 9, 10, kn=1.0, st=0.3, nh=2, pr=2 / 3, drive="thermal", amp=0.4, ncell_y=5),
             I.make_case("b2", 5, 12, kn=0.02, st=3.0, nh=3, pr=1.0, drive="shear", amp=0.05)]
    for prec in (0, 1):
        for c in cases:
            c.precision = prec
        batch = hb.Solver(cases)
        states = [I.initial_state(c, seed=10 + k) for k, c in enumerate(cases)]
        for k, st in enumerate(states):
            batch.set_state(k, *st)
        batch.iterate(7)
        for k, c in enumerate(cases):
            one = hb.Solver(c)
            one.set_state(0, *states[k])
            one.iterate(7)
            for a, b in zip(batch.get_state(k), one.get_state(0)):
                assert np.array_equal(a, b)
            one.destroy()
        batch.destroy()


def test_checkpoint_resume_is_bitwise(hb):
    c = I.make_case("ck", 7, 10, kn=0.1, st=2.0, nh=2, pr=2 / 3, drive="thermal", amp=0.3, precision=1)
    s = hb.Solver(c)
    s.set_state(0, *I.initial_state(c, seed=4))
    s.iterate(6)
    mid = s.get_state(0)
    s.iterate(6)
    full = s.get_state(0)
    s2 = hb.Solver(c)
    s2.set_state(0, *mid)
    s2.iterate(6)
    for a, b in zip(full, s2.get_state(0)):
        assert np.array_equal(a, b)


def test_fields_and_harmonics_match_oracle(hb):
    c = I.make_case("fh", 6, 10, kn=0.2, st=1.0, nh=2, pr=2 / 3, drive="thermal", amp=0.3)
    init, g, o, _, _ = run_both(hb, c, 4)
    s = hb.Solver(c)
    s.set_state(0, *g)
    P = O.Problem(c)
    lv = []
    for n in range(c.nt):
        fo = O.fields(P, o[1], o[2], n)
        lv.append(fo)
        np.testing.assert_allclose(s.level_fields(0, n), fo, rtol=1e-9, atol=1e-12)
    H = O.harmonics(np.stack(lv))
    for k in range(c.n_harmonics + 1):
        np.testing.assert_allclose(s.harmonic(0, k), H[k], rtol=1e-9, atol=1e-12)


def test_nan_input_is_reported_as_diverged(hb):
    c = I.make_case("nan", 5, 8, kn=0.1, st=1.0, nh=1, drive="shear")
    s = hb.Solver(c)
    W, h, b = I.initial_state(c, seed=2)
    h[1, 7, 5] = np.nan
    s.set_state(0, W, h, b)
    rc, its, res = s.iterate(50)
    assert rc == hb.DIVERGED
    assert its[0] < 50


def test_iterate_to_residual_stops_and_reports(hb):
    c = I.make_case("conv", 6, 8, kn=0.5, st=1.0, nh=1, drive="shear")
    s = hb.Solver(c)
    rc, its, res = s.iterate(20000, tol_rho=1e-9)
    assert rc == hb.OK, (rc, its, res)
    assert res[0, 0] <= 1e-9 and its[0] >= 10
    hist = s.residual_history(0, 5)
    assert hist[-1, 0] == res[0, 0]


# spectral source at the new pseudo-time iterate (hbugks_physics.spectral_implicit = 1) against the oracle's
# same option: the macro update solves (I + dG omega E) across levels per cell, the micro update applies the
# inverse of diag(D) + dG omega E per cell to every velocity
IMPLICIT = [CASES_FP64[0], CASES_FP64[2], CASES_FP64[3], CASES_FP64[-4], CASES_FP64[-3]]


@pytest.mark.parametrize("name,factory,niter", IMPLICIT, ids=[c[0] for c in IMPLICIT])
@pytest.mark.parametrize("precision", [0, 1])
def test_implicit_spectral_matches_oracle(hb, name, factory, niter, precision):
    case = factory()
    case.spectral_implicit = 1
    case.precision = precision
    init, g, o, res_g, res_o = run_both(hb, case, niter)
    if precision == 0:
        for k in range(3):
            close(g[k], o[k], init[k], 1e-10, 1e-13)
    else:
        close(g[0], o[0], init[0], 2e-5, 2e-9)
        close(g[1], o[1], init[1], 2e-5, 2e-7)
        close(g[2], o[2], init[2], 2e-5, 2e-7)


# The configuration of the large thermal benchmark (64 x 64 midpoint velocities on [-4, 4], N_H = 5, Kn 0.05,
# St 5, Pr 2/3, bottom wall T0 (1 + 0.5 sin wt)) on a 16 x 16 mesh: four interior tiles of 4 x 4 cells (the
# paired first pass), wall and corner tiles, every spectral offset d = 1..5, from a seeded state.  Each precision
# runs with pinned micro-update variants (FP64 needs the smaller tiles at N_T = 11 for shared memory; FP32-split
# also runs the two-block 4 x 2 variant that the autotuner picks for the 128 x 128 benchmark).
_ORACLE_CACHE = {}


def _bench_grid_case():
    return I.make_case("bench_grid16", 16, 64, kn=0.05, st=5.0, nh=5, pr=2 / 3, drive="thermal", amp=0.5)


def _oracle_run(key, case, niter, seed):
    if key not in _ORACLE_CACHE:
        W0, h0, b0 = I.initial_state(case, seed=seed)
        P = O.Problem(case)
        W, h, b = W0.copy(), h0.copy(), b0.copy()
        res = O.iterate(P, W, h, b, niter)
        _ORACLE_CACHE[key] = ((W0, h0, b0), (W, h, b), res)
    return _ORACLE_CACHE[key]


@pytest.mark.parametrize("precision,variant", [(0, (4, 2, 1)), (0, (2, 2, 1)), (1, (4, 4, 1)), (1, (8, 4, 1)),
                                               (1, (4, 2, 2))],
                         ids=["fp64_tile4x2", "fp64_tile2x2", "fp32split_tile4x4", "fp32split_tile8x4",
                              "fp32split_tile4x2_two_blocks"])
def test_bench_grid_nh5_matches_oracle(hb, precision, variant):
    case = _bench_grid_case()
    init, o, res_o = _oracle_run("bench_grid16", case, 2, seed=7)
    case.precision = precision
    s = hb.Solver(case)
    s.set_micro_variant(0, *variant)
    assert s.micro_variant(0) == variant
    s.set_state(0, *init)
    rc, its, res_g = s.iterate(2)
    g = s.get_state(0)
    s.destroy()
    if precision == 0:
        for k in range(3):
            close(g[k], o[k], init[k], 1e-10, 1e-13)
        np.testing.assert_allclose(res_g[0], res_o[-1], rtol=1e-8, atol=1e-16)
    else:
        close(g[0], o[0], init[0], 2e-5, 2e-9)
        close(g[1], o[1], init[1], 2e-5, 2e-7)
        close(g[2], o[2], init[2], 2e-5, 2e-7)


# the two level counts no other case uses (N_T = 9 and 13), both precisions
CASES_NH46 = [
    ("nh4_thermal", lambda: I.make_case("n4", 9, 12, kn=0.1, st=2.0, nh=4, pr=2 / 3, drive="thermal", amp=0.3,
                                        ncell_y=6), 3),
    ("nh6_shear", lambda: I.make_case("n6", 6, 10, kn=0.3, st=1.0, nh=6, pr=2 / 3, drive="shear", amp=0.02,
                                      ncell_y=9), 3),
]


@pytest.mark.parametrize("name,factory,niter", CASES_NH46, ids=[c[0] for c in CASES_NH46])
@pytest.mark.parametrize("precision", [0, 1])
def test_nh4_nh6_match_oracle(hb, name, factory, niter, precision):
    case = factory()
    case.precision = precision
    init, g, o, res_g, res_o = run_both(hb, case, niter)
    if precision == 0:
        for k in range(3):
            close(g[k], o[k], init[k], 1e-10, 1e-13)
    else:
        close(g[0], o[0], init[0], 2e-5, 2e-9)
        close(g[1], o[1], init[1], 2e-5, 2e-7)
        close(g[2], o[2], init[2], 2e-5, 2e-7)
