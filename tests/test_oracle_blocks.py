"""Pins of the oracle's building blocks against what the paper and the mathematics fix.

Every expected value here comes from a closed form, a high-precision evaluation (mpmath), an
independent numerical integration of the paper's defining integral, or a golden fixture derived by
hand from a printed formula -- never from the oracle itself or from the CUDA path.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_03479_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ Eq. D_explicit (matrix E)

def test_E_nt3_matches_hand_worked_fixture():
    M = np.loadtxt(os.path.join(GOLD, "E_NT3.txt"))
    np.testing.assert_allclose(O.E_matrix(3), M / math.sqrt(3.0), rtol=0, atol=2e-16)


@pytest.mark.parametrize("nt", [3, 5, 7, 9, 11])
def test_E_exact_on_trig_polynomials(nt):
    """Eq. derivative_derivation: omega E f(t_n) = f'(t_n) for f = cos(k w t), sin(k w t), k <= N_H."""
    E = O.E_matrix(nt)
    nh = (nt - 1) // 2
    th = 2.0 * math.pi * np.arange(nt) / nt
    for k in range(0, nh + 1):
        for f, df in ((np.cos(k * th), -k * np.sin(k * th)), (np.sin(k * th), k * np.cos(k * th))):
            np.testing.assert_allclose(E @ f, df, atol=1e-13 * max(1, k))


@pytest.mark.parametrize("nt", [3, 5, 7, 11])
def test_E_aliases_above_nh(nt):
    """Negative control: at k = N_H + 1 the collocation derivative is wrong (aliasing)."""
    E = O.E_matrix(nt)
    k = (nt - 1) // 2 + 1
    th = 2.0 * math.pi * np.arange(nt) / nt
    assert np.max(np.abs(E @ np.sin(k * th) - k * np.cos(k * th))) > 0.5


@pytest.mark.parametrize("nt", [3, 5, 7, 9, 11])
def test_E_skew_and_spectrum(nt):
    """Sec 2.2: E is real skew-symmetric for odd N_T, eigenvalues i k (k = -N_H..N_H), radius N_H."""
    E = O.E_matrix(nt)
    np.testing.assert_allclose(E, -E.T, atol=1e-15)
    np.testing.assert_allclose(E.sum(axis=1), 0.0, atol=1e-14)
    ev = np.sort(np.linalg.eigvals(E).imag)
    nh = (nt - 1) // 2
    np.testing.assert_allclose(ev, np.arange(-nh, nh + 1), atol=1e-12)
    np.testing.assert_allclose(np.linalg.eigvals(E).real, 0.0, atol=1e-12)


@pytest.mark.parametrize("nt", [3, 5, 7])
def test_E_equals_i_Dinv_K_D(nt):
    """Eq. derivative_derivation with D^{-1} built column by column as printed in Eq. D_matrix."""
    nh = (nt - 1) // 2
    ks = [0] + list(range(1, nh + 1)) + list(range(-nh, 0))      # K = diag(0, 1..N_H, -N_H..-1)
    t = 2.0 * math.pi * np.arange(nt) / nt                        # omega t_n
    Dinv = np.array([[np.exp(1j * k * tn) for k in ks] for tn in t])
    D = np.linalg.inv(Dinv)
    Emat = 1j * Dinv @ np.diag(ks) @ D
    np.testing.assert_allclose(Emat.imag, 0.0, atol=1e-13)
    np.testing.assert_allclose(O.E_matrix(nt), Emat.real, atol=1e-13)


# ------------------------------------------------------------------ Eq. C_coeffs

mp = pytest.importorskip("mpmath")


def _C_mp(dG, tau):
    mp.mp.dps = 60
    dG, tau = mp.mpf(dG), mp.mpf(tau)
    e = mp.exp(-dG / tau)
    return [dG - tau * (1 - e),
            2 * tau ** 2 * (1 - e) - tau * dG - tau * dG * e,
            dG ** 2 / 2 - tau * dG + tau ** 2 * (1 - e),
            tau * (1 - e),
            tau * dG * e - tau ** 2 * (1 - e)]


@pytest.mark.parametrize("x", [1e-9, 1e-6, 1e-4, 3e-3, 0.05, 0.3, 0.7, 0.999, 1.0, 1.001, 2.0, 7.5, 40.0, 800.0])
@pytest.mark.parametrize("tau", [1e-3, 0.7, 5.0])
def test_C_coeffs_high_precision(x, tau):
    dG = x * tau
    got = O.ugks_coeffs(dG, tau)
    ref = [float(v) for v in _C_mp(dG, tau)]
    for g, r in zip(got, ref):
        assert abs(g - r) <= 1e-13 * abs(r) + 1e-300, (x, tau, got, ref)


def test_C_coeffs_are_the_time_integrals_of_the_integral_solution():
    """Eq. integral_solution integrated over [0, dG] with h+ = h+_0 [1 + a.x' + A G'] and h_0(x) = h_0 + sigma x:
    C1 multiplies h+_0, C2 (u.a) h+_0, C3 A h+_0, C4 h_0, C5 (u.sigma), by independent quadrature."""
    from scipy import integrate
    tau, dG = 0.37, 0.81
    def eq(G, poly):       # (1/tau) int_0^G poly(G, G') e^{-(G-G')/tau} dG'
        return integrate.quad(lambda Gp: poly(G, Gp) * math.exp(-(G - Gp) / tau) / tau, 0.0, G, epsabs=1e-14)[0]
    c1 = integrate.quad(lambda G: eq(G, lambda G, Gp: 1.0), 0, dG, epsabs=1e-14)[0]
    # x' = x_f - u (G - G') relative to the face: a.u term -> -(G - G')
    c2 = integrate.quad(lambda G: eq(G, lambda G, Gp: -(G - Gp)), 0, dG, epsabs=1e-14)[0]
    c3 = integrate.quad(lambda G: eq(G, lambda G, Gp: Gp), 0, dG, epsabs=1e-14)[0]
    c4 = integrate.quad(lambda G: math.exp(-G / tau), 0, dG, epsabs=1e-14)[0]
    c5 = integrate.quad(lambda G: -G * math.exp(-G / tau), 0, dG, epsabs=1e-14)[0]
    np.testing.assert_allclose(O.ugks_coeffs(dG, tau), [c1, c2, c3, c4, c5], rtol=1e-10)


def test_C_coeffs_limits():
    dG = 0.013
    C = O.ugks_coeffs(dG, 1e-13)     # collision dominated: C1 -> dG, C3 -> dG^2/2, C2, C4, C5 -> 0
    assert abs(C[0] - dG) < 1e-10 * dG and abs(C[3]) < 1e-10 * dG
    assert abs(C[1]) < 1e-10 * dG ** 2 and abs(C[2] - dG * dG / 2) < 1e-10 * dG ** 2 and abs(C[4]) < 1e-10 * dG ** 2
    C = O.ugks_coeffs(dG, 1e9)       # free transport: C4 -> dG, C5 -> -dG^2/2, C1, C2, C3 -> 0
    assert abs(C[3] - dG) < 1e-8 * dG and abs(C[4] + dG * dG / 2) < 1e-8 * dG * dG
    assert abs(C[0]) < 1e-8 * dG and abs(C[1]) < 1e-8 * dG ** 2 and abs(C[2]) < 1e-8 * dG ** 2
    for x in (1e-5, 0.5, 1.0, 3.0):
        C = O.ugks_coeffs(x * 0.4, 0.4)
        assert abs(C[0] + C[3] - x * 0.4) <= 4e-16 * x * 0.4


# ------------------------------------------------------------------ Maxwellian slope inversion

def _continuous_moments_of_a_psi_g(a, U, V, lam, n=24):
    """Moments (per unit density) of (a.psi) g with psi = (1, u, v, (u^2+v^2+xi^2)/2) for the 3-D
    Maxwellian (u, v, xi) by tensor Gauss-Hermite quadrature (exact for polynomials of degree < 2n)."""
    x, wx = np.polynomial.hermite.hermgauss(n)
    s = 1.0 / math.sqrt(lam)
    u = U + s * x
    v = V + s * x
    xi = s * x
    w = wx / math.sqrt(math.pi)
    uu, vv, xx = np.meshgrid(u, v, xi, indexing="ij")
    ww = w[:, None, None] * w[None, :, None] * w[None, None, :]
    e = 0.5 * (uu ** 2 + vv ** 2 + xx ** 2)
    ap = a[0] + a[1] * uu + a[2] * vv + a[3] * e
    return np.array([np.sum(ww * ap * p) for p in (1.0, uu, vv, e)])


@pytest.mark.parametrize("seed", range(6))
def test_micro_slope_round_trip(seed):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=4)
    U, V, lam = rng.normal() * 0.3, rng.normal() * 0.3, 0.5 + rng.random() * 2
    w = _continuous_moments_of_a_psi_g(a, U, V, lam)
    np.testing.assert_allclose(O.micro_slope(w, U, V, lam), a, rtol=1e-11, atol=1e-12)


# ------------------------------------------------------------------ equilibria and moments

def _fine_problem(n=200, L=8.0, pr=2.0 / 3.0):
    c = I.make_case("fine", 2, n, kn=0.1, st=1.0, nh=1, pr=pr, half_width=L)
    return O.Problem(c)


def test_reduced_maxwellian_moments_on_fine_grid():
    P = _fine_problem()
    rho, U, V, lam = 1.3, 0.21, -0.17, 0.8
    H, B = O.maxwell_grid(P, rho, U, V, lam)
    W, q = O.moments(P, H, B)
    # continuous: W = (rho, rho U, rho V, rho |U|^2/2 + 3 rho/(4 lam)), q = 0
    np.testing.assert_allclose(W, [rho, rho * U, rho * V, 0.5 * rho * (U * U + V * V) + 0.75 * rho / lam],
                               rtol=1e-12)
    np.testing.assert_allclose(q, 0.0, atol=1e-12)


def test_reduced_shakhov_is_the_xi_integral_of_eq_shakhov():
    """H+ and B+ against a direct Gauss-Hermite integration over xi of (g+ - g) and xi^2 (g+ - g)."""
    c = I.make_case("s", 2, 6, kn=0.1, st=1.0, nh=1, pr=2.0 / 3.0, half_width=2.0)
    P = O.Problem(c)
    rho, U, V, lam, qx, qy = 1.1, 0.05, -0.08, 1.2, 0.013, -0.021
    Hp, Bp = O.shakhov_grid(P, rho, U, V, lam, qx, qy)
    x, wx = np.polynomial.hermite.hermgauss(30)
    RT = 1.0 / (2 * lam)
    p = rho * RT
    for jv, vv in enumerate(c.v):
        for iu, uu in enumerate(c.u):
            a = jv * c.nu + iu
            cx, cy = uu - U, vv - V
            # g = rho (lam/pi)^{3/2} exp(-lam(|c|^2 + xi^2)); substitute xi = y / sqrt(lam)
            xi = x / math.sqrt(lam)
            g = rho * (lam / math.pi) ** 1.5 * np.exp(-lam * (cx * cx + cy * cy)) * (1.0 / math.sqrt(lam))
            corr = (1 - c.pr) * (cx * qx + cy * qy) / (5 * p * RT) * ((cx * cx + cy * cy + xi * xi) / RT - 5)
            Hp_ref = np.sum(wx * g * corr)
            Bp_ref = np.sum(wx * g * corr * xi * xi)
            assert abs(Hp[a] - Hp_ref) < 1e-13 * (abs(Hp_ref) + 1e-300) + 1e-17
            assert abs(Bp[a] - Bp_ref) < 1e-13 * (abs(Bp_ref) + 1e-300) + 1e-17


def test_shakhov_conserves_and_sets_heat_flux():
    """g+ - g carries no mass, momentum or energy, and the heat flux of g+ is (1 - Pr) q."""
    P = _fine_problem(pr=2.0 / 3.0)
    rho, U, V, lam, qx, qy = 0.9, -0.12, 0.07, 1.4, 0.03, -0.02
    H, B = O.maxwell_grid(P, rho, U, V, lam)
    Hp, Bp = O.shakhov_grid(P, rho, U, V, lam, qx, qy)
    Wc, _ = O.moments(P, Hp, Bp)
    np.testing.assert_allclose(Wc, 0.0, atol=1e-12)
    _, q = O.moments(P, H + Hp, B + Bp)
    np.testing.assert_allclose(q, [(1 - 2.0 / 3.0) * qx, (1 - 2.0 / 3.0) * qy], rtol=1e-10)


# ------------------------------------------------------------------ limiter, steps, parameters

def test_van_leer_special_cases():
    for s in (0.3, -2.0, 1e-9):
        assert O.van_leer(s, s) == pytest.approx(s, rel=1e-15)
    assert O.van_leer(1.0, -1.0) == 0.0
    assert O.van_leer(0.0, 5.0) == 0.0
    assert O.van_leer(0.0, 0.0) == 0.0
    rng = np.random.default_rng(3)
    for _ in range(200):
        s1, s2 = rng.normal(size=2)
        v = O.van_leer(s1, s2)
        assert v == pytest.approx(O.van_leer(s2, s1), rel=1e-15)
        if s1 * s2 > 0:
            assert abs(v) <= 2 * min(abs(s1), abs(s2)) + 1e-15 and np.sign(v) == np.sign(s1)
            assert v == pytest.approx(2 * s1 * s2 / (s1 + s2), rel=1e-14)


def test_local_step_closed_form():
    """Eqs. dt_hb and nu_conv on a uniform state at rest: u~ = v~ = 4 + sqrt(gamma/2 T)."""
    c = I.make_case("dt", 5, 8, kn=0.1, st=3.0, nh=2, stretched_ratio=1.1)
    P = O.Problem(c)
    W, h, b = I.initial_state(c)
    dG = O.cell_steps(P, W)
    dx = np.diff(c.xnodes)
    dy = np.diff(c.ynodes)
    cs = math.sqrt(5.0 / 3.0 / 2.0)
    for j in range(c.ny):
        for i in range(c.nx):
            nu = (dy[j] * (4 + cs) + dx[i] * (4 + cs)) / (dx[i] * dy[j])
            assert dG[j * c.nx + i] == pytest.approx(0.8 / (nu + 3.0 * 2), rel=1e-14)


def _uniform_W(case, rho=1.0, U=0.0, V=0.0, T=1.0):
    """Conservative variables of a uniform state on every level (D + K = 3 degrees of freedom, R T0 = 1/2)."""
    W = np.zeros((case.nt, case.nc, 4))
    W[..., 0] = rho
    W[..., 1] = rho * U
    W[..., 2] = rho * V
    W[..., 3] = 0.5 * rho * (U * U + V * V) + 0.75 * rho * T
    return W


@pytest.mark.parametrize("nh", [1, 2, 5])
def test_local_step_spectral_term_is_the_spectral_radius_of_omega_E(nh):
    """Eq. dt_hb names omega N_H the spectral radius of the temporal differentiation matrix.  Between two
    Strouhal numbers on the same state and mesh the convective term cancels: CFL (1/dG_2 - 1/dG_1) must equal
    the difference of the largest |eigenvalue| of omega E, computed by numpy from the oracle's E."""
    c1 = I.make_case("s1", 5, 8, kn=0.1, st=0.7, nh=nh, stretched_ratio=1.1)
    c2 = I.make_case("s2", 5, 8, kn=0.1, st=6.0, nh=nh, stretched_ratio=1.1)
    W = I.initial_state(c1, seed=4)[0]
    d1 = O.cell_steps(O.Problem(c1), W)
    d2 = O.cell_steps(O.Problem(c2), W)
    E = O.E_matrix(c1.nt)
    rad = lambda st: float(np.max(np.abs(np.linalg.eigvals(O.omega_from_st(st) * E))))
    np.testing.assert_allclose(c1.cfl / d2 - c1.cfl / d1, rad(6.0) - rad(0.7), rtol=1e-11)
    assert rad(1.0) == pytest.approx(nh, rel=1e-12)


def test_local_step_convective_term_follows_cell_size_and_signal_speed():
    """Eq. nu_conv on a uniform square mesh, uniform states: halving the cells doubles the convective rate;
    widening the velocity space by dL adds dL (1/dx + 1/dy); a flow along x faster than the velocity-space bound
    replaces the bound on x only; four times the temperature doubles the sound-speed part; the hottest level
    sets the step of every level.  The spectral term is removed with a vanishing Strouhal number."""
    st = 1e-12

    def nu(case, W):
        return case.cfl / O.cell_steps(O.Problem(case), W) - O.omega_from_st(st) * case.n_harmonics

    c4 = I.make_case("m4", 4, 8, kn=0.1, st=st, nh=1)
    c8 = I.make_case("m8", 8, 8, kn=0.1, st=st, nh=1)
    n4 = nu(c4, _uniform_W(c4))
    n8 = nu(c8, _uniform_W(c8))
    np.testing.assert_allclose(n8, 2.0 * n4[0], rtol=1e-13)
    inv = 4.0 + 4.0                                           # 1/dx + 1/dy on the 4 x 4 unit square
    wide = I.make_case("w", 4, 8, kn=0.1, st=st, nh=1, half_width=6.0)
    np.testing.assert_allclose(nu(wide, _uniform_W(wide)) - n4, 2.0 * inv, rtol=1e-13)
    np.testing.assert_allclose(nu(c4, _uniform_W(c4, U=9.0)) - n4, (9.0 - 4.0) * 4.0, rtol=1e-13)
    cs = math.sqrt((5.0 / 3.0) * 0.5)                         # sqrt(gamma R T0), gamma = 5/3, R T0 = 1/2
    np.testing.assert_allclose(nu(c4, _uniform_W(c4, T=4.0)) - n4, cs * inv, rtol=1e-12)
    Wmix = _uniform_W(c4)
    Wmix[1] = _uniform_W(c4, T=4.0)[1]                        # one hot level
    np.testing.assert_allclose(nu(c4, Wmix), nu(c4, _uniform_W(c4, T=4.0)), rtol=1e-14)


def test_kn_and_st_maps_match_hand_values():
    rows = np.loadtxt(os.path.join(GOLD, "kn_map.txt"))
    for kn, mu0 in rows:
        assert O.mu0_from_kn(kn) == pytest.approx(mu0, rel=2e-9)
    assert O.omega_from_st(2.5) == pytest.approx(2.5, rel=1e-15)


def test_relaxation_time_power_law():
    c = I.tiny_case(kn=0.2)
    P = O.Problem(c)
    mu0 = O.mu0_from_kn(0.2)
    for rho, T in ((1.0, 1.0), (0.5, 1.7), (2.0, 0.6)):
        lam = 1.0 / T
        assert O.relax_time(P, rho, lam) == pytest.approx(mu0 * T ** 0.81 / (rho * T / 2.0), rel=1e-14)


def test_tanh_mesh_ratio():
    x = I.tanh_nodes(64, 1.1)
    d = np.diff(x)
    r = d[1:] / d[:-1]
    assert np.max(np.maximum(r, 1 / r)) == pytest.approx(1.1, rel=1e-9)
    np.testing.assert_allclose(d, d[::-1], rtol=1e-12)


@pytest.mark.parametrize("nt", [3, 5, 7, 11])
def test_harmonics_sign_and_scale_of_eq_dft_general(nt):
    """Eq. dft_general with the kernel e^{-i k omega t_n}, omega t_n = 2 pi n / N_T: samples of
    A cos(omega t + phi) + B sin(2 omega t) + C give C at k = 0, (A/2) e^{+i phi} at k = 1 and -i B/2 at k = 2
    (a transform with the opposite sign of the exponent gives the conjugates; one without the 1/N_T scales them)."""
    th = 2 * math.pi * np.arange(nt) / nt
    for A, phi, B, Cc in ((0.8, 0.3, 0.1, 1.5), (1.3, -1.1, -0.25, -0.2), (0.5, 2.5, 0.0, 0.0)):
        q = A * np.cos(th + phi) + (B * np.sin(2 * th) if nt >= 5 else 0.0) + Cc
        H = O.harmonics(np.stack([np.array([x]) for x in q]))[:, 0]
        assert abs(H[0] - Cc) < 1e-14
        assert abs(H[1] - 0.5 * A * np.exp(1j * phi)) < 1e-14
        if nt >= 5:
            assert abs(H[2] - (-0.5j * B)) < 1e-14
