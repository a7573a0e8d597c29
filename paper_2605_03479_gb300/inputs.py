"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module is input data only: cavity meshes, discrete-velocity grids, case parameters, wall
waveforms and seeded initial states.  It computes no step of the HB-UGKS method (no flux, moment,
update or residual) and imports neither the CUDA binding nor the CPU oracle.

Units (as in the cavity benchmarks of Sec 3): lengths in cavity heights H = 1, velocities in
sqrt(2 R T0) = 1 (so R T0 = 1/2, lambda0 = 1/(2 R T0) = 1), densities in rho0 = 1, temperatures in T0 = 1.

The cavity workloads follow the shear-driven case of Sec 3.1 (lid oscillating in its own plane,
Eq. lid_velocity) and the thermally driven case of Sec 3.2 (one wall with an oscillating temperature),
at the sizes of the five benchmark configurations (see ``config1`` .. ``config5``).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

# wall ids: 0 bottom (y = 0), 1 right (x = 1), 2 top (y = 1), 3 left (x = 0)
BOTTOM, RIGHT, TOP, LEFT = 0, 1, 2, 3


def rest_wall(T: float = 1.0) -> List[float]:
    """[U_mean, V_mean, T_mean, U_re, U_im, V_re, V_im, T_re, T_im]; level n state = mean + Re(amp e^{i 2 pi n/N_T})."""
    return [0.0, 0.0, T, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0]


@dataclasses.dataclass
class Case:
    name: str
    xnodes: np.ndarray
    ynodes: np.ndarray
    u: np.ndarray
    wu: np.ndarray
    v: np.ndarray
    wv: np.ndarray
    umax: float
    vmax: float
    kn: float
    st: float
    n_harmonics: int
    pr: float = 1.0
    cfl: float = 0.8
    w_vss: float = 0.81
    alpha_vss: float = 1.0
    gamma: float = 5.0 / 3.0
    face_step: int = 0          # 0 min, 1 harmonic mean
    precision: int = 0          # 0 FP64, 1 FP32-split
    td_steps: int = 0           # > 0: explicit time-domain UGKS with this many steps per period (N_H = 0)
    spectral_implicit: int = 0  # 1: spectral source at the new pseudo-time iterate (solved across levels)
    walls: List[List[float]] = dataclasses.field(default_factory=lambda: [rest_wall() for _ in range(4)])

    @property
    def nx(self): return len(self.xnodes) - 1

    @property
    def ny(self): return len(self.ynodes) - 1

    @property
    def nu(self): return len(self.u)

    @property
    def nv(self): return len(self.v)

    @property
    def nt(self): return 2 * self.n_harmonics + 1

    @property
    def nc(self): return self.nx * self.ny

    @property
    def nvel(self): return self.nu * self.nv

    def updates_per_iteration(self) -> int:
        return self.nc * self.nvel * self.nt


# --------------------------------------------------------------------------- meshes

def uniform_nodes(n: int, length: float = 1.0) -> np.ndarray:
    return np.linspace(0.0, length, n + 1)


def tanh_nodes(n: int, ratio: float) -> np.ndarray:
    """Nodes clustered toward both ends: x_j = (1 + tanh(beta (2 j/n - 1)) / tanh(beta)) / 2, with beta found
    by bisection so that the largest ratio between adjacent cell widths equals `ratio`."""
    j = np.arange(n + 1)

    def nodes(beta):
        return 0.5 * (1.0 + np.tanh(beta * (2.0 * j / n - 1.0)) / math.tanh(beta))

    def max_ratio(beta):
        d = np.diff(nodes(beta))
        r = d[1:] / d[:-1]
        return float(np.max(np.maximum(r, 1.0 / r)))

    lo, hi = 1e-6, 20.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if max_ratio(mid) < ratio:
            lo = mid
        else:
            hi = mid
    x = nodes(0.5 * (lo + hi))
    x[0], x[-1] = 0.0, 1.0
    return x


def wall_refined_nodes(n: int, ds_min: float, length: float = 1.0) -> np.ndarray:
    """Nodes on [0, length] of the same tanh family, refined toward both walls so that the two wall cells are
    ds_min wide (the paper's cavity meshes, Sec 3.1.1: 90 rows, 0.001 H at every wall).  beta by bisection:
    the wall cell width length/2 (1 - tanh(beta (1 - 2/n)) / tanh(beta)) falls monotonically with beta."""
    if not (0.0 < ds_min < length / n):
        raise ValueError("ds_min must lie below the uniform spacing")
    j = np.arange(n + 1)

    def nodes(beta):
        return 0.5 * length * (1.0 + np.tanh(beta * (2.0 * j / n - 1.0)) / math.tanh(beta))

    lo, hi = 1e-6, 40.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if nodes(mid)[1] > ds_min:
            lo = mid
        else:
            hi = mid
    x = nodes(0.5 * (lo + hi))
    x[0], x[-1] = 0.0, length
    return x


# ------------------------------------------------------------------- velocity grids

def midpoint_grid(n: int, half_width: float = 4.0):
    """Cell-centred uniform rule on [-L, L]: nodes -L + (j + 1/2) 2L/n, weights 2L/n (no node at 0 for even n)."""
    h = 2.0 * half_width / n
    x = -half_width + (np.arange(n) + 0.5) * h
    return x, np.full(n, h)


def gauss_hermite_grid(n: int):
    """n-point Gauss-Hermite rule as a discrete-velocity grid: the nodes of the weight e^{-u^2} (the rest
    Maxwellian's shape in these units) and the weights w_j e^{u_j^2}, so that sum_j W_j f(u_j) approximates
    the plain integral of f.  Exact for f = polynomial x e^{-u^2} up to degree 2n - 1.  The nodes reach past
    +-4 (6.59 for n = 28)."""
    x, w = np.polynomial.hermite.hermgauss(n)
    return x, w * np.exp(x * x)


# ------------------------------------------------------------------- case builders

def make_case(name: str, ncell: int, nvel: int, *, kn: float, st: float, nh: int, pr: float = 1.0,
              stretched_ratio: float | None = None, drive: str = "shear", amp: float = 0.01,
              precision: int = 0, cfl: float = 0.8, half_width: float = 4.0, ncell_y: int | None = None,
              nvel_y: int | None = None, aspect: float = 1.0, ds_min: float | None = None,
              vgrid: str = "midpoint", lid_mean: float = 0.0) -> Case:
    """A cavity [0,A] x [0,1] (A = aspect) with ncell x ncell_y cells and an nvel x nvel_y velocity grid.

    Mesh: uniform; tanh-stretched to an adjacent-cell ratio (stretched_ratio); or refined toward every wall to
    a wall cell of ds_min (the same ds_min on both axes).  Velocity grid: the midpoint rule on [-L, L]
    (vgrid "midpoint") or the Gauss-Hermite rule (vgrid "gauss_hermite"; its largest node bounds the speeds).
    drive = "shear": top lid U_w = lid_mean + amp cos(omega t) (Eq. lid_velocity), all walls at T0.
    drive = "thermal": bottom wall T_w = T0 (1 + amp sin(omega t)), all walls at rest.
    drive = "thermal_top": top wall T_w = T0 (1 + amp cos(omega t)), all walls at rest (Sec 3.2).
    drive = "rest": every wall at rest and at T0."""
    ny = ncell if ncell_y is None else ncell_y
    if ds_min is not None:
        xn, yn = wall_refined_nodes(ncell, ds_min, aspect), wall_refined_nodes(ny, ds_min)
    elif stretched_ratio:
        xn, yn = aspect * tanh_nodes(ncell, stretched_ratio), tanh_nodes(ny, stretched_ratio)
    else:
        xn, yn = uniform_nodes(ncell, aspect), uniform_nodes(ny)
    nvy = nvel if nvel_y is None else nvel_y
    if vgrid == "midpoint":
        (u, wu), (v, wv) = midpoint_grid(nvel, half_width), midpoint_grid(nvy, half_width)
        umax = vmax = half_width
    elif vgrid == "gauss_hermite":
        (u, wu), (v, wv) = gauss_hermite_grid(nvel), gauss_hermite_grid(nvy)
        umax, vmax = float(np.max(np.abs(u))), float(np.max(np.abs(v)))
    else:
        raise ValueError(vgrid)
    walls = [rest_wall() for _ in range(4)]
    if drive == "shear":
        walls[TOP][0] = lid_mean
        walls[TOP][3] = amp                   # U_re: amp cos(theta)
    elif drive == "thermal":
        walls[BOTTOM][8] = -amp               # T_im = -amp: Re(-i amp e^{i theta}) = amp sin(theta)
    elif drive == "thermal_top":
        walls[TOP][7] = amp                   # T_re = amp: amp cos(theta)
    elif drive != "rest":
        raise ValueError(drive)
    return Case(name=name, xnodes=xn, ynodes=yn, u=u, wu=wu, v=v, wv=wv, umax=umax, vmax=vmax,
                kn=kn, st=st, n_harmonics=nh, pr=pr, cfl=cfl, precision=precision, walls=walls)


def config1() -> Case:
    """Shear cavity, FP64: 32x32 uniform, 24x24 velocities, BGK, Kn 0.1, St 1, N_H 1, lid 0.01 cos."""
    return make_case("shear32_v24_nh1", 32, 24, kn=0.1, st=1.0, nh=1, pr=1.0, drive="shear", amp=0.01)


def config2_cases() -> List[Case]:
    """Shear cavity, FP64: 64x64 tanh-stretched (ratio 1.1), 32x32 velocities, Shakhov Pr 2/3,
    Kn in {0.01, 0.1, 1, 10} x St in {0.1, 1, 10}, N_H 1."""
    out = []
    for kn in (0.01, 0.1, 1.0, 10.0):
        for st in (0.1, 1.0, 10.0):
            out.append(make_case(f"shear64t_v32_kn{kn:g}_st{st:g}", 64, 32, kn=kn, st=st, nh=1, pr=2.0 / 3.0,
                                 stretched_ratio=1.1, drive="shear", amp=0.01))
    return out


def config3(precision: int = 1) -> Case:
    """Thermal cavity: 64x64 uniform, 48x48 velocities, Shakhov, bottom wall T0(1 + 0.5 sin), Kn 0.5, St 1, N_H 3."""
    return make_case("thermal64_v48_nh3", 64, 48, kn=0.5, st=1.0, nh=3, pr=2.0 / 3.0, drive="thermal", amp=0.5,
                     precision=precision)


def config4_cases(seed: int = 20260503, n: int = 48, precision: int = 1) -> List[Case]:
    """48 uneven cases drawn with numpy PCG64(seed) in the order: drive in {shear, thermal} (p = 1/2);
    N_cell in {32, 40, ..., 96}; N_vel in {24, 32, 40, 48}; N_H in {1, 2, 3}; log10 Kn ~ U[-2, 1];
    log10 St ~ U[-1, 1].  Shakhov Pr 2/3; shear lid 0.01 cos, thermal bottom wall 0.5 sin."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cells = list(range(32, 97, 8))
    vels = [24, 32, 40, 48]
    out = []
    for k in range(n):
        drive = "shear" if rng.random() < 0.5 else "thermal"
        nc = int(cells[rng.integers(len(cells))])
        nv = int(vels[rng.integers(len(vels))])
        nh = int(rng.integers(1, 4))
        kn = float(10.0 ** rng.uniform(-2.0, 1.0))
        st = float(10.0 ** rng.uniform(-1.0, 1.0))
        out.append(make_case(f"batch{k:02d}_{drive}{nc}_v{nv}_nh{nh}", nc, nv, kn=kn, st=st, nh=nh, pr=2.0 / 3.0,
                             drive=drive, amp=0.01 if drive == "shear" else 0.5, precision=precision))
    return out


def config5(precision: int = 1) -> Case:
    """Large thermal cavity: 128x128 uniform, 64x64 velocities, Shakhov, bottom wall T0(1 + 0.5 sin),
    Kn 0.05, St 5, N_H 5 (N_T = 11)."""
    return make_case("thermal128_v64_nh5", 128, 64, kn=0.05, st=5.0, nh=5, pr=2.0 / 3.0, drive="thermal",
                     amp=0.5, precision=precision)


# ----------------------------------------------------- the paper's own cavity workloads (Sec 3)

PAPER_ROWS = 90            # cells across the cavity height (Sec 3.1.1)
PAPER_DS_MIN = 0.001       # wall cell width in cavity heights (Sec 3.1.1)


def kn_from_reynolds(re: float, u_mean: float, w_vss: float = 0.81, alpha_vss: float = 1.0) -> float:
    """The Knudsen number whose reference viscosity (Eq. def_Kn) is mu(T0) = rho0 U_mean H / Re
    (Eq. def_Re_mu0), with rho0 = H = 1 and sqrt(2 R T0) = 1, so that the cases of the continuum limit
    (Sec 3.3) pass through the same Kn input as every other case."""
    c_vss = 4.0 * alpha_vss * (5.0 - 2.0 * w_vss) * (7.0 - 2.0 * w_vss) / (5.0 * (alpha_vss + 1.0) * (alpha_vss + 2.0))
    return c_vss * (u_mean / re) / math.sqrt(math.pi)


def paper_shear_case(kn: float, st: float, aspect: float = 1.0, *, nh: int = 1, amp: float = 0.0015,
                     precision: int = 0, rows: int = PAPER_ROWS, ds_min: float = PAPER_DS_MIN) -> Case:
    """Shear-driven cavity of Sec 3.1: aspect A = L/H with round(A rows) x rows cells refined to ds_min at
    every wall, lid 0.0015 cos(omega t), Shakhov Pr 2/3; 28 x 28 Gauss-Hermite velocities for Kn <= 0.1,
    the 64 x 64 midpoint rule on [-4, 4] otherwise."""
    gh = kn <= 0.1
    ncell = int(round(aspect * rows))
    return make_case(f"paper_shear_A{aspect:g}_kn{kn:g}_st{st:g}", ncell, 28 if gh else 64, kn=kn, st=st, nh=nh,
                     pr=2.0 / 3.0, drive="shear", amp=amp, precision=precision, ncell_y=rows, aspect=aspect,
                     ds_min=ds_min, vgrid="gauss_hermite" if gh else "midpoint")


def paper_thermal_case(kn: float, st: float = 2.0, *, nh: int = 2, amp: float = 0.3, precision: int = 0,
                       rows: int = PAPER_ROWS, ds_min: float = PAPER_DS_MIN) -> Case:
    """Thermally driven square cavity of Sec 3.2: the shear case's mesh, top wall T0 (1 + 0.3 cos(omega t)),
    N_H = 2, Shakhov Pr 2/3, one velocity grid for every Kn (the 64 x 64 midpoint rule on [-4, 4])."""
    return make_case(f"paper_thermal_kn{kn:g}_st{st:g}_nh{nh}", rows, 64, kn=kn, st=st, nh=nh, pr=2.0 / 3.0,
                     drive="thermal_top", amp=amp, precision=precision, ds_min=ds_min)


def continuum_case(re: float, *, u_mean: float = 0.15, amp: float = 0.0015, st: float = 1.0, precision: int = 0,
                   rows: int = PAPER_ROWS, ds_min: float = PAPER_DS_MIN) -> Case:
    """Continuum limit of Sec 3.3: lid U_w = 0.15 + 0.0015 cos(omega t), viscosity from Re (Eq. def_Re_mu0),
    16 x 16 uniform velocities on [-4, 4], N_H = 1, Shakhov Pr 2/3."""
    return make_case(f"continuum_re{re:g}", rows, 16, kn=kn_from_reynolds(re, u_mean), st=st, nh=1,
                     pr=2.0 / 3.0, drive="shear", amp=amp, lid_mean=u_mean, precision=precision, ds_min=ds_min)


# ------------------------------------------------------------------- initial states

def splitmix64(seed: int, count: int) -> np.ndarray:
    """`count` outputs of the SplitMix64 generator (Steele, Lea, Flood 2014), as uint64."""
    mask = (1 << 64) - 1
    z = seed & mask
    out = np.zeros(count, dtype=np.uint64)
    for k in range(count):
        z = (z + 0x9E3779B97F4A7C15) & mask
        x = z
        x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & mask
        x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & mask
        x = x ^ (x >> 31)
        out[k] = x
    return out


def unit_uniform(seed: int, count: int) -> np.ndarray:
    """SplitMix64 outputs mapped to [-1, 1) through their top 53 bits."""
    r = splitmix64(seed, count)
    return (r >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def primitive_fields(case: Case, seed: int | None = None, amp: float = 0.01):
    """Primitive fields rho, U, V, T per level and cell, shape (nt, nc) each.

    seed None: the uniform rest state rho = 1, U = V = 0, T = 1 on every level ("fluid initially at rest").
    Otherwise a smooth seeded perturbation of that state: for each level and variable, a sum of the 9 modes
    cos(pi kx x) cos(pi ky y), kx, ky in 0..2, with coefficients from SplitMix64(seed) scaled by `amp`;
    rho and T are multiplied by (1 + field), U and V are set to the field."""
    nt, nx, ny = case.nt, case.nx, case.ny
    xc = 0.5 * (case.xnodes[1:] + case.xnodes[:-1])
    yc = 0.5 * (case.ynodes[1:] + case.ynodes[:-1])
    X, Y = np.meshgrid(xc, yc)                       # (ny, nx): cell c = j nx + i
    rho = np.ones((nt, nx * ny))
    U = np.zeros((nt, nx * ny))
    V = np.zeros((nt, nx * ny))
    T = np.ones((nt, nx * ny))
    if seed is None:
        return rho, U, V, T
    coef = unit_uniform(seed, nt * 4 * 9).reshape(nt, 4, 9)
    for n in range(nt):
        flds = []
        for q in range(4):
            f = np.zeros_like(X)
            for k in range(9):
                kx, ky = k // 3, k % 3
                f += coef[n, q, k] * np.cos(math.pi * kx * X) * np.cos(math.pi * ky * Y)
            flds.append(amp * f.reshape(-1) / 3.0)
        rho[n] *= 1.0 + flds[0]
        U[n] = flds[1]
        V[n] = flds[2]
        T[n] *= 1.0 + flds[3]
    return rho, U, V, T


def initial_state(case: Case, seed: int | None = None, amp: float = 0.01):
    """Initial (W, h, b) in the canonical layout: W (nt, nc, 4) = (rho, rho U, rho V, rho E) with
    rho E = rho |U|^2/2 + 3 rho T / 4 (D + K = 3 degrees of freedom, R T0 = 1/2), and h, b (nt, nc, nvel) the
    reduced Gaussians rho (lam/pi) exp(-lam |u - U|^2) and that divided by 2 lam, lam = 1/T, on the
    velocity grid (velocity a = jv nu + iu)."""
    rho, U, V, T = primitive_fields(case, seed, amp)
    nt, nc = rho.shape
    W = np.zeros((nt, nc, 4))
    W[..., 0] = rho
    W[..., 1] = rho * U
    W[..., 2] = rho * V
    W[..., 3] = 0.5 * rho * (U * U + V * V) + 0.75 * rho * T
    uu, vv = np.meshgrid(case.u, case.v)            # (nv, nu): velocity a = jv nu + iu
    uu, vv = uu.reshape(-1), vv.reshape(-1)
    lam = 1.0 / T
    c2 = (uu[None, None, :] - U[..., None]) ** 2 + (vv[None, None, :] - V[..., None]) ** 2
    h = rho[..., None] * (lam[..., None] / math.pi) * np.exp(-lam[..., None] * c2)
    b = h / (2.0 * lam[..., None])
    return np.ascontiguousarray(W), np.ascontiguousarray(h), np.ascontiguousarray(b)


def tiny_case(name="tiny", ncell=6, nvel=8, *, kn=0.1, st=1.0, nh=1, pr=1.0, drive="shear", amp=0.01,
              precision=0, **kw) -> Case:
    """Small cases the CPU oracle iterates in well under a second."""
    return make_case(name, ncell, nvel, kn=kn, st=st, nh=nh, pr=pr, drive=drive, amp=amp, precision=precision, **kw)


def all_configs() -> Sequence[Case]:
    return [config1(), *config2_cases(), config3(), *config4_cases(), config5()]
