"""Python access to the plain FP64 CPU oracle of HB-UGKS (``hbugks_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
cpu_baseline / reference leg; never by the product package.  It shares no code with the CUDA path.

Besides loading the C oracle it holds the two small definitions the tests need next to it:
  * the Knudsen-number -> reference-viscosity map of Eq. def_Kn and the Strouhal map of Eq. def_St,
  * the harmonic extraction of Eq. dft_general (a plain loop over levels).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hbugks_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (gcc, -O2, plain ISO C; same source on x86 and Arm)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OrcProblem(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("xn", C.POINTER(C.c_double)), ("yn", C.POINTER(C.c_double)),
        ("nu", C.c_int), ("nv", C.c_int),
        ("u", C.POINTER(C.c_double)), ("wu", C.POINTER(C.c_double)),
        ("v", C.POINTER(C.c_double)), ("wv", C.POINTER(C.c_double)),
        ("umax", C.c_double), ("vmax", C.c_double),
        ("nt", C.c_int),
        ("omega", C.c_double), ("mu0", C.c_double), ("w_vss", C.c_double), ("pr", C.c_double),
        ("cfl", C.c_double), ("face_step", C.c_int), ("gam", C.c_double), ("lam_ref", C.c_double),
        ("wall", (C.c_double * 9) * 4),
        ("theta0", C.c_double), ("dt_fixed", C.c_double), ("first_order", C.c_int),
        ("spectral_implicit", C.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            d, pd, pi = C.c_double, C.POINTER(C.c_double), C.c_int
            P = C.POINTER(OrcProblem)
            _lib.orc_E_matrix.argtypes = [pi, pd]
            _lib.orc_ugks_coeffs.argtypes = [d, d, pd]
            _lib.orc_micro_slope.argtypes = [pd, d, d, d, pd]
            _lib.orc_hb_iterate.argtypes = [P, pd, pd, pd, pi, pd]
            _lib.orc_hb_iterate.restype = C.c_int
            _lib.orc_fields.argtypes = [P, pd, pd, pi, pd]
            _lib.orc_maxwell_grid.argtypes = [P, d, d, d, d, pd, pd]
            _lib.orc_shakhov_grid.argtypes = [P, d, d, d, d, d, d, pd, pd]
            _lib.orc_moments.argtypes = [P, pd, pd, pd, pd]
            _lib.orc_cell_steps.argtypes = [P, pd, pd]
            _lib.orc_van_leer.argtypes = [d, d]
            _lib.orc_van_leer.restype = d
            _lib.orc_relax_time.argtypes = [P, d, d]
            _lib.orc_relax_time.restype = d
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ------------------------------------------------------------------------ parameter maps

def vss_factor(w_vss: float = 0.81, alpha: float = 1.0) -> float:
    """Prefactor 4 alpha (5 - 2w)(7 - 2w) / (5 (alpha + 1)(alpha + 2)) of Eq. def_Kn."""
    return 4.0 * alpha * (5.0 - 2.0 * w_vss) * (7.0 - 2.0 * w_vss) / (5.0 * (alpha + 1.0) * (alpha + 2.0))


def mu0_from_kn(kn: float, w_vss: float = 0.81, alpha: float = 1.0, rho0: float = 1.0, H: float = 1.0,
                RT0: float = 0.5) -> float:
    """Eq. def_Kn solved for mu(T0): Kn = F * mu / (rho0 H sqrt(2 pi R T0))."""
    return kn * rho0 * H * math.sqrt(2.0 * math.pi * RT0) / vss_factor(w_vss, alpha)


def omega_from_st(st: float, H: float = 1.0, RT0: float = 0.5) -> float:
    """Eq. def_St: St = omega H / sqrt(2 R T0)."""
    return st * math.sqrt(2.0 * RT0) / H


# ------------------------------------------------------------------------ problem wrapper

class Problem:
    """One cavity case in the oracle's terms.  Keeps the numpy arrays the C struct points to alive."""

    def __init__(self, case, *, theta0: float = 0.0, dt_fixed: float = 0.0, first_order: bool = False,
                 nt: int | None = None):
        self.case = case
        self.xn = np.ascontiguousarray(case.xnodes, dtype=np.float64)
        self.yn = np.ascontiguousarray(case.ynodes, dtype=np.float64)
        self.u = np.ascontiguousarray(case.u, dtype=np.float64)
        self.wu = np.ascontiguousarray(case.wu, dtype=np.float64)
        self.v = np.ascontiguousarray(case.v, dtype=np.float64)
        self.wv = np.ascontiguousarray(case.wv, dtype=np.float64)
        s = OrcProblem()
        s.nx, s.ny = len(self.xn) - 1, len(self.yn) - 1
        s.xn, s.yn = _p(self.xn), _p(self.yn)
        s.nu, s.nv = len(self.u), len(self.v)
        s.u, s.wu, s.v, s.wv = _p(self.u), _p(self.wu), _p(self.v), _p(self.wv)
        s.umax, s.vmax = case.umax, case.vmax
        s.nt = nt if nt is not None else 2 * case.n_harmonics + 1
        s.omega = omega_from_st(case.st)
        s.mu0 = mu0_from_kn(case.kn, case.w_vss, case.alpha_vss)
        s.w_vss, s.pr, s.cfl = case.w_vss, case.pr, case.cfl
        s.face_step, s.gam, s.lam_ref = case.face_step, case.gamma, 1.0
        for k in range(4):
            for q in range(9):
                s.wall[k][q] = case.walls[k][q]
        s.theta0, s.dt_fixed, s.first_order = theta0, dt_fixed, int(first_order)
        s.spectral_implicit = int(getattr(case, "spectral_implicit", 0))
        self.s = s

    @property
    def nx(self): return self.s.nx

    @property
    def ny(self): return self.s.ny

    @property
    def nc(self): return self.s.nx * self.s.ny

    @property
    def nvel(self): return self.s.nu * self.s.nv

    @property
    def nt(self): return self.s.nt

    def ref(self):
        return C.byref(self.s)


# ------------------------------------------------------------------------ entry points

def E_matrix(nt: int) -> np.ndarray:
    E = np.zeros((nt, nt))
    lib().orc_E_matrix(nt, _p(E))
    return E


def ugks_coeffs(dG: float, tau: float) -> np.ndarray:
    Cc = np.zeros(5)
    lib().orc_ugks_coeffs(dG, tau, _p(Cc))
    return Cc


def micro_slope(w, U: float, V: float, lam: float) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    a = np.zeros(4)
    lib().orc_micro_slope(_p(w), U, V, lam, _p(a))
    return a


def van_leer(s1: float, s2: float) -> float:
    return lib().orc_van_leer(s1, s2)


def maxwell_grid(P: Problem, rho, U, V, lam):
    H = np.zeros(P.nvel)
    B = np.zeros(P.nvel)
    lib().orc_maxwell_grid(P.ref(), rho, U, V, lam, _p(H), _p(B))
    return H, B


def shakhov_grid(P: Problem, rho, U, V, lam, qx, qy):
    Hp = np.zeros(P.nvel)
    Bp = np.zeros(P.nvel)
    lib().orc_shakhov_grid(P.ref(), rho, U, V, lam, qx, qy, _p(Hp), _p(Bp))
    return Hp, Bp


def moments(P: Problem, h, b):
    h = np.ascontiguousarray(h, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    W = np.zeros(4)
    q = np.zeros(2)
    lib().orc_moments(P.ref(), _p(h), _p(b), _p(W), _p(q))
    return W, q


def cell_steps(P: Problem, W) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    dG = np.zeros(P.nc)
    lib().orc_cell_steps(P.ref(), _p(W), _p(dG))
    return dG


def relax_time(P: Problem, rho, lam) -> float:
    return lib().orc_relax_time(P.ref(), rho, lam)


def iterate(P: Problem, W, h, b, niter: int):
    """Advance (W, h, b) in place by `niter` pseudo-time iterations; returns the residual history (niter, 4).

    Layouts: W (nt, nc, 4), h and b (nt, nc, nvel), float64 C-contiguous; cell c = j nx + i,
    velocity a = jv nu + iu."""
    for a in (W, h, b):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    assert W.shape == (P.nt, P.nc, 4) and h.shape == (P.nt, P.nc, P.nvel) and b.shape == h.shape
    res = np.zeros((max(niter, 1), 4))
    lib().orc_hb_iterate(P.ref(), _p(W), _p(h), _p(b), niter, _p(res))
    return res[:niter]


FIELD_NAMES = ("rho", "U", "V", "T", "tau_xy", "qx", "qy", "p")


def fields(P: Problem, h, b, level: int) -> np.ndarray:
    """(8, nc) array of rho, U, V, T/T0, tau_xy, q_x, q_y, p at one level, from the moments of h, b."""
    out = np.zeros((8, P.nc))
    lib().orc_fields(P.ref(), _p(np.ascontiguousarray(h)), _p(np.ascontiguousarray(b)), level, _p(out))
    return out


def harmonics(level_values: np.ndarray) -> np.ndarray:
    """Eq. dft_general: q_hat_k = 1/N_T sum_n q_n exp(-i k omega t_n), omega t_n = 2 pi n / N_T,
    for k = 0..N_H; level_values has the level axis first."""
    nt = level_values.shape[0]
    nh = (nt - 1) // 2
    out = np.zeros((nh + 1,) + level_values.shape[1:], dtype=np.complex128)
    for k in range(nh + 1):
        for n in range(nt):
            out[k] += level_values[n] * np.exp(-1j * k * 2.0 * math.pi * n / nt)
        out[k] /= nt
    return out
