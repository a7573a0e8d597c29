"""Python binding of the HB-UGKS C ABI (include/hbugks.h): argument marshalling only.

Every step of the pseudo-time iteration runs in the CUDA kernels of ``csrc/``; this module converts
Python/numpy arguments to the C structures, owns the device workspace through a PyTorch tensor and calls
the library.  There is no fallback: if the compiled library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhbugks.so")
_lib = None
_lock = threading.Lock()

OK, NOT_CONVERGED, EINVAL, ECUDA, ENOMEM, DIVERGED, TIMEOUT = 0, 1, -1, -2, -3, -4, -5
FIELD_NAMES = ("rho", "U", "V", "T", "tau_xy", "qx", "qy", "p")


class HbugksError(RuntimeError):
    def __init__(self, status: int, what: str):
        detail = f" [{lib().hbugks_cuda_error_string().decode()}]" if status == ECUDA else ""
        super().__init__(f"{what}: {status_string(status)} ({status}){detail}")
        self.status = status


class Mesh(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("xnodes", C.POINTER(C.c_double)),
                ("ynodes", C.POINTER(C.c_double))]


class VGrid(C.Structure):
    _fields_ = [("nu", C.c_int), ("nv", C.c_int), ("u", C.POINTER(C.c_double)), ("wu", C.POINTER(C.c_double)),
                ("v", C.POINTER(C.c_double)), ("wv", C.POINTER(C.c_double)), ("umax", C.c_double),
                ("vmax", C.c_double)]


class Physics(C.Structure):
    _fields_ = [("kn", C.c_double), ("st", C.c_double), ("pr", C.c_double), ("cfl", C.c_double),
                ("w_vss", C.c_double), ("alpha_vss", C.c_double), ("gamma", C.c_double),
                ("n_harmonics", C.c_int), ("face_step", C.c_int), ("precision", C.c_int), ("td_steps", C.c_int),
                ("spectral_implicit", C.c_int)]


class Wall(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("u_mean", "v_mean", "T_mean", "u_re", "u_im", "v_re", "v_im",
                                          "T_re", "T_im")]


class Case(C.Structure):
    _fields_ = [("mesh", Mesh), ("vgrid", VGrid), ("phys", Physics), ("walls", Wall * 4)]


EXPORTED = ("hbugks_workspace_bytes", "hbugks_create", "hbugks_destroy", "hbugks_set_wall", "hbugks_init_uniform",
            "hbugks_set_state", "hbugks_get_state", "hbugks_iterate", "hbugks_set_active",
            "hbugks_residual_history", "hbugks_get_level_fields", "hbugks_get_harmonic", "hbugks_iteration_count",
            "hbugks_status_string", "hbugks_enqueue_iterations", "hbugks_profile_kernels",
            "hbugks_harmonic_noalloc", "hbugks_launches_per_iteration", "hbugks_get_tile_shape",
            "hbugks_set_tile_shape", "hbugks_cuda_error_string", "hbugks_test_expire_wait",
            "hbugks_copy_state", "hbugks_set_loop_mode", "hbugks_get_micro_variant",
            "hbugks_set_micro_variant")


def lib():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"HB-UGKS CUDA library not built: {LIB_PATH} missing "
                                   "(run paper_2605_03479_gb300/build.py)")
            L = C.CDLL(LIB_PATH)
            pd, vp, i, d, sz = C.POINTER(C.c_double), C.c_void_p, C.c_int, C.c_double, C.c_size_t
            pc = C.POINTER(Case)
            L.hbugks_workspace_bytes.argtypes = [i, pc]
            L.hbugks_workspace_bytes.restype = sz
            L.hbugks_create.argtypes = [i, pc, vp, sz, vp, C.POINTER(vp)]
            L.hbugks_destroy.argtypes = [vp]
            L.hbugks_destroy.restype = None
            L.hbugks_set_wall.argtypes = [vp, i, i, C.POINTER(Wall)]
            L.hbugks_init_uniform.argtypes = [vp, i, d, d, d, d]
            L.hbugks_set_state.argtypes = [vp, i, pd, pd, pd]
            L.hbugks_get_state.argtypes = [vp, i, pd, pd, pd]
            L.hbugks_iterate.argtypes = [vp, i, d, C.POINTER(C.c_int), pd]
            L.hbugks_set_active.argtypes = [vp, C.POINTER(C.c_int)]
            L.hbugks_residual_history.argtypes = [vp, i, i, pd]
            L.hbugks_get_level_fields.argtypes = [vp, i, i, pd]
            L.hbugks_get_harmonic.argtypes = [vp, i, i, pd, pd]
            L.hbugks_iteration_count.argtypes = [vp, i]
            L.hbugks_iteration_count.restype = C.c_longlong
            L.hbugks_status_string.argtypes = [i]
            L.hbugks_status_string.restype = C.c_char_p
            L.hbugks_enqueue_iterations.argtypes = [vp, i]
            L.hbugks_profile_kernels.argtypes = [vp, i, pd]
            L.hbugks_harmonic_noalloc.argtypes = [i, i, i, i, vp, vp, vp, vp, i, vp, vp, i, vp, vp, vp]
            L.hbugks_launches_per_iteration.argtypes = [vp]
            L.hbugks_cuda_error_string.argtypes = []
            L.hbugks_cuda_error_string.restype = C.c_char_p
            L.hbugks_get_tile_shape.argtypes = [vp, i, C.POINTER(i), C.POINTER(i)]
            L.hbugks_set_tile_shape.argtypes = [vp, i, i, i]
            L.hbugks_get_micro_variant.argtypes = [vp, i, C.POINTER(i), C.POINTER(i), C.POINTER(i)]
            L.hbugks_set_micro_variant.argtypes = [vp, i, i, i, i]
            L.hbugks_test_expire_wait.argtypes = [vp]
            L.hbugks_copy_state.argtypes = [vp, i, vp, i]
            L.hbugks_set_loop_mode.argtypes = [vp, i]
            for name in EXPORTED:
                if name not in ("hbugks_workspace_bytes", "hbugks_destroy", "hbugks_iteration_count",
                                "hbugks_status_string", "hbugks_cuda_error_string"):
                    getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().hbugks_status_string(int(s)).decode()


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(rc: int, what: str, allow=(OK,)):
    if rc not in allow:
        raise HbugksError(rc, what)
    return rc


class _CaseArgs:
    """C structure of one case plus the numpy arrays it points to (kept alive)."""

    def __init__(self, case):
        self.arrays = [np.ascontiguousarray(x, dtype=np.float64) for x in
                       (case.xnodes, case.ynodes, case.u, case.wu, case.v, case.wv)]
        xn, yn, u, wu, v, wv = self.arrays
        c = Case()
        c.mesh = Mesh(len(xn) - 1, len(yn) - 1, _dp(xn), _dp(yn))
        c.vgrid = VGrid(len(u), len(v), _dp(u), _dp(wu), _dp(v), _dp(wv), case.umax, case.vmax)
        c.phys = Physics(case.kn, case.st, case.pr, case.cfl, case.w_vss, case.alpha_vss, case.gamma,
                         case.n_harmonics, case.face_step, case.precision, case.td_steps,
                         case.spectral_implicit)
        for k in range(4):
            c.walls[k] = Wall(*[float(x) for x in case.walls[k]])
        self.c = c


NOALLOC_MAX_DOUBLES = 1 << 19


def harmonic_noalloc(nx, ny, nu, nv, u, wu, v, wv, nt, h, b, k, re, im, stream=None) -> int:
    """k-th harmonic of the 8 fields from a state already in device memory, without a handle or any device
    allocation (see hbugks_harmonic_noalloc in include/hbugks.h).  Array arguments are CUDA tensors (FP64,
    canonical layout); re and im are written in place.  Returns the status code."""
    def ptr(t):
        return C.c_void_p(t.data_ptr())
    st = stream.cuda_stream if stream is not None else 0
    return int(lib().hbugks_harmonic_noalloc(nx, ny, nu, nv, ptr(u), ptr(wu), ptr(v), ptr(wv), nt, ptr(h), ptr(b),
                                             k, ptr(re), ptr(im), C.c_void_p(st)))


def workspace_bytes(cases: Sequence) -> int:
    args = [_CaseArgs(c) for c in cases]
    arr = (Case * len(args))(*[a.c for a in args])
    return int(lib().hbugks_workspace_bytes(len(args), arr))


class Solver:
    """A handle over one or more cavity cases (a batch), with its device workspace owned by a torch tensor."""

    def __init__(self, cases, device: str = "cuda:0", stream=None, workspace_fill: int | None = None):
        """workspace_fill: a byte value written over the whole workspace before the handle is created (the
        tests fill it with 0xFF, NaN in both precisions, to show that nothing reads memory it has not written)."""
        import torch
        if not isinstance(cases, (list, tuple)):
            cases = [cases]
        self.cases = list(cases)
        self._args = [_CaseArgs(c) for c in self.cases]
        arr = (Case * len(self._args))(*[a.c for a in self._args])
        nbytes = int(lib().hbugks_workspace_bytes(len(self._args), arr))
        if nbytes == 0:
            raise HbugksError(EINVAL, "hbugks_workspace_bytes")
        self.device = torch.device(device)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        if workspace_fill is not None:
            self.workspace.fill_(int(workspace_fill))
            torch.cuda.synchronize(self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        _check(lib().hbugks_create(len(self._args), arr, C.c_void_p(aligned), nbytes,
                                   C.c_void_p(self.stream.cuda_stream), C.byref(h)), "hbugks_create")
        self.h = h
        self.workspace_bytes = nbytes

    # ------------------------------------------------------------------ lifecycle
    def destroy(self):
        if getattr(self, "h", None):
            lib().hbugks_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    # ------------------------------------------------------------------ state
    def set_wall(self, case_index: int, wall: int, values):
        w = Wall(*[float(x) for x in values])
        _check(lib().hbugks_set_wall(self.h, case_index, wall, C.byref(w)), "hbugks_set_wall")

    def init_uniform(self, case_index: int = -1, rho=1.0, u=0.0, v=0.0, T=1.0):
        _check(lib().hbugks_init_uniform(self.h, case_index, rho, u, v, T), "hbugks_init_uniform")

    def set_state(self, case_index: int, W, h, b):
        W, h, b = (np.ascontiguousarray(x, dtype=np.float64) for x in (W, h, b))
        c = self.cases[case_index]
        assert W.size == c.nt * c.nc * 4 and h.size == c.nt * c.nc * c.nvel and b.size == h.size
        _check(lib().hbugks_set_state(self.h, case_index, _dp(W), _dp(h), _dp(b)), "hbugks_set_state")

    def get_state(self, case_index: int = 0):
        c = self.cases[case_index]
        W = np.zeros((c.nt, c.nc, 4))
        h = np.zeros((c.nt, c.nc, c.nvel))
        b = np.zeros_like(h)
        _check(lib().hbugks_get_state(self.h, case_index, _dp(W), _dp(h), _dp(b)), "hbugks_get_state")
        return W, h, b

    def get_W(self, case_index: int = 0) -> np.ndarray:
        """Conservative variables W[level][cell][4] only (no copy of the distributions)."""
        c = self.cases[case_index]
        W = np.zeros((c.nt, c.nc, 4))
        _check(lib().hbugks_get_state(self.h, case_index, _dp(W), None, None), "hbugks_get_state")
        return W

    # ------------------------------------------------------------------ iteration
    def iterate(self, max_iters: int, tol_rho: float = 0.0):
        """Returns (status, iterations per case, last residual per case (ncases, 4))."""
        n = len(self.cases)
        its = (C.c_int * n)()
        res = np.zeros((n, 4))
        rc = lib().hbugks_iterate(self.h, int(max_iters), float(tol_rho), its, _dp(res))
        _check(rc, "hbugks_iterate", allow=(OK, NOT_CONVERGED, DIVERGED, TIMEOUT))
        return rc, np.array(its[:], dtype=np.int64), res

    def set_loop_mode(self, mode: int):
        """0: device-side loop (one graph launch per call), 1: host-polled graphs of 16 iterations."""
        _check(lib().hbugks_set_loop_mode(self.h, int(mode)), "hbugks_set_loop_mode")

    def copy_state_from(self, case_index: int, other: "Solver", other_case: int = 0):
        """Take the state of `other`'s case (converted to this handle's precision); see hbugks_copy_state."""
        _check(lib().hbugks_copy_state(self.h, case_index, other.h, other_case), "hbugks_copy_state")

    def test_expire_wait(self):
        """Make the next iteration's micro update report its first (completed) wait as expired."""
        _check(lib().hbugks_test_expire_wait(self.h), "hbugks_test_expire_wait")

    def enqueue_iterations(self, n: int):
        _check(lib().hbugks_enqueue_iterations(self.h, int(n)), "hbugks_enqueue_iterations")

    def set_active(self, flags):
        arr = (C.c_int * len(self.cases))(*[int(bool(f)) for f in flags])
        _check(lib().hbugks_set_active(self.h, arr), "hbugks_set_active")

    def residual_history(self, case_index: int, n: int):
        out = np.zeros((n, 4))
        _check(lib().hbugks_residual_history(self.h, case_index, n, _dp(out)), "hbugks_residual_history")
        return out

    def iteration_count(self, case_index: int = 0) -> int:
        return int(lib().hbugks_iteration_count(self.h, case_index))

    def profile_kernels(self, n: int):
        """Average ms per iteration of (face moments, face parameters, macro update, micro update, residual),
        from CUDA events around each launch on the stream the kernels run on."""
        ms = np.zeros(5)
        _check(lib().hbugks_profile_kernels(self.h, int(n), _dp(ms)), "hbugks_profile_kernels")
        return ms

    def launches_per_iteration(self) -> int:
        return int(lib().hbugks_launches_per_iteration(self.h))

    def tile_shape(self, case_index: int = 0) -> tuple[int, int]:
        """Micro-update tile (cells along x, y per CTA) chosen for a case by the autotuner or pinned."""
        tx, ty = C.c_int(0), C.c_int(0)
        _check(lib().hbugks_get_tile_shape(self.h, case_index, C.byref(tx), C.byref(ty)), "get_tile_shape")
        return tx.value, ty.value

    def set_tile_shape(self, case_index: int, tx: int, ty: int) -> None:
        """Pin the micro-update tile of a case (4x4, 4x2, 2x2 or 8x4, one velocity block per CTA)."""
        _check(lib().hbugks_set_tile_shape(self.h, case_index, tx, ty), "set_tile_shape")

    def micro_variant(self, case_index: int = 0) -> tuple[int, int, int]:
        """Micro-update variant of a case: tile (tx, ty) and velocity blocks per CTA."""
        tx, ty, vpl = C.c_int(0), C.c_int(0), C.c_int(0)
        _check(lib().hbugks_get_micro_variant(self.h, case_index, C.byref(tx), C.byref(ty), C.byref(vpl)),
               "get_micro_variant")
        return tx.value, ty.value, vpl.value

    def set_micro_variant(self, case_index: int, tx: int, ty: int, vpl: int) -> None:
        """Pin the micro-update variant of a case (a tile with 1 velocity block per CTA, or 4x2 with 2)."""
        _check(lib().hbugks_set_micro_variant(self.h, case_index, tx, ty, vpl), "set_micro_variant")

    # ------------------------------------------------------------------ fields
    def level_fields(self, case_index: int, level: int):
        c = self.cases[case_index]
        out = np.zeros((8, c.nc))
        _check(lib().hbugks_get_level_fields(self.h, case_index, level, _dp(out)), "hbugks_get_level_fields")
        return out

    def harmonic(self, case_index: int, k: int):
        c = self.cases[case_index]
        re = np.zeros((8, c.nc))
        im = np.zeros((8, c.nc))
        _check(lib().hbugks_get_harmonic(self.h, case_index, k, _dp(re), _dp(im)), "hbugks_get_harmonic")
        return re + 1j * im
