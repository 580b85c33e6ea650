"""FP64 CPU oracle of the explicit finite-volume hydro stage update.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
CUDA library never links, loads or calls it, and this package never imports
the CUDA library.

The arithmetic lives in ``hard_oracle.c`` (plain C, FP64, ``-ffp-contract=off``
so every operation is a separately rounded IEEE operation on x86 and Arm).
This module only builds it and marshals numpy arrays through ctypes.

Pinned by ``tests/test_oracle_*.py`` (exact Riemann solutions, conservation,
mirror symmetry, convergence order, HLLC unit properties, Heun form).  The
HLLC wave-speed choice (Davis bounds) and the unsplit CFL rule are
conventions the paper does not fix; they are exercised but not pinned by an
independent result ("parity unpinned" for those two choices only).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hard_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhard_oracle.so")
_lock = threading.Lock()
_lib = None

BC_PERIODIC, BC_OUTFLOW, BC_REFLECT = 0, 1, 2
SCHEME_PLM_HLLC, SCHEME_WENO5Z_HLL = 0, 1
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def compile_oracle(src: str = _SRC, out: str = _LIB_PATH, extra=()) -> str:
    """Compile the C oracle into a shared library (OpenMP over cells)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-shared", "-fPIC", *extra, src, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def _declare(lib):
    lib.orc_minmod.restype = ctypes.c_double
    lib.orc_minmod.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.orc_hllc.restype = None
    lib.orc_hllc.argtypes = [_D, _D, ctypes.c_double, _D]
    lib.orc_hll.restype = None
    lib.orc_hll.argtypes = [_D, _D, ctypes.c_double, _D]
    lib.orc_weno5z.restype = ctypes.c_double
    lib.orc_weno5z.argtypes = [_D]
    lib.orc_rad_exchange.restype = ctypes.c_int
    lib.orc_rad_exchange.argtypes = [ctypes.c_int, _D, ctypes.c_double, _D, _D]
    grid = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _I, ctypes.c_double]
    sgrid = [ctypes.c_int] + grid
    lib.orc_advect_E_step.restype = ctypes.c_int
    lib.orc_advect_E_step.argtypes = grid + [_D, _D, ctypes.c_double]
    lib.orc_rusanov_E.restype = ctypes.c_double
    lib.orc_rusanov_E.argtypes = [ctypes.c_double] * 4
    lib.orc_rhs_E.restype = ctypes.c_int
    lib.orc_rhs_E.argtypes = grid + [_D, _D, _D]
    lib.orc_rhs_s.restype = ctypes.c_int
    lib.orc_rhs_s.argtypes = sgrid + [_D, _D]
    lib.orc_stage_s.restype = ctypes.c_int
    lib.orc_stage_s.argtypes = sgrid + [ctypes.c_int, _D, _D, _D, ctypes.c_double]
    lib.orc_step_s.restype = ctypes.c_int
    lib.orc_step_s.argtypes = sgrid + [_D, _D, ctypes.c_double]
    lib.orc_run_s.restype = ctypes.c_int
    lib.orc_run_s.argtypes = sgrid + [_D, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, _D]
    lib.orc_run_fixed_s.restype = ctypes.c_int
    lib.orc_run_fixed_s.argtypes = sgrid + [_D, ctypes.c_int, _D]
    lib.orc_rhs.restype = ctypes.c_int
    lib.orc_rhs.argtypes = grid + [_D, _D]
    lib.orc_stage.restype = ctypes.c_int
    lib.orc_stage.argtypes = grid + [ctypes.c_int, _D, _D, _D, ctypes.c_double]
    lib.orc_step.restype = ctypes.c_int
    lib.orc_step.argtypes = grid + [_D, _D, ctypes.c_double]
    lib.orc_step_heun.restype = ctypes.c_int
    lib.orc_step_heun.argtypes = grid + [_D, _D, ctypes.c_double]
    lib.orc_max_rate.restype = ctypes.c_double
    lib.orc_max_rate.argtypes = grid + [_D]
    lib.orc_run.restype = ctypes.c_int
    lib.orc_run.argtypes = grid + [_D, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, _D]
    lib.orc_run_fixed.restype = ctypes.c_int
    lib.orc_run_fixed.argtypes = grid + [_D, ctypes.c_int, _D]
    lib.orc_totals.restype = None
    lib.orc_totals.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D]
    lib.orc_set_threads.restype = None
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    lib.orc_get_threads.restype = ctypes.c_int
    lib.orc_get_threads.argtypes = []
    six = [ctypes.c_double] * 7
    lib.orc_riemann_star.restype = ctypes.c_int
    lib.orc_riemann_star.argtypes = six + [_D, _D]
    lib.orc_riemann_sample.restype = ctypes.c_int
    lib.orc_riemann_sample.argtypes = six + [ctypes.c_double, _D]
    lib.orc_riemann_extent.restype = ctypes.c_int
    lib.orc_riemann_extent.argtypes = six + [_D, _D]
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library.  A non-default ``path``
    (or the HARD_ORACLE_LIB environment variable) loads a separately built
    copy; the mutation tests use it to run the pins on a planted mistake."""
    global _lib
    if path is None and os.environ.get("HARD_ORACLE_LIB"):
        path = os.environ["HARD_ORACLE_LIB"]      # a separately built copy
    if path is not None:
        with _lock:
            if _lib is None or getattr(_lib, "_path", None) != path:
                _lib = _declare(ctypes.CDLL(path))
                _lib._path = path
        return _lib
    with _lock:
        if _lib is None:
            stale = (not os.path.exists(_LIB_PATH)
                     or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
            if stale:
                compile_oracle()
            _lib = _declare(ctypes.CDLL(_LIB_PATH))
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _c64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Grid:
    """Uniform Cartesian grid: ``shape=(nz, ny, nx)``, extents ``(lx, ly, lz)``,
    boundary kinds per face ``(x-, x+, y-, y+, z-, z+)``; ``scheme`` 0 is
    PLM-minmod + HLLC, 1 is WENO5-Z + HLL (three cells per active axis at
    least)."""

    def __init__(self, shape, gamma, bc=BC_PERIODIC, extent=(1.0, 1.0, 1.0), lib=None,
                 scheme=SCHEME_PLM_HLLC):
        nz, ny, nx = shape
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.gamma = float(gamma)
        bc6 = [bc] * 6 if np.isscalar(bc) else list(bc)
        if len(bc6) != 6:
            raise ValueError("bc needs one kind or six (x-, x+, y-, y+, z-, z+)")
        self.bc6 = np.array(bc6, dtype=np.int32)
        self.extent = tuple(float(e) for e in extent)
        self.dxyz = np.array([self.extent[0] / self.nx, self.extent[1] / self.ny,
                              self.extent[2] / self.nz], dtype=np.float64)
        self.lib = lib if lib is not None else load()
        self.scheme = int(scheme)
        if self.scheme not in (SCHEME_PLM_HLLC, SCHEME_WENO5Z_HLL):
            raise ValueError("scheme must be 0 (PLM + HLLC) or 1 (WENO5-Z + HLL)")
        if self.scheme == SCHEME_WENO5Z_HLL and any(1 < n < 3 for n in (self.nx, self.ny, self.nz)):
            raise ValueError("WENO5-Z needs at least three cells along every active axis")

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def _g(self):
        return (self.scheme, self.nx, self.ny, self.nz, _dp(self.dxyz),
                self.bc6.ctypes.data_as(_I), self.gamma)

    def _g0(self):
        return self._g()[1:]

    def _check(self, U):
        U = _c64(U)
        if U.shape != (5, self.nz, self.ny, self.nx):
            raise ValueError(f"U must be (5,{self.nz},{self.ny},{self.nx}), got {U.shape}")
        return U

    def rhs(self, U):
        U = self._check(U)
        L = np.empty_like(U)
        self.lib.orc_rhs_s(*self._g(), _dp(U), _dp(L))
        return L

    def stage(self, stage, U0, Ucur, dt):
        U0, Ucur = self._check(U0), self._check(Ucur)
        out = np.empty_like(Ucur)
        self.lib.orc_stage_s(*self._g(), int(stage), _dp(U0), _dp(Ucur), _dp(out), float(dt))
        return out

    def step(self, U, dt):
        U = self._check(U)
        out = np.empty_like(U)
        self.lib.orc_step_s(*self._g(), _dp(U), _dp(out), float(dt))
        return out

    def step_heun(self, U, dt):
        U = self._check(U)
        out = np.empty_like(U)
        if self.scheme != SCHEME_PLM_HLLC:
            raise NotImplementedError("the Heun-form cross-check covers scheme 0")
        self.lib.orc_step_heun(*self._g0(), _dp(U), _dp(out), float(dt))
        return out

    def max_rate(self, U):
        U = self._check(U)
        return float(self.lib.orc_max_rate(*self._g0(), _dp(U)))

    def run(self, U, nsteps, cfl, t_end=0.0, t0=0.0):
        """Returns (U_final, t_final, dt_schedule)."""
        U = self._check(U).copy()
        t = np.array([t0], dtype=np.float64)
        dts = np.zeros(max(int(nsteps), 1), dtype=np.float64)
        n = self.lib.orc_run_s(*self._g(), _dp(U), int(nsteps), float(cfl), float(t_end),
                               _dp(t), _dp(dts))
        if n < 0:
            raise FloatingPointError("non-positive or non-finite signal rate")
        return U, float(t[0]), dts[:n].copy()

    def run_fixed(self, U, dts):
        U = self._check(U).copy()
        dts = _c64(dts)
        self.lib.orc_run_fixed_s(*self._g(), _dp(U), int(dts.size), _dp(dts))
        return U

    def advect_E(self, U, E, dt):
        """One Heun step of the radiation energy advection (WENO5-Z states,
        Rusanov flux) with U's velocity field held fixed; returns E'."""
        U = self._check(U)
        E = _c64(E).copy()
        if E.shape != (self.nz, self.ny, self.nx):
            raise ValueError("E must have the cell shape")
        if self.lib.orc_advect_E_step(*self._g0(), _dp(U), _dp(E), float(dt)):
            raise ValueError("the advection needs three cells along every active axis")
        return E

    def rhs_E(self, U, E):
        U = self._check(U)
        E = _c64(E)
        L = np.empty_like(E)
        if self.lib.orc_rhs_E(*self._g0(), _dp(U), _dp(E), _dp(L)):
            raise ValueError("the advection needs three cells along every active axis")
        return L

    def totals(self, U):
        U = self._check(U)
        out = np.zeros(5, dtype=np.float64)
        self.lib.orc_totals(self.nx, self.ny, self.nz, _dp(self.dxyz), _dp(U), _dp(out))
        return out


def minmod(a, b, lib=None):
    return float((lib or load()).orc_minmod(float(a), float(b)))


def weno5z(v, lib=None):
    """WENO5-Z value at the right face of the middle of five cell averages."""
    v = _c64(v)
    if v.shape != (5,):
        raise ValueError("weno5z takes five cell averages")
    return float((lib or load()).orc_weno5z(_dp(v)))


def rad_exchange(U, Er, dt, c, kappa, a_rad, cv, lib=None):
    """One backward-Euler step of the radiative heating / cooling exchange on
    the conserved state U (5, ...) and the radiation energy density Er (...).
    Returns (U', Er', largest Newton step count)."""
    U = _c64(U).copy()
    Er = _c64(Er).copy()
    n = Er.size
    if U.shape[0] != 5 or U[0].size != n:
        raise ValueError("U must be (5, ...) with Er of the cell shape")
    prm = np.array([c, kappa, a_rad, cv], dtype=np.float64)
    it = (lib or load()).orc_rad_exchange(int(n), _dp(prm), float(dt), _dp(U), _dp(Er))
    return U, Er, int(it)


def rusanov_E(EL, ER, uL, uR, lib=None):
    """Rusanov flux of E u from the face states."""
    return float((lib or load()).orc_rusanov_E(float(EL), float(ER), float(uL), float(uR)))


def hll(WL, WR, gamma, lib=None):
    """x-normal HLL flux of two primitive states (rho, u, v, w, p)."""
    WL, WR = _c64(WL), _c64(WR)
    F = np.zeros(5)
    (lib or load()).orc_hll(_dp(WL), _dp(WR), float(gamma), _dp(F))
    return F


def hllc(WL, WR, gamma, lib=None):
    """x-normal HLLC flux of primitive states (rho, u, v, w, p)."""
    WL, WR = _c64(WL), _c64(WR)
    F = np.zeros(5, dtype=np.float64)
    (lib or load()).orc_hllc(_dp(WL), _dp(WR), float(gamma), _dp(F))
    return F


def riemann_star(WL3, WR3, gamma, lib=None):
    """Exact star pressure and velocity for 1D states (rho, u, p)."""
    ps, us = ctypes.c_double(), ctypes.c_double()
    rc = (lib or load()).orc_riemann_star(*map(float, WL3), *map(float, WR3), float(gamma),
                                         ctypes.byref(ps), ctypes.byref(us))
    if rc:
        raise ValueError("vacuum-generating or unsolvable Riemann data")
    return ps.value, us.value


def riemann_sample(WL3, WR3, gamma, xi, lib=None):
    """Exact solution (rho, u, p) at similarity coordinates ``xi`` (array)."""
    lib = lib or load()
    xi = np.atleast_1d(_c64(xi))
    out = np.empty((xi.size, 3), dtype=np.float64)
    w = np.zeros(3, dtype=np.float64)
    args = (*map(float, WL3), *map(float, WR3), float(gamma))
    for q, s in enumerate(xi):
        if lib.orc_riemann_sample(*args, float(s), _dp(w)):
            raise ValueError("vacuum-generating or unsolvable Riemann data")
        out[q] = w
    return out


def riemann_extent(WL3, WR3, gamma, lib=None):
    lo, hi = ctypes.c_double(), ctypes.c_double()
    rc = (lib or load()).orc_riemann_extent(*map(float, WL3), *map(float, WR3), float(gamma),
                                           ctypes.byref(lo), ctypes.byref(hi))
    if rc:
        raise ValueError("vacuum-generating or unsolvable Riemann data")
    return lo.value, hi.value


def set_threads(n: int):
    load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(load().orc_get_threads())


def cons_from_prim(W, gamma):
    """Primitive (rho, u, v, w, p) -> conserved, Eq. "fluxes" with p = (gamma-1) e."""
    W = _c64(W)
    rho, u, v, w, p = W
    return np.stack([rho, rho * u, rho * v, rho * w,
                     p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)])


def prim_from_cons(U, gamma):
    U = _c64(U)
    rho = U[0]
    u, v, w = U[1] / rho, U[2] / rho, U[3] / rho
    p = (gamma - 1.0) * (U[4] - 0.5 * rho * (u * u + v * v + w * w))
    return np.stack([rho, u, v, w, p])
