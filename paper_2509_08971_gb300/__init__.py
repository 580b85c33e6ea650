"""GB300 (sm_103a) explicit finite-volume hydro stage update.

Thin Python binding of the C ABI in ``include/hard_hydro.h``: the functions
below carry the C names and only marshal arguments; every step of the update
runs in ``libhard_hydro.so`` (built in-tree by :mod:`.build`).  There is no
CPU fallback: without the library every call raises.

``HardHydro`` wraps a handle for torch tensors of shape (5, nz, ny, nx) on the
current CUDA device and stream.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhard_hydro.so")

HARD_BC_PERIODIC, HARD_BC_OUTFLOW, HARD_BC_REFLECT, HARD_BC_HALO = 0, 1, 2, 3
HARD_F32, HARD_F64 = 0, 1
HARD_KERNEL_FUSED, HARD_KERNEL_PLAIN = 0, 1
HARD_SCHEME_PLM_HLLC, HARD_SCHEME_WENO5Z_HLL = 0, 1
HARD_OK, HARD_EINVAL, HARD_ENOMEM, HARD_ECUDA = 0, -1, -2, -3
HARD_ENONPHYS, HARD_ETIMEOUT, HARD_EUNSUPPORTED = -4, -5, -6

_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class HardHydroError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = hard_hydro_strerror(code) if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


def _declare(lib):
    sig = {
        "hard_hydro_create": (_vp, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_int]),
        "hard_hydro_set": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, _ip]),
        "hard_hydro_set_kernel": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
        "hard_hydro_set_scheme": (ctypes.c_int, [_vp, ctypes.c_int]),
        "hard_hydro_rad_exchange": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double,
                                                   ctypes.POINTER(ctypes.c_double), _vp]),
        "hard_hydro_advect_E": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, _vp]),
        "hard_hydro_fld_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_double), _vp]),
        "hard_hydro_tile_count": (ctypes.c_int, [_vp]),
        "hard_hydro_tile_info": (ctypes.c_int, [_vp, ctypes.c_int, _ip]),
        "hard_hydro_stage": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_double,
                                            _vp]),
        "hard_hydro_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, _vp]),
        "hard_hydro_cfl_dt": (ctypes.c_int, [_vp, _vp, ctypes.c_double, _dp, _vp]),
        "hard_hydro_cfl_dt_dev": (ctypes.c_int, [_vp, _vp, ctypes.c_double, _vp, _vp]),
        "hard_hydro_advance": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_double,
                                              ctypes.c_double, _vp, _vp, _vp, _vp]),
        "hard_hydro_advance_host": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_double,
                                                   ctypes.c_double, _dp, _vp]),
        "hard_hydro_totals": (ctypes.c_int, [_vp, _vp, _dp, _vp]),
        "hard_hydro_step_noalloc": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, _vp]),
        "hard_hydro_step_backward": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_double, _vp,
                                                    _vp]),
        "hard_hydro_get_error": (ctypes.c_int, [_vp]),
        "hard_hydro_noalloc_get_error": (ctypes.c_int, []),
        "hard_hydro_set_cells": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double]),
        "hard_hydro_stage_ex": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_double,
                                               _vp, _vp, _vp]),
        "hard_hydro_set_zghost": (ctypes.c_int, [_vp, _vp, _vp]),
        "hard_hydro_pack_zhalo": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
        "hard_hydro_set_zghost_adjoint": (ctypes.c_int, [_vp, _vp, _vp]),
        "hard_hydro_stage_vjp_faces": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp,
                                                      ctypes.c_double, _vp, _vp]),
        "hard_hydro_add_zghost_cotangent": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
        "hard_hydro_stage_vjp_cells": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp,
                                                      ctypes.c_int, _vp, _vp, _vp]),
        "hard_hydro_local_rate": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
        "hard_hydro_finalize_dt": (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_double,
                                                  _vp, _vp, _vp]),
        "hard_batch_create": (_vp, [ctypes.c_int, _ip, _ip, _ip, _dp, _ip, ctypes.c_int]),
        "hard_batch_offset": (ctypes.c_longlong, [_vp, ctypes.c_int]),
        "hard_batch_elements": (ctypes.c_longlong, [_vp]),
        "hard_batch_tile_count": (ctypes.c_int, []),
        "hard_batch_set_tile": (ctypes.c_int, [_vp, ctypes.c_int]),
        "hard_hydro_step_batched": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_double, _vp,
                                                   _vp]),
        "hard_batch_get_error": (ctypes.c_int, [_vp]),
        "hard_batch_destroy": (None, [_vp]),
        "hard_hydro_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "hard_hydro_destroy": (None, [_vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def lib():
    """The loaded CUDA library.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with paper_2509_08971_gb300.build.build() "
                "(nvcc, sm_103a); there is no CPU fallback")
        _lib = _declare(ctypes.CDLL(LIB_PATH))
    return _lib


# ---- C names, argument marshalling only ------------------------------------

def hard_hydro_create(nx, ny, nz, gamma, bc):
    return lib().hard_hydro_create(int(nx), int(ny), int(nz), float(gamma), int(bc))


def hard_hydro_set(h, dtype, lx, ly, lz, bc_per_face=None):
    arr = None if bc_per_face is None else (ctypes.c_int * 6)(*[int(b) for b in bc_per_face])
    return lib().hard_hydro_set(h, int(dtype), float(lx), float(ly), float(lz), arr)


def hard_hydro_set_kernel(h, kernel, tile):
    return lib().hard_hydro_set_kernel(h, int(kernel), int(tile))


def hard_hydro_set_scheme(h, scheme):
    return lib().hard_hydro_set_scheme(h, int(scheme))


def hard_hydro_set_cells(h, dx, dy, dz):
    return lib().hard_hydro_set_cells(h, float(dx), float(dy), float(dz))


def hard_hydro_stage_ex(h, stage, U0, Ucur, Uout, dt, dt_dev, rate_dev, stream):
    return lib().hard_hydro_stage_ex(h, int(stage), U0, Ucur, Uout, float(dt), dt_dev, rate_dev,
                                     stream)


def hard_hydro_set_zghost(h, ghost_lo, ghost_hi):
    return lib().hard_hydro_set_zghost(h, ghost_lo, ghost_hi)


def hard_hydro_pack_zhalo(h, U, send_lo, send_hi, stream):
    return lib().hard_hydro_pack_zhalo(h, U, send_lo, send_hi, stream)


def hard_hydro_set_zghost_adjoint(h, gw_lo, gw_hi):
    return lib().hard_hydro_set_zghost_adjoint(h, gw_lo, gw_hi)


def hard_hydro_stage_vjp_faces(h, stage, Uc, G, dt, g_gamma, stream):
    return lib().hard_hydro_stage_vjp_faces(h, int(stage), Uc, G, float(dt), g_gamma, stream)


def hard_hydro_add_zghost_cotangent(h, from_lo, from_hi, stream):
    return lib().hard_hydro_add_zghost_cotangent(h, from_lo, from_hi, stream)


def hard_hydro_stage_vjp_cells(h, stage, Uc, G, gUc, accumulate, gU0, g_gamma, stream):
    return lib().hard_hydro_stage_vjp_cells(h, int(stage), Uc, G, gUc, int(bool(accumulate)),
                                            gU0, g_gamma, stream)


def hard_hydro_local_rate(h, U, rate_dev, stream):
    return lib().hard_hydro_local_rate(h, U, rate_dev, stream)


def hard_hydro_finalize_dt(h, rate_dev, cfl, t_end, t_dev, dt_dev, stream):
    return lib().hard_hydro_finalize_dt(h, rate_dev, float(cfl), float(t_end), t_dev, dt_dev,
                                        stream)


def hard_hydro_noalloc_get_error():
    return lib().hard_hydro_noalloc_get_error()


def hard_hydro_advect_E(h, U, Er, dt, stream):
    return lib().hard_hydro_advect_E(h, U, Er, float(dt), stream)


def hard_hydro_fld_step(h, U, Er, dt, c, kappa, rtol, max_cycles, stream):
    """Returns (rc, cycles, relative residual)."""
    cyc = ctypes.c_int(0)
    res = ctypes.c_double(-1.0)
    rc = lib().hard_hydro_fld_step(h, U, Er, float(dt), float(c), float(kappa), float(rtol),
                                   int(max_cycles), ctypes.byref(cyc), ctypes.byref(res), stream)
    return rc, cyc.value, res.value


def hard_hydro_rad_exchange(h, U, Er, dt, prm, stream):
    arr = (ctypes.c_double * 4)(*[float(v) for v in prm])
    return lib().hard_hydro_rad_exchange(h, U, Er, float(dt), arr, stream)


def hard_hydro_tile_count(h):
    return lib().hard_hydro_tile_count(h)


def hard_hydro_tile_info(h, tile):
    out = (ctypes.c_int * 4)()
    rc = lib().hard_hydro_tile_info(h, int(tile), out)
    return rc, tuple(out)


def hard_hydro_stage(h, stage, U0, Ucur, Uout, dt, stream):
    return lib().hard_hydro_stage(h, int(stage), U0, Ucur, Uout, float(dt), stream)


def hard_hydro_step(h, U_in, U_out, dt, stream):
    return lib().hard_hydro_step(h, U_in, U_out, float(dt), stream)


def hard_hydro_cfl_dt(h, U, cfl, stream):
    dt = ctypes.c_double(0.0)
    rc = lib().hard_hydro_cfl_dt(h, U, float(cfl), ctypes.byref(dt), stream)
    return rc, dt.value


def hard_hydro_cfl_dt_dev(h, U, cfl, dt_dev, stream):
    return lib().hard_hydro_cfl_dt_dev(h, U, float(cfl), dt_dev, stream)


def hard_hydro_advance(h, U, nsteps, cfl, t_end, t_dev, dt_log_dev, totals_log_dev, stream):
    return lib().hard_hydro_advance(h, U, int(nsteps), float(cfl), float(t_end), t_dev,
                                    dt_log_dev, totals_log_dev, stream)


def hard_hydro_advance_host(h, U_host_in, U_host_out, nsteps, cfl, t_end, t_host, stream):
    t = ctypes.c_double(float(t_host))
    rc = lib().hard_hydro_advance_host(h, U_host_in, U_host_out, int(nsteps), float(cfl),
                                       float(t_end), ctypes.byref(t), stream)
    return rc, t.value


def hard_hydro_totals(h, U, stream):
    out = (ctypes.c_double * 5)()
    rc = lib().hard_hydro_totals(h, U, out, stream)
    return rc, list(out)


def hard_hydro_step_noalloc(h, U_in, U_out, dt, stream):
    """hard_hydro_step without any device allocation: the intermediate stage
    lives in the library's fixed 64 MiB device array (see the C header)."""
    return lib().hard_hydro_step_noalloc(h, U_in, U_out, float(dt), stream)


def hard_batch_create(nprob, nx, ny, nz, gamma, bc, dtype):
    ia = lambda v: (ctypes.c_int * nprob)(*[int(x) for x in v])
    da = (ctypes.c_double * nprob)(*[float(x) for x in gamma])
    return lib().hard_batch_create(int(nprob), ia(nx), ia(ny), ia(nz) if nz is not None else None,
                                   da, ia(bc), int(dtype))


def hard_batch_offset(b, p):
    return lib().hard_batch_offset(b, int(p))


def hard_batch_elements(b):
    return lib().hard_batch_elements(b)


def hard_batch_tile_count():
    return lib().hard_batch_tile_count()


def hard_batch_set_tile(b, tile):
    return lib().hard_batch_set_tile(b, int(tile))


def hard_hydro_step_batched(b, U_packed, nsteps, cfl, t_dev, stream):
    return lib().hard_hydro_step_batched(b, U_packed, int(nsteps), float(cfl), t_dev, stream)


def hard_batch_get_error(b):
    return lib().hard_batch_get_error(b)


def hard_batch_destroy(b):
    if b:
        lib().hard_batch_destroy(b)


def hard_hydro_step_backward(h, U_in, gU_out, gU_in, dt, g_gamma, stream):
    return lib().hard_hydro_step_backward(h, U_in, gU_out, gU_in, float(dt), g_gamma, stream)


def hard_hydro_get_error(h):
    return lib().hard_hydro_get_error(h)


def hard_hydro_strerror(code):
    return lib().hard_hydro_strerror(int(code)).decode()


def hard_hydro_destroy(h):
    if h:
        lib().hard_hydro_destroy(h)


def check(rc, what=""):
    if rc != HARD_OK:
        raise HardHydroError(rc, what)
    return rc


# ---- torch convenience ----------------------------------------------------

class HardHydro:
    """A mesh handle bound to torch tensors U of shape (5, nz, ny, nx)."""

    def __init__(self, shape, gamma, bc=HARD_BC_PERIODIC, dtype=None, extent=(1.0, 1.0, 1.0),
                 kernel=HARD_KERNEL_FUSED, tile=-1, scheme=HARD_SCHEME_PLM_HLLC):
        import torch
        self.torch = torch
        nz, ny, nx = (int(s) for s in shape)
        self.shape = (nz, ny, nx)
        self.gamma = float(gamma)
        self.dtype = dtype or torch.float32
        if self.dtype not in (torch.float32, torch.float64):
            raise ValueError("dtype must be torch.float32 or torch.float64")
        bc6 = [bc] * 6 if isinstance(bc, int) else list(bc)
        self.bc6 = tuple(int(b) for b in bc6)
        self.extent = tuple(float(e) for e in extent)
        self.scheme = int(scheme)
        self.h = hard_hydro_create(nx, ny, nz, gamma, bc6[0])
        if not self.h:
            raise HardHydroError(HARD_EINVAL, "hard_hydro_create")
        check(hard_hydro_set(self.h, HARD_F64 if self.dtype == torch.float64 else HARD_F32,
                             *extent, bc6), "hard_hydro_set")
        check(hard_hydro_set_kernel(self.h, kernel, tile), "hard_hydro_set_kernel")
        check(hard_hydro_set_scheme(self.h, scheme), "hard_hydro_set_scheme")

    def __del__(self):
        h, self.h = getattr(self, "h", None), None
        if h and _lib is not None:
            hard_hydro_destroy(h)

    def set_kernel(self, kernel, tile=-1):
        check(hard_hydro_set_kernel(self.h, kernel, tile), "hard_hydro_set_kernel")

    def set_scheme(self, scheme):
        check(hard_hydro_set_scheme(self.h, scheme), "hard_hydro_set_scheme")
        self.scheme = int(scheme)

    def advect_E(self, U, Er, dt):
        """In place on Er: one Heun step of the radiation energy advection."""
        if not (Er.is_cuda and Er.is_contiguous() and Er.dtype == self.dtype
                and tuple(Er.shape) == self.shape):
            raise ValueError(f"Er must be a contiguous {self.dtype} CUDA tensor of shape {self.shape}")
        check(hard_hydro_advect_E(self.h, self._check(U), Er.data_ptr(), dt, self._stream()),
              "hard_hydro_advect_E")
        return Er

    def fld_step(self, U, Er, dt, c, kappa, rtol=1e-8, max_cycles=50):
        """In place on Er: one implicit flux-limited diffusion step.  Returns
        (cycles, relative residual)."""
        if not (Er.is_cuda and Er.is_contiguous() and Er.dtype == self.dtype
                and tuple(Er.shape) == self.shape):
            raise ValueError(f"Er must be a contiguous {self.dtype} CUDA tensor of shape {self.shape}")
        rc, cyc, res = hard_hydro_fld_step(self.h, self._check(U), Er.data_ptr(), dt, c, kappa,
                                           rtol, max_cycles, self._stream())
        check(rc, "hard_hydro_fld_step")
        return cyc, res

    def rad_exchange(self, U, Er, dt, c, kappa, a_rad, cv):
        """In place on U (its E_total field) and Er: one backward-Euler step of
        the radiative heating / cooling exchange."""
        if not (Er.is_cuda and Er.is_contiguous() and Er.dtype == self.dtype
                and tuple(Er.shape) == self.shape):
            raise ValueError(f"Er must be a contiguous {self.dtype} CUDA tensor of shape {self.shape}")
        check(hard_hydro_rad_exchange(self.h, self._check(U), Er.data_ptr(), dt,
                                      (c, kappa, a_rad, cv), self._stream()),
              "hard_hydro_rad_exchange")
        return U, Er

    def tile_count(self):
        return hard_hydro_tile_count(self.h)

    def tile_info(self, tile):
        rc, info = hard_hydro_tile_info(self.h, tile)
        check(rc, "hard_hydro_tile_info")
        return info

    def _stream(self):
        return self.torch.cuda.current_stream().cuda_stream

    def _check(self, U):
        if not (U.is_cuda and U.is_contiguous() and U.dtype == self.dtype
                and tuple(U.shape) == (5, *self.shape)):
            raise ValueError(f"U must be a contiguous CUDA {self.dtype} tensor of shape "
                             f"{(5, *self.shape)}, got {tuple(U.shape)} {U.dtype} {U.device}")
        return U.data_ptr()

    def empty(self):
        return self.torch.empty((5, *self.shape), dtype=self.dtype, device="cuda")

    def stage(self, stage, U0, Ucur, dt, out=None):
        out = self.empty() if out is None else out
        p0 = self._check(U0) if U0 is not None else None
        check(hard_hydro_stage(self.h, stage, p0, self._check(Ucur), self._check(out), dt,
                               self._stream()), "hard_hydro_stage")
        return out

    def step(self, U, dt, out=None):
        out = self.empty() if out is None else out
        check(hard_hydro_step(self.h, self._check(U), self._check(out), dt, self._stream()),
              "hard_hydro_step")
        return out

    def cfl_dt(self, U, cfl):
        rc, dt = hard_hydro_cfl_dt(self.h, self._check(U), cfl, self._stream())
        check(rc, "hard_hydro_cfl_dt")
        return dt

    def advance(self, U, nsteps, cfl, t_end=0.0, t=None, log_dt=False, log_totals=False):
        """In place on U.  Returns (t_tensor, dt_log or None, totals_log or None),
        all device tensors (float64)."""
        torch = self.torch
        if t is None:
            t = torch.zeros((), dtype=torch.float64, device=U.device)
        dtl = torch.zeros(max(nsteps, 1), dtype=torch.float64, device=U.device) if log_dt else None
        tl = (torch.zeros((max(nsteps, 1), 5), dtype=torch.float64, device=U.device)
              if log_totals else None)
        check(hard_hydro_advance(self.h, self._check(U), nsteps, cfl, t_end, t.data_ptr(),
                                 dtl.data_ptr() if dtl is not None else None,
                                 tl.data_ptr() if tl is not None else None, self._stream()),
              "hard_hydro_advance")
        return t, dtl, tl

    def advance_host(self, U_host, nsteps, cfl, t_end=0.0, t0=0.0, out=None):
        """U_host: a contiguous host torch tensor (pinned for full bandwidth)."""
        out = U_host if out is None else out
        rc, t = hard_hydro_advance_host(self.h, U_host.data_ptr(), out.data_ptr(), nsteps, cfl,
                                        t_end, t0, self._stream())
        check(rc, "hard_hydro_advance_host")
        return out, t

    def totals(self, U):
        rc, out = hard_hydro_totals(self.h, self._check(U), self._stream())
        check(rc, "hard_hydro_totals")
        return out

    def step_backward(self, U, gU_out, dt, g_gamma, out=None):
        """VJP of one step at U with fixed dt; adds d/dgamma to g_gamma (device FP64 scalar)."""
        out = self.empty() if out is None else out
        check(hard_hydro_step_backward(self.h, self._check(U), self._check(gU_out),
                                       self._check(out), dt, g_gamma.data_ptr(), self._stream()),
              "hard_hydro_step_backward")
        return out

    def get_error(self):
        return hard_hydro_get_error(self.h)


class HardBatch:
    """Independent 1D/2D problems advanced together by one persistent launch.
    Problem p is nx[p] x ny[p] cells (ny = 1: 1D) with its own gamma and
    boundary kind; states live in one packed device tensor."""

    def __init__(self, nx, ny, gamma, bc=HARD_BC_OUTFLOW, dtype=None, tile=0):
        import torch
        self.torch = torch
        self.nprob = len(nx)
        self.nx = [int(v) for v in nx]
        self.ny = [int(v) for v in ny]
        self.dtype = dtype or torch.float32
        gam = [float(gamma)] * self.nprob if isinstance(gamma, (int, float)) else list(gamma)
        bcs = [int(bc)] * self.nprob if isinstance(bc, int) else list(bc)
        self.gammas = tuple(float(g) for g in gam)
        self.bcs = tuple(int(b) for b in bcs)
        self.b = hard_batch_create(self.nprob, self.nx, self.ny, [1] * self.nprob, gam, bcs,
                                   HARD_F64 if self.dtype == torch.float64 else HARD_F32)
        if not self.b:
            raise HardHydroError(HARD_EINVAL, "hard_batch_create")
        self.offsets = [hard_batch_offset(self.b, p) for p in range(self.nprob)]
        self.elements = hard_batch_elements(self.b)
        check(hard_batch_set_tile(self.b, tile), "hard_batch_set_tile")

    def __del__(self):
        b, self.b = getattr(self, "b", None), None
        if b and _lib is not None:
            hard_batch_destroy(b)

    def set_tile(self, tile):
        check(hard_batch_set_tile(self.b, tile), "hard_batch_set_tile")

    def empty(self):
        return self.torch.zeros(self.elements, dtype=self.dtype, device="cuda")

    def view(self, packed, p):
        """Problem p's state as a (5, 1, ny, nx) view of the packed tensor."""
        n = 5 * self.nx[p] * self.ny[p]
        o = self.offsets[p]
        return packed[o:o + n].view(5, 1, self.ny[p], self.nx[p])

    def pack(self, states):
        packed = self.empty()
        for p, U in enumerate(states):
            self.view(packed, p).copy_(self.torch.as_tensor(U, dtype=self.dtype))
        return packed

    def step(self, packed, nsteps, cfl, t=None):
        """Advance every problem by nsteps steps in place; returns t (device, FP64)."""
        torch = self.torch
        if t is None:
            t = torch.zeros(self.nprob, dtype=torch.float64, device=packed.device)
        if not (packed.is_cuda and packed.is_contiguous() and packed.dtype == self.dtype
                and packed.numel() == self.elements):
            raise ValueError("packed state must be a contiguous CUDA tensor of hard_batch_elements")
        check(hard_hydro_step_batched(self.b, packed.data_ptr(), nsteps, cfl, t.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream),
              "hard_hydro_step_batched")
        return t

    def capture(self, packed, nsteps, cfl, t):
        """A CUDA graph of one batched call on these buffers (replay() re-runs it)."""
        torch = self.torch
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                check(hard_hydro_step_batched(self.b, packed.data_ptr(), nsteps, cfl, t.data_ptr(),
                                              s.cuda_stream), "hard_hydro_step_batched")
        torch.cuda.current_stream().wait_stream(s)
        return g

    def tune(self, packed, cfl, steps=5, cache_path=None):
        """Pick the fastest batched tile set on this batch (autotune.tune_batch)."""
        from . import autotune
        return autotune.tune_batch(self, packed, cfl, steps=steps, cache_path=cache_path)

    def get_error(self):
        return hard_batch_get_error(self.b)
