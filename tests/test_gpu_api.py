"""GPU tests of the C ABI beyond element-wise parity: error paths, the device
status flag, full-size sampled parity in the benchmarked launch configuration,
determinism and tiling independence."""
import os

import numpy as np
import pytest

import hydro_inputs as H
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
hh = pytest.importorskip("paper_2509_08971_gb300")


def dev(U, dtype):
    return torch.tensor(np.ascontiguousarray(U), dtype=dtype, device="cuda")


def test_argument_errors():
    L = hh.lib()
    assert hh.hard_hydro_create(0, 4, 4, 1.4, 0) is None
    assert hh.hard_hydro_create(4, 4, 4, 1.0, 0) is None
    assert hh.hard_hydro_create(4, 4, 4, 1.4, 7) is None
    h = hh.hard_hydro_create(8, 8, 8, 1.4, 0)
    assert h
    s = torch.cuda.current_stream().cuda_stream
    U = torch.ones((5, 8, 8, 8), device="cuda")
    V = torch.empty_like(U)
    assert hh.hard_hydro_set(h, 5, 1, 1, 1) == hh.HARD_EINVAL
    assert hh.hard_hydro_set(h, 0, -1, 1, 1) == hh.HARD_EINVAL
    assert hh.hard_hydro_set(h, 0, 1, 1, 1, [0, 1, 0, 0, 0, 0]) == hh.HARD_EINVAL
    assert hh.hard_hydro_set_kernel(h, 3, 0) == hh.HARD_EINVAL
    assert hh.hard_hydro_set_kernel(h, 0, 99) == hh.HARD_EINVAL
    assert hh.hard_hydro_step(h, None, V.data_ptr(), 1e-3, s) == hh.HARD_EINVAL
    assert hh.hard_hydro_step(h, U.data_ptr(), V.data_ptr(), 0.0, s) == hh.HARD_EINVAL
    assert hh.hard_hydro_step(h, U.data_ptr(), V.data_ptr(), float("nan"), s) == hh.HARD_EINVAL
    assert hh.hard_hydro_step(h, U.data_ptr() + 4, V.data_ptr(), 1e-3, s) == hh.HARD_EINVAL
    assert hh.hard_hydro_stage(h, 3, None, U.data_ptr(), V.data_ptr(), 1e-3, s) == hh.HARD_EINVAL
    assert hh.hard_hydro_stage(h, 1, None, U.data_ptr(), U.data_ptr(), 1e-3, s) == hh.HARD_EINVAL
    assert hh.hard_hydro_stage(h, 2, None, U.data_ptr(), V.data_ptr(), 1e-3, s) == hh.HARD_EINVAL
    assert hh.hard_hydro_advance(h, U.data_ptr(), 1, 0.4, 1.0, None, None, None, s) == hh.HARD_EINVAL
    assert hh.hard_hydro_cfl_dt(h, U.data_ptr(), -1.0, s)[0] == hh.HARD_EINVAL
    assert hh.hard_hydro_strerror(hh.HARD_ENONPHYS).startswith("non-physical")
    hh.hard_hydro_destroy(h)
    del L


def test_nonphysical_input_sets_flag():
    shape = (4, 6, 8)
    U = H.prim_to_cons([np.ones(shape), np.zeros(shape), np.zeros(shape), np.zeros(shape),
                        np.ones(shape)], 1.4)
    U[0, 2, 3, 4] = -1.0                     # negative density
    m = hh.HardHydro(shape, 1.4, 0)
    out = m.step(dev(U, torch.float32), 1e-3)
    torch.cuda.synchronize()
    assert m.get_error() == hh.HARD_ENONPHYS
    assert m.get_error() == hh.HARD_OK       # read clears
    U[0, 2, 3, 4] = float("nan")
    rc, _ = hh.hard_hydro_cfl_dt(m.h, dev(U, torch.float32).data_ptr(), 0.4,
                                 torch.cuda.current_stream().cuda_stream)
    assert rc == hh.HARD_ENONPHYS
    del out


def test_allocation_failure_is_reported(monkeypatch):
    monkeypatch.setenv("HARD_HYDRO_FAIL_ALLOC", "1")
    m = hh.HardHydro((8, 8, 8), 1.4, 0)
    U = torch.ones((5, 8, 8, 8), device="cuda")
    with pytest.raises(hh.HardHydroError) as e:
        m.step(U, 1e-3)
    assert e.value.code == hh.HARD_ENOMEM
    monkeypatch.delenv("HARD_HYDRO_FAIL_ALLOC")
    m.step(U, 1e-3)                          # recovers once allocation works


def test_bounded_wait_timeout_is_reported(monkeypatch):
    """Failure detection of the TMA ring: with HARD_HYDRO_STARVE_TMA=1 the
    ring's barriers expect bytes that are never sent (no copy is issued, so
    nothing is in flight), every bounded wait runs out, and the stage reports
    HARD_ETIMEOUT instead of hanging; the next stage runs normally."""
    shape = (16, 8, 32)             # rows of 32 floats: the TMA path, one block
    gam = 5.0 / 3.0
    U = dev(H.smooth_3d(0, seed=5, gamma=gam, shape=shape), torch.float32)
    m = hh.HardHydro(shape, gam, hh.HARD_BC_PERIODIC, kernel=hh.HARD_KERNEL_FUSED)
    plain = hh.HardHydro(shape, gam, hh.HARD_BC_PERIODIC, kernel=hh.HARD_KERNEL_PLAIN)
    dt = m.cfl_dt(U, 0.4)
    monkeypatch.setenv("HARD_HYDRO_STARVE_TMA", "1")
    m.stage(1, None, U, dt)
    assert m.get_error() == hh.HARD_ETIMEOUT
    monkeypatch.delenv("HARD_HYDRO_STARVE_TMA")
    got = m.stage(1, None, U, dt)
    assert m.get_error() == hh.HARD_OK
    assert torch.equal(got, m.stage(1, None, U, dt))
    _close_f32(got, plain.stage(1, None, U, dt))


def _oracle_window_step(U, c, dt, gam, half=4):
    """Oracle step of the cell c = (k, j, i) of a periodic mesh from its own
    (2*half+1)^3 periodic neighbourhood: a two-stage update reaches 4 cells."""
    k, j, i = c
    nz, ny, nx = U.shape[1:]
    idx = [np.arange(k - half, k + half + 1) % nz, np.arange(j - half, j + half + 1) % ny,
           np.arange(i - half, i + half + 1) % nx]
    W = U[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]]
    w = 2 * half + 1
    g = oracle.Grid((w, w, w), gam, oracle.BC_OUTFLOW)
    g.dxyz = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    return g.step(W, dt)[:, half, half, half]


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 3e-6), (torch.float64, 1e-12)])
def test_full_size_sampled_parity(dtype, tol):
    """The 256^3 smooth-flow workload in the launch configuration the bench
    times (default tile, fused kernel, device time loop): one step, then 48
    sampled cells against the oracle run on each cell's neighbourhood."""
    n = 256
    gam = 5.0 / 3.0
    U = H.smooth_3d(n, seed=0, gamma=gam)
    if dtype == torch.float32:
        U = U.astype(np.float32).astype(np.float64)     # the oracle sees the FP32 input
    m = hh.HardHydro((n, n, n), gam, 0, dtype=dtype)
    Ud = dev(U, dtype)
    _, dtl, _ = m.advance(Ud, 1, 0.4, log_dt=True)
    dt = float(dtl[0])
    got = Ud.double().cpu().numpy()
    rng = np.random.default_rng(5)
    cells = [tuple(rng.integers(0, n, 3)) for _ in range(46)] + [(0, 0, 0), (n - 1, n - 1, n - 1)]
    scale = np.max(np.abs(U), axis=(1, 2, 3))
    for c in cells:
        ref = _oracle_window_step(U, c, dt, gam)
        err = np.abs(got[(slice(None),) + c] - ref) / scale
        assert np.all(err <= tol), (c, err)


# The FP32 TMA kernel and the FP32 plain-load kernel evaluate the same scheme
# in different instruction orders (the TMA kernel passes x-face states between
# lanes, sums the divergence per axis before scaling), so their results agree
# to rounding, not bit for bit.  One step moves each value by O(dt/dx) of the
# fluxes; a few FP32 ulps of the largest value per field bound the difference.
F32_STEP_RTOL = 4e-7


def _close_f32(a, b, rtol=F32_STEP_RTOL):
    a = a.double()
    b = b.double()
    for f in range(5):
        scale = float(b[f].abs().max())
        err = float((a[f] - b[f]).abs().max())
        assert err <= rtol * scale, (f, err, scale)


def _tma_tiles(m):
    """Tiles whose FP32 fused step runs the TMA kernel (32-wide tiles)."""
    return [t for t in range(m.tile_count()) if m.tile_info(t)[0] == 32]


def test_deterministic_and_tile_independent():
    """Each kernel is deterministic, and every tile shape of one kernel
    evaluates each face flux with the same arithmetic in the same order:
    bit-identical results across tiles and z-chunks.  The TMA and plain
    kernels agree to FP32 rounding."""
    shape = (40, 33, 72)            # x a multiple of 4: the fused kernel takes the TMA path
    gam = 1.4
    g = np.random.default_rng(0)
    U = g.uniform(0.5, 1.5, (5,) + shape) * np.array([1, 0.1, 0.1, 0.1, 3])[:, None, None, None]
    U = dev(U, torch.float32)
    m = hh.HardHydro(shape, gam, [2, 1, 0, 0, 1, 2])
    base = m.step(U, 1e-4)
    again = m.step(U, 1e-4)
    assert torch.equal(base, again)
    for tile in _tma_tiles(m):
        m.set_kernel(hh.HARD_KERNEL_FUSED, tile)
        assert torch.equal(m.step(U, 1e-4), base), tile
    m.set_kernel(hh.HARD_KERNEL_PLAIN, 0)
    plain = m.step(U, 1e-4)
    for tile in range(m.tile_count()):
        m.set_kernel(hh.HARD_KERNEL_PLAIN, tile)
        assert torch.equal(m.step(U, 1e-4), plain), tile
    _close_f32(base, plain)


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_fused_matches_plain_f32(bc):
    """The TMA-fed kernel and the plain-load kernel agree to FP32 rounding on
    every boundary kind (ragged tiles in x and y), and the TMA kernel gives
    the same bits on every tile shape."""
    shape = (37, 30, 100)
    gam = 5.0 / 3.0
    U = dev(H.smooth_3d(0, seed=3, gamma=gam, shape=shape), torch.float32)
    fused = hh.HardHydro(shape, gam, bc, kernel=hh.HARD_KERNEL_FUSED)
    plain = hh.HardHydro(shape, gam, bc, kernel=hh.HARD_KERNEL_PLAIN)
    dt = fused.cfl_dt(U, 0.4)
    a = fused.step(U, dt)
    b = plain.step(U, dt)
    _close_f32(a, b)
    for tile in _tma_tiles(fused):
        fused.set_kernel(hh.HARD_KERNEL_FUSED, tile)
        assert torch.equal(fused.step(U, dt), a), tile
