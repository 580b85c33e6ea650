"""GPU parity: the CUDA stage kernels (through the C ABI) against the FP64 CPU
oracle, element by element.

Tolerances (per field f, c16 reading of "max relative per field"):
  FP64: max_i |a_i - b_i| / max_i |b_i| <= 1e-12
  FP32: relative L1  sum |a - b| / sum |b| <= 1e-5 on smooth flows and
        <= 1e-3 on shocked flows (against the FP64 oracle).
"""
import math

import numpy as np
import pytest

import hydro_inputs as H
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

hh = pytest.importorskip("paper_2509_08971_gb300")

F64_TOL = 1e-12


def max_rel(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(5, -1)
    b = np.asarray(b, dtype=np.float64).reshape(5, -1)
    scale = np.maximum(np.max(np.abs(b), axis=1), 1e-300)
    return np.max(np.abs(a - b), axis=1) / scale


def rel_l1(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(5, -1)
    b = np.asarray(b, dtype=np.float64).reshape(5, -1)
    scale = np.maximum(np.sum(np.abs(b), axis=1), 1e-300)
    return np.sum(np.abs(a - b), axis=1) / scale


def dev(U, dtype):
    return torch.tensor(np.ascontiguousarray(U), dtype=dtype, device="cuda")


def host(T):
    return T.double().cpu().numpy()


def random_state(shape, gamma, seed, amp=0.3):
    g = np.random.default_rng(seed)
    nz, ny, nx = shape
    z = H.centres(nz)[:, None, None]
    y = H.centres(ny)[None, :, None]
    x = H.centres(nx)[None, None, :]

    def field(base, a):
        c = g.uniform(-1, 1, 4)
        return np.broadcast_to(base + a * np.sin(2 * np.pi * (x + c[0] * y + 2 * c[1] * z) + 3 * c[2])
                               + 0.2 * a * np.cos(2 * np.pi * (2 * x - y + c[3] * z)), shape)

    W = np.stack([field(1.0, amp), field(0.3, 1.0), field(-0.2, 1.0), field(0.1, 1.0),
                  field(1.0, amp)])
    return H.prim_to_cons(W, gamma)


SHAPES = [
    (1, 1, 300),       # 1D x, ragged over 128-wide tiles
    (1, 37, 1),        # 1D along y (kernel x = physical y)
    (29, 1, 1),        # 1D along z
    (1, 19, 45),       # 2D x-y, ragged both ways
    (13, 1, 40),       # 2D x-z
    (17, 21, 1),       # 2D y-z
    (11, 13, 37),      # 3D, ragged tiles and a short z chunk
    (70, 9, 8),        # 3D, z longer than one chunk (TMA path: rows of 16-byte multiples)
    (23, 21, 44),      # 3D TMA path, ragged in x, y and z
    (9, 10, 8),        # 3D TMA path, one tile touching both x walls
]
BCS = [(0,) * 6, (1,) * 6, (2,) * 6, (2, 1, 0, 0, 1, 2)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("kernel", [0, 1])
def test_stage_f64_matches_oracle(shape, bc, kernel):
    gam = 1.4
    U = random_state(shape, gam, seed=hash((shape, bc)) % 1000)
    # an axis of one cell cannot be periodic on one side only; keep the pairs consistent
    g = oracle.Grid(shape, gam, list(bc), extent=(1.0, 0.7, 1.3))
    dt = 0.3 / g.max_rate(U)
    m = hh.HardHydro(shape, gam, list(bc), dtype=torch.float64, extent=(1.0, 0.7, 1.3),
                     kernel=kernel)
    Ud = dev(U, torch.float64)
    U1 = m.stage(1, None, Ud, dt)
    ref1 = g.stage(1, U, U, dt)
    assert np.all(max_rel(host(U1), ref1) <= F64_TOL), max_rel(host(U1), ref1)
    U2 = m.stage(2, Ud, U1, dt)
    ref2 = g.stage(2, U, ref1, dt)
    assert np.all(max_rel(host(U2), ref2) <= F64_TOL), max_rel(host(U2), ref2)
    assert m.get_error() == hh.HARD_OK


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 2), (2, 2, 2)])
def test_tiny_meshes_f64(shape):
    gam = 1.4
    U = random_state(shape, gam, seed=3)
    for bc in (0, 1, 2):
        g = oracle.Grid(shape, gam, bc)
        rate = g.max_rate(U)
        dt = 0.3 / rate if rate > 0 else 1e-3      # no active axis: any dt
        m = hh.HardHydro(shape, gam, bc, dtype=torch.float64)
        got = host(m.step(dev(U, torch.float64), dt))
        assert np.all(max_rel(got, g.step(U, dt)) <= F64_TOL)


@pytest.mark.parametrize("tile", range(6))
def test_every_3d_tile_f64(tile):
    shape = (67, 19, 70)
    gam = 5.0 / 3.0
    U = random_state(shape, gam, seed=tile)
    g = oracle.Grid(shape, gam, oracle.BC_PERIODIC)
    dt = 0.4 / g.max_rate(U)
    ref = g.step(U, dt)
    m = hh.HardHydro(shape, gam, 0, dtype=torch.float64, tile=tile)
    assert np.all(max_rel(host(m.step(dev(U, torch.float64), dt)), ref) <= F64_TOL)


def test_riemann_1d_100_steps_f64():
    """Seeded two-state problem of the 1D configuration: 400 cells, outflow,
    CFL 0.4, device-resident time loop to t = 0.15 (or 100 steps)."""
    for seed in range(4):
        pb = H.riemann_1d(seed)
        n = 400
        U = pb.U(n)
        g = oracle.Grid((1, 1, n), pb.gamma, oracle.BC_OUTFLOW)
        ref, t_ref, dts_ref = g.run(U, 100, 0.4, t_end=0.15)
        m = hh.HardHydro((1, 1, n), pb.gamma, hh.HARD_BC_OUTFLOW, dtype=torch.float64)
        Ud = dev(U, torch.float64)
        t, dtl, _ = m.advance(Ud, 100, 0.4, t_end=0.15, log_dt=True)
        got = host(Ud)
        assert np.all(max_rel(got, ref) <= F64_TOL), (seed, max_rel(got, ref))
        assert float(t) == pytest.approx(t_ref, rel=1e-14)
        dtl = dtl.cpu().numpy()[:len(dts_ref)]
        np.testing.assert_allclose(dtl, dts_ref, rtol=1e-13)


def test_smooth_3d_64_100_steps_f64_and_f32():
    """3D periodic smooth flow (entropy wave + 8 acoustic modes), gamma = 5/3,
    at 64^3 for 100 steps: FP64 within 1e-12 max-relative, FP32 within 1e-5
    relative L1 of the FP64 oracle; conservation to roundoff."""
    n = 64
    gam = 5.0 / 3.0
    U = H.smooth_3d(n, seed=0, gamma=gam)
    g = oracle.Grid((n, n, n), gam, oracle.BC_PERIODIC)
    ref, t_ref, dts = g.run(U, 100, 0.4)
    m64 = hh.HardHydro((n, n, n), gam, 0, dtype=torch.float64)
    U64 = dev(U, torch.float64)
    t64, _, tot = m64.advance(U64, 100, 0.4, log_totals=True)
    assert np.all(max_rel(host(U64), ref) <= F64_TOL), max_rel(host(U64), ref)
    assert float(t64) == pytest.approx(t_ref, rel=1e-14)
    T0, T1 = g.totals(U), tot.cpu().numpy()[-1]
    assert np.all(np.abs(T1 - T0) <= 1e-12 * (np.abs(T0) + 1.0))
    m32 = hh.HardHydro((n, n, n), gam, 0, dtype=torch.float32)
    U32 = dev(U, torch.float32)
    m32.advance(U32, 100, 0.4)
    err = rel_l1(host(U32), ref)
    assert np.all(err <= 1e-5), err


def test_shocked_1d_f32():
    for seed in range(4):
        pb = H.riemann_1d(seed)
        n = 400
        U = pb.U(n)
        g = oracle.Grid((1, 1, n), pb.gamma, oracle.BC_OUTFLOW)
        ref, t_ref, _ = g.run(U, 100, 0.4, t_end=0.15)
        m = hh.HardHydro((1, 1, n), pb.gamma, hh.HARD_BC_OUTFLOW, dtype=torch.float32)
        Ud = dev(U, torch.float32)
        t = torch.zeros((), dtype=torch.float64, device="cuda")
        m.advance(Ud, 100, 0.4, t_end=0.15, t=t)
        err = rel_l1(host(Ud), ref)
        # momentum may be ~0 on average: judge it on the scale of rho |u|
        assert np.all(err[[0, 4]] <= 1e-3), (seed, err)
        assert abs(float(t) - t_ref) <= 1e-5 * t_ref


def test_cfl_dt_matches_oracle():
    shape = (9, 14, 33)
    gam = 1.4
    U = random_state(shape, gam, seed=9)
    g = oracle.Grid(shape, gam, 0, extent=(1.0, 2.0, 0.5))
    ref = 0.4 / g.max_rate(U)
    m = hh.HardHydro(shape, gam, 0, dtype=torch.float64, extent=(1.0, 2.0, 0.5))
    assert m.cfl_dt(dev(U, torch.float64), 0.4) == ref
    m32 = hh.HardHydro(shape, gam, 0, dtype=torch.float32, extent=(1.0, 2.0, 0.5))
    assert m32.cfl_dt(dev(U, torch.float32), 0.4) == pytest.approx(ref, rel=1e-6)


def test_totals_match_oracle():
    shape = (20, 30, 40)
    gam = 1.4
    U = random_state(shape, gam, seed=4)
    g = oracle.Grid(shape, gam, 0)
    ref = g.totals(U)
    for dtype, tol in ((torch.float64, 1e-13), (torch.float32, 1e-6)):
        m = hh.HardHydro(shape, gam, 0, dtype=dtype)
        got = np.array(m.totals(dev(U, dtype)))
        assert np.all(np.abs(got - ref) <= tol * (np.abs(ref) + 1.0)), (dtype, got, ref)


def test_advance_host_matches_device_loop():
    shape = (16, 16, 16)
    gam = 5.0 / 3.0
    U = H.smooth_3d(16, seed=2, gamma=gam)
    m = hh.HardHydro(shape, gam, 0, dtype=torch.float32)
    Ud = dev(U, torch.float32)
    m.advance(Ud, 7, 0.4)
    Uh = torch.tensor(U, dtype=torch.float32).pin_memory()
    out, t = m.advance_host(Uh, 7, 0.4)
    assert torch.equal(out, Ud.cpu())


@pytest.mark.parametrize("shape", [(24, 10, 36), (7, 5, 9), (1, 12, 20), (1, 1, 50)])
@pytest.mark.parametrize("bc", [0, 1, 2])
def test_uniform_state_is_a_fixed_point(shape, bc):
    """A uniform state (at rest next to reflecting walls, moving otherwise) is
    a fixed point of the scheme: every face sees the same two states, so the
    flux difference vanishes exactly, whatever the flux rounds to.  Bit-exact
    in both precisions, both kernels (the TMA path for rows of 32-bit
    multiples, plain loads otherwise), 1D to 3D, ragged tiles."""
    vel = (0.0, 0.0, 0.0) if bc == 2 else (0.3, -0.2, 0.1)
    W = [np.full(shape, v) for v in (1.3,) + vel + (0.7,)]
    U = H.prim_to_cons(W, 1.4)
    for dtype in (torch.float32, torch.float64):
        for kernel in (hh.HARD_KERNEL_FUSED, hh.HARD_KERNEL_PLAIN):
            m = hh.HardHydro(shape, 1.4, bc, dtype=dtype, kernel=kernel)
            Ud = dev(U, dtype)
            V = m.step(Ud, 1e-3)
            assert torch.equal(V, Ud), (dtype, kernel)
            assert m.get_error() == hh.HARD_OK
