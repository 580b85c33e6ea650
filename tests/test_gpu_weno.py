"""GPU parity of the second scheme (WENO5-Z face states + HLL flux) against
the FP64 oracle, through the C ABI.

Tolerances as for the default scheme: FP64 max-relative per field <= 1e-12;
FP32 relative L1 per field <= 1e-5 on smooth flows, <= 1e-3 on shocked ones.
"""
import numpy as np
import pytest

import hydro_inputs as H
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
hh = pytest.importorskip("paper_2509_08971_gb300")

from test_gpu_parity import F64_TOL, dev, host, max_rel, random_state, rel_l1  # noqa: E402

W5 = oracle.SCHEME_WENO5Z_HLL

SHAPES = [
    (1, 1, 300),       # 1D x, ragged over the 128-wide tile
    (1, 37, 1),        # 1D along y
    (29, 1, 1),        # 1D along z
    (1, 19, 45),       # 2D x-y, ragged both ways
    (13, 1, 40),       # 2D x-z
    (17, 21, 1),       # 2D y-z
    (11, 13, 37),      # 3D, ragged tiles and a short z chunk
    (70, 9, 8),        # 3D, z longer than one chunk
    (3, 3, 3),         # the smallest mesh the scheme takes
]
BCS = [(0,) * 6, (1,) * 6, (2,) * 6, (2, 1, 0, 0, 1, 2)]


def _handle(shape, gam, bc, dtype, **kw):
    return hh.HardHydro(shape, gam, list(bc), dtype=dtype, scheme=hh.HARD_SCHEME_WENO5Z_HLL, **kw)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", BCS)
def test_weno_stage_f64_matches_oracle(shape, bc):
    gam = 1.4
    U = random_state(shape, gam, seed=hash((shape, bc)) % 1000)
    g = oracle.Grid(shape, gam, list(bc), extent=(1.0, 0.7, 1.3), scheme=W5)
    dt = 0.3 / g.max_rate(U)
    m = _handle(shape, gam, bc, torch.float64, extent=(1.0, 0.7, 1.3))
    Ud = dev(U, torch.float64)
    U1 = m.stage(1, None, Ud, dt)
    ref1 = g.stage(1, U, U, dt)
    assert np.all(max_rel(host(U1), ref1) <= F64_TOL), max_rel(host(U1), ref1)
    U2 = m.stage(2, Ud, U1, dt)
    ref2 = g.stage(2, U, ref1, dt)
    assert np.all(max_rel(host(U2), ref2) <= F64_TOL), max_rel(host(U2), ref2)
    assert m.get_error() == hh.HARD_OK


def test_weno_sod_100_steps_f64_and_f32():
    """Sod (Sec. 3.1), 400 cells, outflow, CFL 0.4, the device time loop to
    t = 0.2: FP64 within 1e-12 of the oracle with the same dt schedule; FP32
    within the shocked-flow tolerance."""
    pb = H.sod()
    n = 400
    U = pb.U(n)
    g = oracle.Grid((1, 1, n), pb.gamma, oracle.BC_OUTFLOW, scheme=W5)
    ref, t_ref, dts = g.run(U, 1000, 0.4, t_end=0.2)
    for dtype in (torch.float64, torch.float32):
        m = _handle((1, 1, n), pb.gamma, (1,) * 6, dtype)
        Ud = dev(U, dtype)
        t = torch.zeros((), dtype=torch.float64, device="cuda")
        _, dtl, _ = m.advance(Ud, 1000, 0.4, t_end=0.2, t=t, log_dt=True)
        if dtype == torch.float64:
            assert np.all(max_rel(host(Ud), ref) <= F64_TOL), max_rel(host(Ud), ref)
            np.testing.assert_allclose(dtl.cpu().numpy()[:len(dts)], dts, rtol=1e-13)
            assert float(t) == pytest.approx(t_ref, rel=1e-14)
        else:
            err = rel_l1(host(Ud), ref)
            assert np.all(err[[0, 1, 4]] <= 1e-3), err


def test_weno_smooth_3d_f64_and_f32():
    """3D periodic smooth flow at 48^3, 20 steps: FP64 within 1e-12, FP32
    within 1e-5 relative L1 of the oracle; totals conserved."""
    n = 48
    gam = 5.0 / 3.0
    U = H.smooth_3d(n, seed=1, gamma=gam)
    g = oracle.Grid((n, n, n), gam, oracle.BC_PERIODIC, scheme=W5)
    ref, t_ref, _ = g.run(U, 20, 0.4)
    m64 = _handle((n, n, n), gam, (0,) * 6, torch.float64)
    U64 = dev(U, torch.float64)
    t64, _, tot = m64.advance(U64, 20, 0.4, log_totals=True)
    assert np.all(max_rel(host(U64), ref) <= F64_TOL), max_rel(host(U64), ref)
    assert float(t64) == pytest.approx(t_ref, rel=1e-14)
    T0 = g.totals(U)
    assert np.all(np.abs(tot.cpu().numpy()[-1] - T0) <= 1e-12 * (np.abs(T0) + 1.0))
    m32 = _handle((n, n, n), gam, (0,) * 6, torch.float32)
    U32 = dev(U, torch.float32)
    m32.advance(U32, 20, 0.4)
    err = rel_l1(host(U32), ref)
    assert np.all(err <= 1e-5), err


def _oracle_window_step(U, c, dt, gam, half=6):
    """Oracle step of cell c = (k, j, i) of a periodic mesh from its own
    (2*half+1)^3 periodic neighbourhood: a two-stage WENO update reaches 6
    cells."""
    k, j, i = c
    nz, ny, nx = U.shape[1:]
    idx = [np.arange(k - half, k + half + 1) % nz, np.arange(j - half, j + half + 1) % ny,
           np.arange(i - half, i + half + 1) % nx]
    W = U[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]]
    w = 2 * half + 1
    g = oracle.Grid((w, w, w), gam, oracle.BC_OUTFLOW, scheme=W5)
    g.dxyz = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    return g.step(W, dt)[:, half, half, half]


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 3e-6), (torch.float64, 1e-12)])
def test_weno_full_size_sampled_parity(dtype, tol):
    """The 256^3 smooth-flow workload in the launch configuration the bench
    times: one device-loop step, then 24 sampled cells against the oracle run
    on each cell's neighbourhood."""
    n = 256
    gam = 5.0 / 3.0
    U = H.smooth_3d(n, seed=0, gamma=gam)
    if dtype == torch.float32:
        U = U.astype(np.float32).astype(np.float64)
    m = _handle((n, n, n), gam, (0,) * 6, dtype)
    Ud = dev(U, dtype)
    _, dtl, _ = m.advance(Ud, 1, 0.4, log_dt=True)
    dt = float(dtl[0])
    got = Ud.double().cpu().numpy()
    rng = np.random.default_rng(9)
    cells = [tuple(rng.integers(0, n, 3)) for _ in range(22)] + [(0, 0, 0), (n - 1, n - 1, n - 1)]
    scale = np.max(np.abs(U), axis=(1, 2, 3))
    for c in cells:
        err = np.abs(got[(slice(None),) + c] - _oracle_window_step(U, c, dt, gam)) / scale
        assert np.all(err <= tol), (c, err)


def test_weno_noalloc_step_and_scheme_rules():
    shape = (12, 10, 20)
    gam = 1.4
    U = random_state(shape, gam, seed=4)
    m = _handle(shape, gam, (0,) * 6, torch.float64)
    Ud = dev(U, torch.float64)
    dt = m.cfl_dt(Ud, 0.4)
    ref = host(m.step(Ud, dt))
    out = torch.empty_like(Ud)
    rc = hh.hard_hydro_step_noalloc(m.h, Ud.data_ptr(), out.data_ptr(), dt,
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == hh.HARD_OK
    assert np.array_equal(host(out), ref)
    gg = torch.zeros((), dtype=torch.float64, device="cuda")
    with pytest.raises(hh.HardHydroError) as e:
        m.step_backward(Ud, torch.ones_like(Ud), dt, gg)
    assert e.value.code == hh.HARD_EUNSUPPORTED
    with pytest.raises(hh.HardHydroError):
        hh.HardHydro((1, 2, 16), gam, 0, scheme=hh.HARD_SCHEME_WENO5Z_HLL)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape,bc", [
    ((11, 13, 37), (2, 1, 0, 0, 1, 2)),    # ragged x segments and a short z chunk
    ((70, 9, 8), (0,) * 6),                # z longer than one march chunk
    ((20, 67, 61), (2,) * 6),              # y longer than one chunk, three x segments
    ((3, 3, 3), (1,) * 6),                 # the smallest mesh
])
def test_weno_sweeps_equal_fused_kernel(dtype, shape, bc):
    """On 3D meshes a handle runs the scheme as three directional sweeps
    (x, then y, then z with the combine); the no-allocation step runs the
    fused kernel.  Both evaluate the same face states, fluxes and flux
    difference in the same order, so one step agrees bit for bit, in either
    precision."""
    gam = 1.4
    U = random_state(shape, gam, seed=11)
    m = _handle(shape, gam, bc, dtype)
    Ud = dev(U, dtype)
    dt = m.cfl_dt(Ud, 0.4)
    ref = m.step(Ud, dt)
    out = torch.empty_like(Ud)
    rc = hh.hard_hydro_step_noalloc(m.h, Ud.data_ptr(), out.data_ptr(), dt,
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == hh.HARD_OK
    assert torch.equal(out, ref)
    assert m.get_error() == hh.HARD_OK
