"""The strong spherical blast configuration on the CUDA path (gamma = 1.4,
ambient rho = 1 with +-1 % seeded noise, p = 1e-5, energy 1 spread over the
cells within four cells of the centre, reflecting walls, CFL 0.3).

* Both kernels against the FP64 CPU oracle on the oracle's own CFL dt
  schedule, 48^3, 20 steps: FP64 within 1e-12 max relative per field, FP32
  within the shocked-flow tolerance 1e-3 relative L1 per field.
* FP32 bulk against the FP64 path on the same dt schedule at 128^3: relative
  L1 per field within 1e-3.
* Without the noise the blast is symmetric under each axis reflection and
  each permutation of the axes (momenta change sign or component with them);
  the FP64 kernels keep that symmetry to rounding, as the oracle does."""
import numpy as np
import pytest

import hydro_inputs as H
import oracle
import oracle_window

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
hh = pytest.importorskip("paper_2509_08971_gb300")

GAMMA = 1.4
CFL = 0.3


def _dt_schedule(m64, U64, nsteps):
    t, dts, _ = m64.advance(U64, nsteps, CFL, log_dt=True)
    return [float(d) for d in dts.cpu()]


@pytest.fixture(scope="module")
def blast_oracle_48():
    """Oracle run of the noisy 48^3 blast: (U0, dt schedule, U after 20 steps)."""
    n, nsteps = 48, 20
    U0 = H.blast_3d(n, seed=3, gamma=GAMMA)
    g = oracle.Grid((n, n, n), GAMMA, oracle.BC_REFLECT)
    U, _, dts = g.run(U0, nsteps, CFL)
    return U0, dts, U


@pytest.mark.parametrize("kernel", [hh.HARD_KERNEL_FUSED, hh.HARD_KERNEL_PLAIN])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_blast_against_oracle(blast_oracle_48, kernel, dtype):
    """The strong-shock regime (p = 1e-5 ambient, pressure ratio ~1e7 at the
    front) through the reflecting-wall ghost map of both kernels (the fused
    one takes the TMA path: rows of 48 values are 16-byte multiples), on the
    oracle's dt schedule."""
    U0, dts, ref = blast_oracle_48
    n = U0.shape[-1]
    m = hh.HardHydro((n, n, n), GAMMA, hh.HARD_BC_REFLECT, dtype=dtype, kernel=kernel)
    Ud = torch.tensor(U0, dtype=dtype, device="cuda")
    for dt in dts:
        Ud = m.step(Ud, float(dt))
    assert m.get_error() == hh.HARD_OK
    got = Ud.double().cpu().numpy().reshape(5, -1)
    b = ref.reshape(5, -1)
    assert float(np.max(np.abs(b[1]))) > 1e-3               # the shock has formed and moved
    if dtype == torch.float64:
        err = np.max(np.abs(got - b), axis=1) / np.max(np.abs(b), axis=1)
        assert np.all(err <= 1e-12), err
    else:
        err = np.sum(np.abs(got - b), axis=1) / np.sum(np.abs(b), axis=1)
        assert np.all(err <= 1e-3), err


def test_blast_fp32_against_fp64_per_field():
    n, nsteps = 128, 20
    U = H.blast_3d(n, seed=0, gamma=GAMMA)
    m64 = hh.HardHydro((n, n, n), GAMMA, hh.HARD_BC_REFLECT, dtype=torch.float64)
    m32 = hh.HardHydro((n, n, n), GAMMA, hh.HARD_BC_REFLECT, dtype=torch.float32)
    U64 = torch.tensor(U, dtype=torch.float64, device="cuda")
    dts = _dt_schedule(m64, U64.clone(), nsteps)
    U32 = torch.tensor(U, dtype=torch.float32, device="cuda")
    for dt in dts:
        U64 = m64.step(U64, dt)
        U32 = m32.step(U32, dt)
    assert m64.get_error() == hh.HARD_OK and m32.get_error() == hh.HARD_OK
    a = U32.double().cpu().numpy().reshape(5, -1)
    b = U64.cpu().numpy().reshape(5, -1)
    err = np.sum(np.abs(a - b), axis=1) / np.sum(np.abs(b), axis=1)
    assert np.all(err <= 1e-3), err
    # the blast has spread: the shock is well off the initial energy spot
    assert float(np.max(np.abs(b[1]))) > 1e-3


def test_blast_symmetry_f64():
    n, nsteps = 48, 30
    U = H.blast_3d(n, noise=False, gamma=GAMMA)
    m = hh.HardHydro((n, n, n), GAMMA, hh.HARD_BC_REFLECT, dtype=torch.float64)
    Ud = torch.tensor(U, dtype=torch.float64, device="cuda")
    m.advance(Ud, nsteps, CFL)
    assert m.get_error() == hh.HARD_OK
    V = Ud.cpu().numpy()
    tol = 1e-12
    rho, mx, my, mz, E = V
    sr, sm, se = np.max(np.abs(rho)), np.max(np.abs(mx)), np.max(np.abs(E))
    assert sm > 1e-6                                   # the blast has moved
    # (z, y, x) layout: reflections along each axis
    assert np.max(np.abs(rho - rho[::-1, :, :])) <= tol * sr
    assert np.max(np.abs(rho - rho[:, ::-1, :])) <= tol * sr
    assert np.max(np.abs(rho - rho[:, :, ::-1])) <= tol * sr
    assert np.max(np.abs(mx + mx[:, :, ::-1])) <= tol * sm
    assert np.max(np.abs(my + my[:, ::-1, :])) <= tol * sm
    assert np.max(np.abs(mz + mz[::-1, :, :])) <= tol * sm
    # permutations of the axes carry the momentum components with them
    assert np.max(np.abs(rho - rho.transpose(1, 0, 2))) <= tol * sr
    assert np.max(np.abs(rho - rho.transpose(0, 2, 1))) <= tol * sr
    assert np.max(np.abs(mx - my.transpose(0, 2, 1))) <= tol * sm
    assert np.max(np.abs(mz - mx.transpose(2, 1, 0))) <= tol * sm
    assert np.max(np.abs(E - E.transpose(2, 1, 0))) <= tol * se


# ---- the headline size: 512^3 in the launch configuration the bench times ----

FULL_N = 512
FULL_STEPS = 3
FULL_HALF = 4 * FULL_STEPS        # a two-stage PLM step reaches 4 cells


@pytest.fixture(scope="module")
def blast_512_f32():
    """The 512^3 blast as the bench builds it (seed 0), in FP32."""
    return H.blast_3d(FULL_N, seed=0, gamma=GAMMA, dtype=np.float32)


@pytest.mark.parametrize("dtype,kernel,tile,tol", [
    (torch.float32, hh.HARD_KERNEL_FUSED, 2, 1e-5),     # the tile the bench's tuner picks
    (torch.float32, hh.HARD_KERNEL_FUSED, 1, 1e-5),
    (torch.float64, hh.HARD_KERNEL_PLAIN, -1, 1e-12),   # the FP64 leg of the bench
])
def test_blast_512_sampled_parity(blast_512_f32, dtype, kernel, tile, tol):
    """The headline workload at its full size: three steps of the 512^3 blast
    on the device time loop (CFL 0.3, reflecting walls), then 44 cells (the
    blast centre and its front, random cells, walls, edges and corners)
    against the oracle run on each cell's window with the device's dt
    schedule; error relative to each field's largest magnitude after the
    steps.  The FP64 kernel sees the FP32 input widened, like the oracle."""
    U = blast_512_f32
    n = FULL_N
    m = hh.HardHydro((n, n, n), GAMMA, hh.HARD_BC_REFLECT, dtype=dtype, kernel=kernel)
    if tile >= 0:
        m.set_kernel(kernel, tile)
    Ud = torch.tensor(U, dtype=dtype, device="cuda")
    _, dtl, _ = m.advance(Ud, FULL_STEPS, CFL, log_dt=True)
    assert m.get_error() == hh.HARD_OK
    dts = [float(d) for d in dtl.cpu()]
    rng = np.random.default_rng(11)
    c0 = n // 2
    cells = [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(20)]
    cells += [tuple(int(v) for v in c0 - 7 + rng.integers(0, 14, 3)) for _ in range(16)]
    cells += [(0, 0, 0), (n - 1, n - 1, n - 1), (0, c0, n - 1), (n - 1, 0, c0),
              (3, c0 - 1, 0), (n - 4, 4, 300), (c0, c0, c0), (c0 - 1, c0 - 1, c0 - 1)]
    idx = torch.tensor(cells, device="cuda")
    got = Ud[:, idx[:, 0], idx[:, 1], idx[:, 2]].double().cpu().numpy()
    scale = Ud.abs().amax(dim=(1, 2, 3)).double().cpu().numpy()
    for q, c in enumerate(cells):
        ref = oracle_window.cell_after(U, c, dts, GAMMA, FULL_HALF)
        err = np.abs(got[:, q] - ref) / scale
        assert np.all(err <= tol), (c, err)
    # the blast has started: the cells next to the energy spot move
    assert np.max(np.abs(got[1:4])) > 0.0
