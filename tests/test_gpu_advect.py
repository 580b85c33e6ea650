"""GPU parity of the radiation energy advection (WENO5-Z states, Rusanov
flux, Heun step with the fluid held fixed) against the oracle."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
hh = pytest.importorskip("paper_2509_08971_gb300")

from test_gpu_parity import F64_TOL, random_state  # noqa: E402

SHAPES = [(1, 1, 300), (1, 37, 1), (29, 1, 1), (1, 19, 45), (13, 1, 40), (17, 21, 1),
          (11, 13, 37), (70, 9, 8), (20, 67, 61), (3, 3, 3)]
BCS = [(0,) * 6, (1,) * 6, (2,) * 6, (2, 1, 0, 0, 1, 2)]


def _E(shape, seed):
    g = np.random.default_rng(seed)
    return 1.0 + 0.5 * g.random(shape) + np.linspace(0.0, 1.0, int(np.prod(shape))).reshape(shape)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", BCS)
def test_advect_f64_matches_oracle(shape, bc):
    gam = 1.4
    U = random_state(shape, gam, seed=hash((shape, bc)) % 1000)
    E = _E(shape, 7)
    g = oracle.Grid(shape, gam, list(bc), extent=(1.0, 0.7, 1.3))
    dt = 0.3 / g.max_rate(U)
    ref = g.advect_E(U, E, dt)
    m = hh.HardHydro(shape, gam, list(bc), dtype=torch.float64, extent=(1.0, 0.7, 1.3))
    Ud = torch.tensor(U, device="cuda")
    Ed = torch.tensor(E, device="cuda")
    m.advect_E(Ud, Ed, dt)
    got = Ed.cpu().numpy()
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= F64_TOL


def test_advect_f32_matches_oracle():
    shape = (24, 20, 36)
    gam = 1.4
    U = random_state(shape, gam, seed=3).astype(np.float32).astype(np.float64)
    E = _E(shape, 8).astype(np.float32).astype(np.float64)
    g = oracle.Grid(shape, gam, oracle.BC_PERIODIC)
    dt = 0.3 / g.max_rate(U)
    ref = g.advect_E(U, E, dt)
    m = hh.HardHydro(shape, gam, 0, dtype=torch.float32)
    Ud = torch.tensor(U, dtype=torch.float32, device="cuda")
    Ed = torch.tensor(E, dtype=torch.float32, device="cuda")
    m.advect_E(Ud, Ed, dt)
    got = Ed.double().cpu().numpy()
    assert np.sum(np.abs(got - ref)) / np.sum(np.abs(ref)) <= 1e-5


def test_advect_full_size_f32_conserves():
    """The 256^3 bench configuration: the periodic total of E is conserved."""
    n = 256
    U = torch.zeros((5, n, n, n), dtype=torch.float32, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(0)
    U[0] = 1.0 + 0.5 * torch.rand((n, n, n), device="cuda", generator=g)
    for a in (1, 2, 3):
        U[a] = U[0] * (torch.rand((n, n, n), device="cuda", generator=g) - 0.5)
    U[4] = 2.5
    E = 1.0 + torch.rand((n, n, n), device="cuda", generator=g)
    tot0 = float(E.double().sum())
    m = hh.HardHydro((n, n, n), 1.4, 0, dtype=torch.float32)
    m.advect_E(U, E, 0.2 / n)
    assert float(E.double().sum()) == pytest.approx(tot0, rel=1e-5)
    assert bool(torch.isfinite(E).all())
