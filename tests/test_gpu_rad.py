"""GPU parity of the radiative heating / cooling exchange (Eq.
"heating-cooling") against the oracle, through the C ABI."""
import numpy as np
import pytest

import hydro_inputs as H
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
hh = pytest.importorskip("paper_2509_08971_gb300")


def _run(pb, shape, dtype, dt, seed):
    U, Er = pb.state(shape, seed=seed, spread=0.5)
    if dtype == torch.float32:                 # the oracle sees the FP32 input
        U, Er = U.astype(np.float32).astype(np.float64), Er.astype(np.float32).astype(np.float64)
    m = hh.HardHydro(shape, pb.gamma, 0, dtype=dtype)
    Ud = torch.tensor(U, dtype=dtype, device="cuda")
    Ed = torch.tensor(Er, dtype=dtype, device="cuda")
    m.rad_exchange(Ud, Ed, dt, *pb.params)
    ref_U, ref_E, _ = oracle.rad_exchange(U, Er, dt, *pb.params)
    return m, Ud.double().cpu().numpy(), Ed.double().cpu().numpy(), ref_U, ref_E, U


CASES = [(H.heating(), 1e-9), (H.heating(), 1e-6), (H.cooling(), 1e-12), (H.cooling(), 1e-8),
         (H.cooling(), 1e3)]


@pytest.mark.parametrize("shape", [(3, 5, 7), (1, 1, 1000), (16, 16, 16)])
@pytest.mark.parametrize("pb,dt", CASES)
def test_exchange_f64_matches_oracle(shape, pb, dt):
    m, U, E, rU, rE, U0 = _run(pb, shape, torch.float64, dt, seed=sum(shape))
    assert np.array_equal(U[:4], U0[:4])                      # mass and momenta untouched
    assert np.max(np.abs(U[4] - rU[4]) / np.abs(rU[4])) <= 1e-14
    assert np.max(np.abs(E - rE) / np.abs(rE)) <= 1e-14
    assert m.get_error() == hh.HARD_OK


@pytest.mark.parametrize("pb,dt", CASES)
def test_exchange_f32_matches_oracle(pb, dt):
    m, U, E, rU, rE, _ = _run(pb, (20, 24, 28), torch.float32, dt, seed=7)
    for got, ref in ((U[4], rU[4]), (E, rE)):
        assert np.sum(np.abs(got - ref)) / np.sum(np.abs(ref)) <= 1e-5
    assert m.get_error() == hh.HARD_OK


def test_exchange_full_size_f32():
    """The 256^3 bench configuration: every cell against the oracle."""
    pb = H.cooling()
    m, U, E, rU, rE, _ = _run(pb, (256, 256, 256), torch.float32, 1e-9, seed=1)
    for got, ref in ((U[4], rU[4]), (E, rE)):
        assert np.sum(np.abs(got - ref)) / np.sum(np.abs(ref)) <= 1e-5


def test_exchange_flags_a_non_physical_cell():
    pb = H.heating()
    shape = (2, 3, 4)
    U, Er = pb.state(shape)
    U[4, 1, 2, 3] = -1.0                                      # negative internal energy
    m = hh.HardHydro(shape, pb.gamma, 0, dtype=torch.float64)
    Ud = torch.tensor(U, device="cuda")
    Ed = torch.tensor(Er, device="cuda")
    m.rad_exchange(Ud, Ed, 1e-9, *pb.params)
    got = Ud.cpu().numpy()
    assert got[4, 1, 2, 3] == -1.0 and Ed.cpu().numpy()[1, 2, 3] == Er[1, 2, 3]
    assert m.get_error() == hh.HARD_ENONPHYS
