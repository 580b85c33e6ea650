"""Pins of the PyTorch FP64 transcription (the autograd reference of the
adjoint): its forward values equal the C oracle's, and its autograd gradient
passes torch.autograd.gradcheck (finite differences) on tiny meshes."""
import numpy as np
import pytest
import torch

import hydro_inputs as H
from oracle import oracle_torch as OT


def random_state(shape, gamma, seed):
    g = np.random.default_rng(seed)
    W = [g.uniform(0.6, 1.6, shape), g.uniform(-0.5, 0.5, shape), g.uniform(-0.5, 0.5, shape),
         g.uniform(-0.5, 0.5, shape), g.uniform(0.6, 1.6, shape)]
    return H.prim_to_cons(W, gamma)


@pytest.mark.parametrize("shape", [(1, 1, 24), (1, 9, 11), (5, 6, 7)])
@pytest.mark.parametrize("bc6", [(0,) * 6, (1,) * 6, (2,) * 6, (2, 1, 0, 0, 1, 2)])
def test_forward_matches_c_oracle(orc, shape, bc6):
    gam = 1.4
    U = random_state(shape, gam, 3)
    g = orc.Grid(shape, gam, list(bc6))
    dt = 0.3 / g.max_rate(U)
    ref = g.step(U, dt)
    got = OT.step(torch.tensor(U), torch.tensor(gam, dtype=torch.float64), dt,
                  torch.tensor(g.dxyz), list(bc6)).numpy()
    scale = np.max(np.abs(ref.reshape(5, -1)), axis=1)
    assert np.all(np.max(np.abs(got - ref).reshape(5, -1), axis=1) <= 1e-13 * scale)


@pytest.mark.parametrize("bc6", [(0,) * 6, (1,) * 6, (2,) * 6])
def test_gradcheck_tiny(bc6):
    gam = 1.4
    shape = (1, 4, 5)
    U = torch.tensor(random_state(shape, gam, 5), requires_grad=True)
    gamma = torch.tensor(gam, dtype=torch.float64, requires_grad=True)
    dxyz = torch.tensor([0.2, 0.25, 1.0], dtype=torch.float64)

    def f(U, gamma):
        return OT.step(U, gamma, 0.01, dxyz, list(bc6))

    assert torch.autograd.gradcheck(f, (U, gamma), eps=1e-6, atol=1e-7, rtol=1e-5)
