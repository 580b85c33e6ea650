"""A run resumed from a checkpoint equals the uninterrupted run bit for bit:
the 64^3 blast (reflecting walls, CFL 0.3) in FP32 on the fused kernel and
the periodic smooth flow in FP64, 12 steps straight against 5 steps, a
checkpoint, a new handle built from it and 7 more steps; the states, the
times and the dt schedules agree exactly."""
import os

import numpy as np
import pytest

import hydro_inputs as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
hh = pytest.importorskip("paper_2509_08971_gb300")
from paper_2509_08971_gb300 import checkpoint  # noqa: E402


@pytest.mark.parametrize("case", ["blast_f32", "smooth_f64"])
def test_resume_equals_uninterrupted(tmp_path, case):
    n, cfl = 64, 0.3
    if case == "blast_f32":
        U0 = H.blast_3d(n, seed=1, gamma=1.4, dtype=np.float32)
        m = hh.HardHydro((n, n, n), 1.4, hh.HARD_BC_REFLECT, dtype=torch.float32)
    else:
        U0 = H.smooth_3d(n, seed=1, gamma=5.0 / 3.0)
        m = hh.HardHydro((n, n, n), 5.0 / 3.0, hh.HARD_BC_PERIODIC, dtype=torch.float64)
    U = torch.tensor(U0, dtype=m.dtype, device="cuda")
    Ua = U.clone()
    t_a, dt_a, _ = m.advance(Ua, 12, cfl, log_dt=True)

    Ub = U.clone()
    t_b, dt_b, _ = m.advance(Ub, 5, cfl, log_dt=True)
    path = os.path.join(tmp_path, "run.ckpt")
    checkpoint.save(path, m, Ub, t_b, 5, dt_b.cpu().tolist())
    del Ub
    c = checkpoint.load(path)
    m2 = c.handle()
    Uc = c.U.clone()
    t_c, dt_c, _ = m2.advance(Uc, 7, cfl, t=torch.tensor(c.t, dtype=torch.float64, device="cuda"),
                              log_dt=True)
    assert m2.get_error() == hh.HARD_OK
    assert torch.equal(Uc, Ua)
    assert float(t_c) == float(t_a)
    assert c.dts + dt_c.cpu().tolist() == dt_a.cpu().tolist()
