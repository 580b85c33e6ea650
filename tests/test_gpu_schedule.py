"""The z-slab two-stage schedule (stage 2 of a slab right after stage 1 of
the slab above it, U1 kept in L2) is bit-identical to the whole-mesh one."""
import numpy as np
import pytest

import hydro_inputs as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
hh = pytest.importorskip("paper_2509_08971_gb300")

from test_gpu_parity import random_state  # noqa: E402

CASES = [((100, 24, 32), 0, 32), ((70, 16, 32), 2, 32), ((130, 8, 32), 1, 32),
         ((96, 16, 40), (2, 1, 0, 0, 1, 2), 32), ((128, 8, 32), 0, 64)]


@pytest.mark.parametrize("shape,bc,Z", CASES)
@pytest.mark.parametrize("dtype,kernel", [(torch.float32, 0), (torch.float64, 0), (torch.float32, 1)])
def test_slab_schedule_is_bit_identical(shape, bc, Z, dtype, kernel):
    gam = 1.4
    bc6 = [bc] * 6 if isinstance(bc, int) else list(bc)
    U0 = torch.tensor(random_state(shape, gam, seed=sum(shape)), dtype=dtype, device="cuda")
    out = []
    for slab in (0, Z):
        m = hh.HardHydro(shape, gam, bc6, dtype=dtype, kernel=kernel, tile=0)
        m.set_schedule(slab)
        U = U0.clone()
        t, dtl, tot = m.advance(U, 6, 0.4, log_dt=True, log_totals=True)
        V = m.step(U0, float(dtl[0]))                     # U_out != U_in
        out.append((U, dtl, tot, V, float(t)))
        assert m.get_error() == hh.HARD_OK
    (a, b) = out
    assert torch.equal(a[0], b[0])
    assert torch.equal(a[1], b[1])
    assert torch.equal(a[2], b[2])
    assert torch.equal(a[3], b[3])
    assert a[4] == b[4]


def test_schedule_argument_checks():
    m = hh.HardHydro((64, 8, 32), 1.4, 0)
    with pytest.raises(hh.HardHydroError):
        m.set_schedule(1)
    with pytest.raises(hh.HardHydroError):
        m.set_schedule(-4)
    m.set_schedule(0)
