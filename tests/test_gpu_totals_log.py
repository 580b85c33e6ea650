"""The conserved totals that the time loop logs per step, and the dt it carries
from one step to the next, on every kernel path: the TMA-fed 3D kernel, the
plain 3D kernel, 2D and 1D meshes, the second scheme, FP64.

* Each logged row (the stage-2 epilogue's per-warp FP64 sums, its per-block
  rows and the finalize launch) equals the standalone totals of the state
  that step left, up to the order of the FP64 sums.  A field sent to the wrong
  slot by the epilogue's warp reduction, or a lost block row, is an error of
  the order of the field itself.
* A multi-step call, where each next dt comes from the rate that stage 2
  folded into its epilogue, is bit-identical to single steps, where dt comes
  from the standalone rate pass: the two evaluate the same signal rate of the
  same cells, and a maximum does not depend on the order of its terms."""
import numpy as np
import pytest

import hydro_inputs as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
hh = pytest.importorskip("paper_2509_08971_gb300")

GAMMA = 1.4
CFL = 0.4
NSTEPS = 4


def _state(shape, seed):
    """Smooth seeded primitives with distinct means per field, so that two
    swapped totals cannot agree by accident."""
    g = np.random.default_rng(seed)
    nz, ny, nx = shape
    z = H.centres(nz)[:, None, None]
    y = H.centres(ny)[None, :, None]
    x = H.centres(nx)[None, None, :]

    def f(base, a):
        c = g.uniform(-1, 1, 3)
        return np.broadcast_to(base + a * np.sin(2 * np.pi * (x + c[0] * y + c[1] * z) + 3 * c[2]),
                               shape)

    W = np.stack([f(1.0, 0.3), f(0.4, 0.3), f(-0.3, 0.3), f(0.2, 0.3), f(1.0, 0.3)])
    return H.prim_to_cons(W, GAMMA)


CASES = [
    ((32, 16, 64), torch.float32, {"kernel": hh.HARD_KERNEL_FUSED}),    # TMA-fed 3D kernel
    ((32, 16, 62), torch.float32, {"kernel": hh.HARD_KERNEL_FUSED}),    # rows not 16-byte: plain
    ((24, 16, 64), torch.float32, {"kernel": hh.HARD_KERNEL_PLAIN}),
    ((1, 40, 72), torch.float32, {"kernel": hh.HARD_KERNEL_FUSED}),     # 2D
    ((1, 1, 300), torch.float32, {"kernel": hh.HARD_KERNEL_FUSED}),     # 1D
    ((32, 16, 64), torch.float32, {"scheme": hh.HARD_SCHEME_WENO5Z_HLL}),
    ((16, 16, 32), torch.float64, {"kernel": hh.HARD_KERNEL_FUSED}),
]


def _scale(U, dV):
    """Per field: the sum of |U_f| dV, the scale an error in a total is judged on."""
    return U.double().abs().reshape(5, -1).sum(dim=1).cpu().numpy() * dV


@pytest.mark.parametrize("shape,dtype,kw", CASES)
def test_logged_totals_and_carried_dt(shape, dtype, kw):
    m = hh.HardHydro(shape, GAMMA, hh.HARD_BC_PERIODIC, dtype=dtype, **kw)
    U0 = torch.tensor(_state(shape, seed=sum(shape)), dtype=dtype, device="cuda")
    nz, ny, nx = shape
    dV = 1.0 / (nx * ny * nz)
    tol = 1e-6 if dtype == torch.float32 else 1e-13

    # one call of NSTEPS steps
    Um = U0.clone()
    tm, dtm, totm = m.advance(Um, NSTEPS, CFL, log_dt=True, log_totals=True)
    assert m.get_error() == hh.HARD_OK
    # NSTEPS calls of one step; each row against the standalone totals
    Us = U0.clone()
    dts, tots = [], []
    for k in range(NSTEPS):
        _, dt1, tot1 = m.advance(Us, 1, CFL, log_dt=True, log_totals=True)
        row = tot1.cpu().numpy()[0]
        ref = np.array(m.totals(Us))
        assert np.all(np.abs(row - ref) <= tol * _scale(Us, dV)), (k, row, ref)
        dts.append(float(dt1[0]))
        tots.append(row)
    assert m.get_error() == hh.HARD_OK

    assert torch.equal(Um, Us)
    assert [float(d) for d in dtm.cpu()] == dts
    assert np.array_equal(totm.cpu().numpy(), np.array(tots))
    assert float(tm) == pytest.approx(sum(dts), rel=1e-15)
    # periodic box: every total is conserved through the steps
    T0 = np.array(m.totals(U0))
    assert np.all(np.abs(np.array(tots) - T0) <= 10 * tol * _scale(U0, dV))
