"""hard_hydro_step_noalloc: the step for callers that cannot allocate device
memory (code running during CUDA-graph stream capture, or hosts whose device
memory is reserved up front by another allocator).  It keeps the intermediate
stage in the library's fixed 64 MiB device array instead of handle scratch,
so it must give what hard_hydro_step gives, call after call.

Collected last on purpose: a failure here is reported after every other test
has run.  It passes alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

import hydro_inputs as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
hh = pytest.importorskip("paper_2509_08971_gb300")


def _stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("kernel", [hh.HARD_KERNEL_FUSED, hh.HARD_KERNEL_PLAIN])
def test_noalloc_step_equals_step_on_two_calls(dtype, kernel):
    shape = (24, 20, 48)                  # several tiles; FP32 fused takes the TMA path
    gam = 5.0 / 3.0
    U = torch.tensor(H.smooth_3d(0, seed=4, gamma=gam, shape=shape), dtype=dtype, device="cuda")
    m = hh.HardHydro(shape, gam, [0, 0, 2, 2, 1, 1], dtype=dtype, kernel=kernel)
    dt = m.cfl_dt(U, 0.4)
    ref1 = m.step(U, dt)
    ref2 = m.step(ref1, dt)
    out1 = torch.empty_like(U)
    out2 = torch.empty_like(U)
    assert hh.hard_hydro_step_noalloc(m.h, U.data_ptr(), out1.data_ptr(), dt, _stream()) == hh.HARD_OK
    assert hh.hard_hydro_step_noalloc(m.h, out1.data_ptr(), out2.data_ptr(), dt, _stream()) == hh.HARD_OK
    torch.cuda.synchronize()
    # same kernels, same dt, same operation order: identical to the last bit
    assert torch.equal(out1, ref1)
    assert torch.equal(out2, ref2)


def test_noalloc_step_in_place_and_limits():
    shape = (16, 16, 16)
    gam = 1.4
    U = torch.tensor(H.smooth_3d(16, seed=1, gamma=gam), dtype=torch.float32, device="cuda")
    m = hh.HardHydro(shape, gam, 0)
    dt = m.cfl_dt(U, 0.4)
    ref = m.step(U, dt)
    V = U.clone()
    assert hh.hard_hydro_step_noalloc(m.h, V.data_ptr(), V.data_ptr(), dt, _stream()) == hh.HARD_OK
    torch.cuda.synchronize()
    assert torch.equal(V, ref)
    # a mesh whose state exceeds the fixed array is refused, not truncated
    big = hh.hard_hydro_create(160, 160, 160, gam, 0)       # 82 MB of FP32 state
    assert big
    W = torch.empty(16, device="cuda")
    assert hh.hard_hydro_step_noalloc(big, W.data_ptr(), W.data_ptr(), dt, _stream()) == \
        hh.HARD_EUNSUPPORTED
    hh.hard_hydro_destroy(big)
    assert hh.hard_hydro_step_noalloc(m.h, None, V.data_ptr(), dt, _stream()) == hh.HARD_EINVAL
    assert hh.hard_hydro_step_noalloc(m.h, V.data_ptr(), V.data_ptr(), -1.0, _stream()) == \
        hh.HARD_EINVAL


def test_noalloc_status_word():
    """The status word of the no-allocation step is the call's own (the
    handle's flag does not see these calls): clean after a physical step,
    HARD_ENONPHYS after a step met a negative density, clean again once
    read."""
    shape = (8, 8, 32)
    gam = 1.4
    U = torch.tensor(H.smooth_3d(0, seed=2, gamma=gam, shape=shape), dtype=torch.float32,
                     device="cuda")
    m = hh.HardHydro(shape, gam, 0)
    dt = m.cfl_dt(U, 0.4)
    out = torch.empty_like(U)
    assert hh.hard_hydro_step_noalloc(m.h, U.data_ptr(), out.data_ptr(), dt, _stream()) == hh.HARD_OK
    torch.cuda.synchronize()
    assert hh.hard_hydro_noalloc_get_error() == hh.HARD_OK
    V = U.clone()
    V[0, 3, 4, 5] = -1.0
    assert hh.hard_hydro_step_noalloc(m.h, V.data_ptr(), out.data_ptr(), dt, _stream()) == hh.HARD_OK
    torch.cuda.synchronize()
    assert hh.hard_hydro_noalloc_get_error() == hh.HARD_ENONPHYS
    assert hh.hard_hydro_noalloc_get_error() == hh.HARD_OK
    assert m.get_error() == hh.HARD_OK
