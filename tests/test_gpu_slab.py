"""Z-slab decomposition on the GPU: the slabs of one mesh, each with its own
handle (HARD_BC_HALO towards its neighbours, the whole mesh's cell widths),
stepped in lock step in one process on one GPU.  The ghost exchange between
them is a device copy of the packed planes (the multi-process exchange over
NCCL/gloo is tests/test_slab_decomposition.py); the stages, the ghost-plane
loads of every kernel path (TMA-fed FP32 and FP64 kernels through the ghost
tensor maps, the plain kernel through its loads), the rate reduction and the
dt are the library's.  The decomposed run equals the whole-mesh device time
loop bit for bit."""
import numpy as np
import pytest

import hydro_inputs as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
hh = pytest.importorskip("paper_2509_08971_gb300")
from paper_2509_08971_gb300 import slab  # noqa: E402


def _advance_slabs(shape, bc6, U0, world, dtype, kernel, nsteps, cfl, gamma):
    layouts = [slab.SlabLayout(shape[0], r, world, bc_z=(bc6[4], bc6[5])) for r in range(world)]
    ms = [slab.slab_handle(shape, L, gamma, bc6, dtype=dtype, kernel=kernel, tile=0)
          for L in layouts]
    bs = [slab.CudaSlabBackend(m, L) for m, L in zip(ms, layouts)]
    Us = [torch.tensor(np.ascontiguousarray(U0[:, L.z0:L.z1]), dtype=dtype, device="cuda")
          for L in layouts]
    U1s = [torch.empty_like(U) for U in Us]

    def exchange(Vs):
        for b, V in zip(bs, Vs):
            b.pack(V)
        for L, b in zip(layouts, bs):
            if L.lo is not None:
                b.ghost_lo.copy_(bs[L.lo].send_hi)
            if L.hi is not None:
                b.ghost_hi.copy_(bs[L.hi].send_lo)

    def rate_max():
        r = torch.stack([b.rate for b in bs]).max()
        for b in bs:
            b.rate.fill_(r)

    for b, U in zip(bs, Us):
        b.local_rate(U)
    rate_max()
    for b in bs:
        b.finalize(cfl, 0.0)
    for step in range(nsteps):
        exchange(Us)
        for b, U, U1 in zip(bs, Us, U1s):
            b.stage(1, U, U, U1, False)
        exchange(U1s)
        for b, U, U1 in zip(bs, Us, U1s):
            b.stage(2, U, U1, U, True)
        rate_max()
        if step + 1 < nsteps:
            for b in bs:
                b.finalize(cfl, 0.0)
    for m in ms:
        assert m.get_error() == hh.HARD_OK
    return torch.cat(Us, dim=1), [float(b.t) for b in bs]


CASES = [
    ((24, 16, 32), [0, 0, 0, 0, 0, 0], 2),      # periodic ring of two: the same peer both ways
    ((32, 32, 32), [2, 2, 2, 2, 2, 2], 2),      # the blast between reflecting walls
    ((26, 12, 32), [0, 0, 1, 1, 0, 0], 3),      # uneven slabs (9, 9, 8 planes), ragged y tiles
    ((20, 10, 36), [1, 1, 2, 2, 1, 1], 4),      # outflow z ends, four slabs of five planes
]


@pytest.mark.parametrize("shape,bc6,world", CASES)
@pytest.mark.parametrize("kernel", [hh.HARD_KERNEL_FUSED, hh.HARD_KERNEL_PLAIN])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_decomposed_equals_whole_mesh(shape, bc6, world, kernel, dtype):
    gamma, cfl, nsteps = 1.4, 0.4, 8
    if bc6[4] == 2:
        U0 = H.blast_3d(shape[0], seed=2, gamma=gamma, p_amb=0.05)
    else:
        U0 = H.smooth_3d(0, seed=2, gamma=gamma, shape=shape)
    m = hh.HardHydro(shape, gamma, bc6, dtype=dtype, kernel=kernel, tile=0)
    V = torch.tensor(U0, dtype=dtype, device="cuda")
    t, _, _ = m.advance(V, nsteps, cfl)
    got, ts = _advance_slabs(shape, bc6, U0, world, dtype, kernel, nsteps, cfl, gamma)
    assert torch.equal(got, V)
    assert all(tt == float(t) for tt in ts)
    assert float((V - torch.tensor(U0, dtype=dtype, device="cuda")).abs().max()) > 1e-6


def test_halo_faces_argument_rules():
    shape = (12, 8, 32)
    L = slab.SlabLayout(24, 0, 2)
    m = slab.slab_handle((24, 8, 32), L, 1.4, [0] * 6)
    U = torch.zeros((5,) + (12, 8, 32), device="cuda")
    U[0] = 1.0
    U[4] = 2.5
    out = torch.empty_like(U)
    # ghost buffers not set yet
    assert hh.hard_hydro_stage(m.h, 1, None, U.data_ptr(), out.data_ptr(), 1e-3,
                               None) == hh.HARD_EINVAL
    # whole steps and the time loop need an exchange between the stages
    assert hh.hard_hydro_step(m.h, U.data_ptr(), out.data_ptr(), 1e-3, None) == hh.HARD_EUNSUPPORTED
    assert hh.hard_hydro_advance(m.h, U.data_ptr(), 1, 0.4, 0.0, None, None, None,
                                 None) == hh.HARD_EUNSUPPORTED
    assert hh.hard_hydro_step_noalloc(m.h, U.data_ptr(), out.data_ptr(), 1e-3,
                                      None) == hh.HARD_EUNSUPPORTED
    assert hh.hard_hydro_set_scheme(m.h, hh.HARD_SCHEME_WENO5Z_HLL) == hh.HARD_EUNSUPPORTED
    # halo faces only on z, only on 3D meshes, never against a periodic face
    h2 = hh.hard_hydro_create(32, 8, 12, 1.4, 1)
    assert hh.hard_hydro_set(h2, hh.HARD_F32, 1, 1, 1, [3, 3, 1, 1, 1, 1]) == hh.HARD_EINVAL
    assert hh.hard_hydro_set(h2, hh.HARD_F32, 1, 1, 1, [1, 1, 1, 1, 3, 0]) == hh.HARD_EINVAL
    assert hh.hard_hydro_set(h2, hh.HARD_F32, 1, 1, 1, [1, 1, 1, 1, 3, 2]) == hh.HARD_OK
    hh.hard_hydro_destroy(h2)
    h3 = hh.hard_hydro_create(32, 1, 12, 1.4, 1)
    assert hh.hard_hydro_set(h3, hh.HARD_F32, 1, 1, 1, [1, 1, 1, 1, 3, 3]) == hh.HARD_EINVAL
    hh.hard_hydro_destroy(h3)
    # stage 1 with a rate output is rejected; the packed planes are the slab's edges
    b = slab.CudaSlabBackend(m, L)
    assert hh.hard_hydro_stage_ex(m.h, 1, None, U.data_ptr(), out.data_ptr(), 1e-3, None,
                                  b.rate.data_ptr(), None) == hh.HARD_EINVAL
    V = torch.arange(U.numel(), dtype=torch.float32, device="cuda").reshape(U.shape)
    b.pack(V)
    assert torch.equal(b.send_lo, V[:, :2]) and torch.equal(b.send_hi, V[:, -2:])


def _backward_slabs(shape, bc6, U0, G0, world, dtype, dt, gamma):
    """The decomposed adjoint of one step (SlabAdjoint's sequence) for all
    slabs in lock step; the exchanges are device copies."""
    layouts = [slab.SlabLayout(shape[0], r, world, bc_z=(bc6[4], bc6[5])) for r in range(world)]
    ms = [slab.slab_handle(shape, L, gamma, bc6, dtype=dtype, kernel=hh.HARD_KERNEL_PLAIN)
          for L in layouts]
    bs = [slab.CudaSlabBackend(m, L) for m, L in zip(ms, layouts)]
    cut = [lambda A, L=L: torch.tensor(np.ascontiguousarray(A[:, L.z0:L.z1]), dtype=dtype,
                                      device="cuda") for L in layouts]
    Us = [c(U0) for c in cut]
    Gs = [c(G0) for c in cut]
    U1s, gUs, gU1s = ([torch.empty_like(U) for U in Us] for _ in range(3))
    for b in bs:
        b.set_dt(dt)

    def exchange(Vs):
        for b, V in zip(bs, Vs):
            b.pack(V)
        for L, b in zip(layouts, bs):
            if L.lo is not None:
                b.ghost_lo.copy_(bs[L.lo].send_hi)
            if L.hi is not None:
                b.ghost_hi.copy_(bs[L.hi].send_lo)

    def reverse():
        for L, b in zip(layouts, bs):
            if L.lo is not None:
                b.adj_recv_lo.copy_(bs[L.lo].adj_send_hi)
            if L.hi is not None:
                b.adj_recv_hi.copy_(bs[L.hi].adj_send_lo)
        for b in bs:
            b.vjp_add()

    exchange(Us)
    for b, U, U1 in zip(bs, Us, U1s):
        b.stage(1, U, U, U1, False)
    exchange(U1s)
    for b, U1, G in zip(bs, U1s, Gs):
        b.vjp_faces(2, U1, G)
    reverse()
    for b, U1, G, gU, gU1 in zip(bs, U1s, Gs, gUs, gU1s):
        b.vjp_cells(2, U1, G, gU1, False, gU)
    exchange(Us)
    for b, U, gU1 in zip(bs, Us, gU1s):
        b.vjp_faces(1, U, gU1)
    reverse()
    for b, U, gU, gU1 in zip(bs, Us, gUs, gU1s):
        b.vjp_cells(1, U, gU1, gU, True, None)
    for m in ms:
        assert m.get_error() == hh.HARD_OK
    return torch.cat(gUs, dim=1), sum(float(b.g_gamma) for b in bs)


ADJ_CASES = [
    ((24, 16, 32), [0, 0, 0, 0, 0, 0], 2),      # periodic ring of two
    ((26, 12, 32), [0, 0, 1, 1, 2, 2], 3),      # reflecting z ends, uneven slabs
]


@pytest.mark.parametrize("shape,bc6,world", ADJ_CASES)
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)])
def test_decomposed_adjoint_matches_whole_mesh(shape, bc6, world, dtype, tol):
    """The slabs' split VJP (face pass, reverse exchange of the ghost
    cotangents, cell pass) equals the whole mesh's hard_hydro_step_backward
    up to the order of the atomic sums (the CPU gloo test checks the same
    sequence against autograd of the transcription)."""
    gamma = 1.4
    U0 = H.smooth_3d(0, seed=3, gamma=gamma, shape=shape)
    G0 = np.random.default_rng(5).standard_normal((5,) + shape)
    m = hh.HardHydro(shape, gamma, bc6, dtype=dtype, kernel=hh.HARD_KERNEL_PLAIN)
    U = torch.tensor(U0, dtype=dtype, device="cuda")
    dt = m.cfl_dt(U, 0.4)
    gg = torch.zeros((), dtype=torch.float64, device="cuda")
    ref = m.step_backward(U, torch.tensor(G0, dtype=dtype, device="cuda"), dt, gg)
    got, got_gg = _backward_slabs(shape, bc6, U0, G0, world, dtype, dt, gamma)
    scale = float(ref.abs().max())
    assert float((got - ref).abs().max()) <= tol * scale
    assert abs(got_gg - float(gg)) <= 1e3 * tol * abs(float(gg))
