"""Z-slab decomposition (the ghost entities of Sec. 2.1, the scaling runs of
Sec. 3.6) on CPU ranks: gloo process groups of 2 and 3 ranks drive the
partition, the ghost exchange and the rate reduction of
``paper_2509_08971_gb300.slab``, with the FP64 oracle as each rank's stage.
The decomposed run must equal the single-rank oracle run of the whole mesh
bit for bit: every cell sees the same neighbours and the same dt.  The CUDA
kernels run the same loop on the GPU (tests/test_gpu_slab.py)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import hydro_inputs as H
import oracle
from paper_2509_08971_gb300 import slab
from paper_2509_08971_gb300 import HARD_BC_HALO

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GAMMA = 1.4
CFL = 0.4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleSlabBackend:
    """Each stage of one rank's slab by the oracle: the slab and its ghost
    planes form an extended mesh whose interior planes are the slab; the
    extended mesh's own z boundary only touches the ghost planes' results,
    which are dropped."""

    def __init__(self, layout, shape, bc6):
        nz, ny, nx = shape
        self.L = layout
        self.bc6 = list(bc6)
        self.dxyz = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
        lo, hi = layout.lo is not None, layout.hi is not None

        def buf(on):
            return torch.zeros((5, 2, ny, nx), dtype=torch.float64) if on else None

        self.send_lo, self.send_hi = buf(lo), buf(hi)
        self.ghost_lo, self.ghost_hi = buf(lo), buf(hi)
        self.rate = torch.zeros(1, dtype=torch.float64)
        self.dt = 0.0
        self.t = 0.0
        self.shape_xy = (ny, nx)

    def _grid(self, planes, halo_lo, halo_hi):
        bc = list(self.bc6)
        bc[4] = oracle.BC_OUTFLOW if halo_lo else self.L.bc_z[0]
        bc[5] = oracle.BC_OUTFLOW if halo_hi else self.L.bc_z[1]
        g = oracle.Grid((planes,) + self.shape_xy, GAMMA, bc)
        g.dxyz = self.dxyz.copy()                   # the whole mesh's widths, bit for bit
        return g

    def pack(self, U):
        if self.send_lo is not None:
            self.send_lo.copy_(U[:, :2])
        if self.send_hi is not None:
            self.send_hi.copy_(U[:, -2:])

    def _ext(self, V):
        parts = ([self.ghost_lo] if self.ghost_lo is not None else []) + [V] + \
                ([self.ghost_hi] if self.ghost_hi is not None else [])
        return torch.cat(parts, dim=1).numpy()

    def stage(self, stage, U0, Ucur, out, with_rate):
        k0 = 2 if self.ghost_lo is not None else 0
        ext = self._ext(Ucur)
        ext0 = self._ext(U0)
        g = self._grid(ext.shape[1], self.ghost_lo is not None, self.ghost_hi is not None)
        res = g.stage(stage, ext0, ext, self.dt)
        out.copy_(torch.from_numpy(res[:, k0:k0 + self.L.planes].copy()))
        if with_rate:
            self.local_rate(out)

    def local_rate(self, U):
        g = self._grid(self.L.planes, False, False)
        self.rate[0] = g.max_rate(U.numpy())

    def finalize(self, cfl, t_end):
        r = float(self.rate[0])
        dt = cfl / r
        if t_end > 0.0 and self.t + dt > t_end:
            dt = max(t_end - self.t, 0.0)
        self.t += dt
        self.dt = dt


def _rank_main(rank, world, port, shape, bc6, nsteps, seed, outdir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        L = slab.SlabLayout(shape[0], rank, world, bc_z=(bc6[4], bc6[5]))
        U0 = H.smooth_3d(0, seed=seed, gamma=GAMMA, shape=shape) if bc6[4] == 0 else \
            H.blast_3d(shape[0], seed=seed, gamma=GAMMA, p_amb=0.1)
        U = torch.from_numpy(np.ascontiguousarray(U0[:, L.z0:L.z1]))
        U1 = torch.empty_like(U)
        backend = OracleSlabBackend(L, shape, bc6)
        stepper = slab.SlabStepper(backend, slab.HaloExchange(L))
        stepper.advance(U, U1, nsteps, CFL)
        np.save(os.path.join(outdir, f"rank{rank}.npy"), U.numpy())
        np.save(os.path.join(outdir, f"t{rank}.npy"), np.array([backend.t]))
    finally:
        dist.destroy_process_group()


def _decomposed(tmp_path, world, shape, bc6, nsteps, seed):
    mp.spawn(_rank_main, args=(world, _free_port(), shape, bc6, nsteps, seed, str(tmp_path)),
             nprocs=world, join=True)
    parts = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    ts = [float(np.load(tmp_path / f"t{r}.npy")[0]) for r in range(world)]
    return np.concatenate(parts, axis=1), ts


def test_partition_and_neighbours():
    assert slab.partition(13, 3) == [(0, 5), (5, 9), (9, 13)]
    assert slab.partition(8, 2) == [(0, 4), (4, 8)]
    per = [slab.SlabLayout(12, r, 3) for r in range(3)]
    assert [(l.lo, l.hi) for l in per] == [(2, 1), (0, 2), (1, 0)]
    assert all(l.bc_z == (HARD_BC_HALO, HARD_BC_HALO) for l in per)
    wall = [slab.SlabLayout(12, r, 3, bc_z=(2, 1)) for r in range(3)]
    assert [(l.lo, l.hi) for l in wall] == [(None, 1), (0, 2), (1, None)]
    assert wall[0].bc_z == (2, HARD_BC_HALO) and wall[2].bc_z == (HARD_BC_HALO, 1)
    one = slab.SlabLayout(12, 0, 1)
    assert (one.lo, one.hi, one.bc_z) == (None, None, (0, 0))
    with pytest.raises(ValueError):
        slab.SlabLayout(5, 2, 3)                       # a slab of fewer than two planes


@pytest.mark.parametrize("world,shape,bc6", [
    (2, (12, 6, 8), [0, 0, 0, 0, 0, 0]),              # periodic z: each rank has both neighbours,
                                                      # the same peer above and below
    (2, (12, 12, 12), [2, 2, 2, 2, 2, 2]),            # reflecting walls: physical z faces
    (3, (13, 6, 8), [0, 0, 1, 1, 0, 0]),              # uneven slabs around a periodic ring
])
def test_decomposed_run_equals_single_rank_oracle(tmp_path, world, shape, bc6):
    nsteps, seed = 6, 4
    got, ts = _decomposed(tmp_path, world, shape, bc6, nsteps, seed)
    U0 = H.smooth_3d(0, seed=seed, gamma=GAMMA, shape=shape) if bc6[4] == 0 else \
        H.blast_3d(shape[0], seed=seed, gamma=GAMMA, p_amb=0.1)
    ref, t_ref, _ = oracle.Grid(shape, GAMMA, bc6).run(U0, nsteps, CFL)
    assert np.array_equal(got, ref)
    assert all(t == t_ref for t in ts)                 # every rank took the same dt
    assert np.max(np.abs(got - U0)) > 1e-6             # the state moved


def test_the_exchange_matters():
    """The equality above has teeth: slabs stepped without the exchange (each
    slab alone, its cut faces treated as outflow walls) differ from the
    single-rank run, so a dropped or misrouted ghost plane cannot pass."""
    shape, bc6, nsteps, seed = (12, 6, 8), [0, 0, 0, 0, 0, 0], 3, 4
    U0 = H.smooth_3d(0, seed=seed, gamma=GAMMA, shape=shape)
    ref, _, dts = oracle.Grid(shape, GAMMA, bc6).run(U0, nsteps, CFL)
    parts = []
    for z0, z1 in slab.partition(shape[0], 2):
        g = oracle.Grid((z1 - z0,) + shape[1:], GAMMA, [0, 0, 0, 0, 1, 1])
        g.dxyz = np.array([1.0 / shape[2], 1.0 / shape[1], 1.0 / shape[0]])
        parts.append(g.run_fixed(U0[:, z0:z1], dts))
    alone = np.concatenate(parts, axis=1)
    assert np.max(np.abs(alone - ref)) > 1e-6 * np.max(np.abs(ref))


def test_lpt_partition_of_independent_problems():
    """The batched configuration shards without an exchange: every problem on
    exactly one rank, the largest load within one problem of the mean, and
    the split deterministic."""
    spec = H.batch_spec(4096, seed=0)
    cost = [int(c) for c in spec.cells]
    for world in (1, 2, 3, 8):
        parts = slab.lpt_partition(cost, world)
        flat = sorted(p for q in parts for p in q)
        assert flat == list(range(len(cost)))
        loads = [sum(cost[p] for p in q) for q in parts]
        assert max(loads) <= sum(loads) / world + max(cost)
        assert parts == slab.lpt_partition(cost, world)
    assert slab.lpt_partition([5, 1, 4, 2, 3], 2) == [[0, 1, 3], [2, 4]]


# ---- the adjoint of a decomposed step (the ghost exchange reversed) ----

class TorchAdjointBackend:
    """One rank's stages and stage VJPs by autograd of the PyTorch oracle
    transcription on the rank's slab extended by its ghost planes: the VJP
    with respect to the ghost planes is the cotangent the neighbours own,
    sent back to them by the exchange (conserved variables here; the CUDA
    backend sends primitive cotangents before its cell pass)."""

    def __init__(self, layout, shape, bc6, gamma):
        from oracle import oracle_torch as ot
        self.ot = ot
        nz, ny, nx = shape
        self.L = layout
        self.gamma = gamma
        self.dxyz = (1.0 / nx, 1.0 / ny, 1.0 / nz)
        lo, hi = layout.lo is not None, layout.hi is not None

        def buf(on):
            return torch.zeros((5, 2, ny, nx), dtype=torch.float64) if on else None

        self.send_lo, self.send_hi = buf(lo), buf(hi)
        self.ghost_lo, self.ghost_hi = buf(lo), buf(hi)
        self.adj_send_lo, self.adj_send_hi = buf(lo), buf(hi)
        self.adj_recv_lo, self.adj_recv_hi = buf(lo), buf(hi)
        self.g_gamma = torch.zeros(1, dtype=torch.float64)
        bc = list(bc6)
        bc[4] = oracle.BC_OUTFLOW if lo else layout.bc_z[0]   # the extension's own walls only
        bc[5] = oracle.BC_OUTFLOW if hi else layout.bc_z[1]   # touch the dropped ghost cells
        self.bc = bc

    def pack(self, U):
        if self.send_lo is not None:
            self.send_lo.copy_(U[:, :2])
        if self.send_hi is not None:
            self.send_hi.copy_(U[:, -2:])

    def _L(self, V, gl, gh, gam):
        parts = ([gl] if gl is not None else []) + [V] + ([gh] if gh is not None else [])
        k0 = 2 if gl is not None else 0
        return self.ot.rhs(torch.cat(parts, dim=1), gam, self.dxyz, self.bc)[:, k0:k0 + V.shape[1]]

    def set_dt(self, dt):
        self.dt = float(dt)

    def stage(self, stage, U0, Ucur, out, with_rate):
        with torch.no_grad():
            Ls = self._L(Ucur, self.ghost_lo, self.ghost_hi, self.gamma)
            out.copy_(Ucur + self.dt * Ls if stage == 1 else 0.5 * U0 + 0.5 * (Ucur + self.dt * Ls))

    def vjp_faces(self, stage, Uc, G):
        b = 1.0 if stage == 1 else 0.5
        V = Uc.clone().requires_grad_(True)
        gl = None if self.ghost_lo is None else self.ghost_lo.clone().requires_grad_(True)
        gh = None if self.ghost_hi is None else self.ghost_hi.clone().requires_grad_(True)
        gam = torch.tensor(self.gamma, dtype=torch.float64, requires_grad=True)
        out = b * (V + self.dt * self._L(V, gl, gh, gam))
        ins = [V, gam] + [t for t in (gl, gh) if t is not None]
        grads = torch.autograd.grad(out, ins, grad_outputs=G)
        self.pending = grads[0]
        self.g_gamma += grads[1]
        k = 2
        if gl is not None:
            self.adj_send_lo.copy_(grads[k])
            k += 1
        if gh is not None:
            self.adj_send_hi.copy_(grads[k])

    def vjp_add(self):
        if self.adj_recv_lo is not None:
            self.pending[:, :2] += self.adj_recv_lo
        if self.adj_recv_hi is not None:
            self.pending[:, -2:] += self.adj_recv_hi

    def vjp_cells(self, stage, Uc, G, gUc, accumulate, gU0):
        if accumulate:
            gUc += self.pending
        else:
            gUc.copy_(self.pending)
        if gU0 is not None:
            gU0.copy_(0.5 * G)


def _adj_inputs(shape, bc6, seed):
    U0 = H.smooth_3d(0, seed=seed, gamma=GAMMA, shape=shape) if bc6[4] == 0 else \
        H.blast_3d(shape[0], seed=seed, gamma=GAMMA, p_amb=0.1)
    G = np.random.default_rng(seed + 100).standard_normal((5,) + tuple(shape))
    dt = 0.3 / oracle.Grid(shape, GAMMA, bc6).max_rate(U0)
    return U0, G, dt


def _adj_rank_main(rank, world, port, shape, bc6, seed, outdir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        L = slab.SlabLayout(shape[0], rank, world, bc_z=(bc6[4], bc6[5]))
        U0, G0, dt = _adj_inputs(shape, bc6, seed)
        U = torch.from_numpy(np.ascontiguousarray(U0[:, L.z0:L.z1]))
        G = torch.from_numpy(np.ascontiguousarray(G0[:, L.z0:L.z1]))
        gU, U1, gU1 = torch.empty_like(U), torch.empty_like(U), torch.empty_like(U)
        backend = TorchAdjointBackend(L, shape, bc6, GAMMA)
        x = slab.HaloExchange(L)
        slab.SlabAdjoint(backend, x).backward_step(U, U1, G, gU, gU1, dt)
        x.sum(backend.g_gamma)
        np.save(os.path.join(outdir, f"g{rank}.npy"), gU.numpy())
        np.save(os.path.join(outdir, f"gg{rank}.npy"), backend.g_gamma.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,shape,bc6", [
    (2, (12, 6, 8), [0, 0, 0, 0, 0, 0]),              # periodic: the same peer above and below
    (3, (13, 13, 13), [2, 2, 1, 1, 2, 2]),            # the blast, reflecting z ends, uneven slabs
])
def test_decomposed_adjoint_equals_whole_mesh_autograd(tmp_path, world, shape, bc6):
    from oracle import oracle_torch as ot
    seed = 6
    mp.spawn(_adj_rank_main, args=(world, _free_port(), shape, bc6, seed, str(tmp_path)),
             nprocs=world, join=True)
    got = np.concatenate([np.load(tmp_path / f"g{r}.npy") for r in range(world)], axis=1)
    ggs = [float(np.load(tmp_path / f"gg{r}.npy")[0]) for r in range(world)]
    U0, G0, dt = _adj_inputs(shape, bc6, seed)
    U = torch.tensor(U0, requires_grad=True)
    gam = torch.tensor(GAMMA, dtype=torch.float64, requires_grad=True)
    nz, ny, nx = shape
    out = ot.step(U, gam, dt, (1.0 / nx, 1.0 / ny, 1.0 / nz), bc6)
    ref, ref_gg = torch.autograd.grad(out, [U, gam], grad_outputs=torch.tensor(G0))
    ref = ref.numpy()
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) <= 1e-12 * scale
    assert all(abs(g - float(ref_gg)) <= 1e-10 * abs(float(ref_gg)) for g in ggs)
    assert np.max(np.abs(got - ref)) < np.max(np.abs(ref))   # not trivially zero
