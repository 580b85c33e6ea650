"""Decomposition of a 3D mesh into z slabs, one per rank of a process group.

The paper distributes its mesh over ranks with exclusive, shared and ghost
entities (the N-Array layout of Sec. 2.1) and scales it over many nodes
(Sec. 3.6).  Here the nz planes are split into contiguous slabs (sizes differ
by at most one plane), each rank advancing its slab with its own handle whose
z faces towards a neighbour are ``HARD_BC_HALO``.  Every stage reads two ghost
planes on each side, so a step is:

    exchange the two boundary planes of U^n with the neighbours,
    stage 1 (U1 = U^n + dt L(U^n)),
    exchange the two boundary planes of U1,
    stage 2 (U^{n+1} = U^n/2 + (U1 + dt L(U1))/2) with the signal rate of U^{n+1},
    the largest rate over all ranks (one all-reduce of one double),
    the next step's dt = cfl / rate (Sec. 3.5's CFL-limited step).

The exchange sends each rank's packed boundary planes ([5][2][ny][nx]) to its
neighbours and receives theirs into its own ghost buffers, by point-to-point
sends of ``torch.distributed`` (NCCL between GPUs, gloo on CPU): no kernel
ever reads another rank's memory.  The stage arithmetic belongs to a backend:
``CudaSlabBackend`` runs this library's kernels; the tests plug in the CPU
oracle to check the partition and exchange logic against a single-rank run.
"""
from __future__ import annotations

from . import (HARD_BC_HALO, HARD_BC_PERIODIC, HardHydro, check, hard_hydro_add_zghost_cotangent,
               hard_hydro_finalize_dt, hard_hydro_local_rate, hard_hydro_pack_zhalo,
               hard_hydro_set_cells, hard_hydro_set_zghost, hard_hydro_set_zghost_adjoint,
               hard_hydro_stage_ex, hard_hydro_stage_vjp_cells, hard_hydro_stage_vjp_faces)


def partition(nz: int, world: int) -> list[tuple[int, int]]:
    """Contiguous plane ranges [z0, z1) of the ranks, lowest rank lowest; the
    first nz % world ranks take one plane more."""
    if world < 1 or nz < 1:
        raise ValueError("need nz >= 1 and world >= 1")
    base, extra = divmod(nz, world)
    out, z = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


class SlabLayout:
    """Rank `rank`'s slab of an nz-plane mesh over `world` ranks.

    ``lo`` / ``hi`` are the ranks holding the planes just below / above the
    slab (periodic z wraps around the ring), or None at a physical z face.
    ``bc_z`` gives the slab's own z face kinds: HARD_BC_HALO towards a
    neighbour, the mesh's kind at a physical face."""

    def __init__(self, nz: int, rank: int, world: int, bc_z=(HARD_BC_PERIODIC, HARD_BC_PERIODIC)):
        if not 0 <= rank < world:
            raise ValueError("rank out of range")
        periodic = bc_z[0] == HARD_BC_PERIODIC
        if periodic != (bc_z[1] == HARD_BC_PERIODIC):
            raise ValueError("periodic must be set on both z faces or on neither")
        self.nz, self.rank, self.world = int(nz), int(rank), int(world)
        self.z0, self.z1 = partition(self.nz, self.world)[self.rank]
        if self.world > 1 and self.z1 - self.z0 < 2:
            raise ValueError("every slab needs at least two planes (two ghost planes per side)")
        if self.world == 1:
            self.lo = self.hi = None
        elif periodic:
            self.lo = (self.rank - 1) % self.world
            self.hi = (self.rank + 1) % self.world
        else:
            self.lo = self.rank - 1 if self.rank > 0 else None
            self.hi = self.rank + 1 if self.rank < self.world - 1 else None
        self.bc_z = (HARD_BC_HALO if self.lo is not None else int(bc_z[0]),
                     HARD_BC_HALO if self.hi is not None else int(bc_z[1]))

    @property
    def planes(self) -> int:
        return self.z1 - self.z0


class HaloExchange:
    """Ghost-plane exchange and the rate reduction over a process group."""

    def __init__(self, layout: SlabLayout, group=None):
        self.layout = layout
        self.group = group

    def run(self, send_lo, send_hi, recv_lo, recv_hi):
        """Send the two bottom planes down and the two top planes up; receive
        the lower neighbour's top planes into recv_lo and the upper
        neighbour's bottom planes into recv_hi.  Upward transfers are posted
        before downward ones on every rank, and tagged apart, so that the two
        messages between the same pair of ranks (two slabs on a periodic
        axis) match whether the backend matches by tag or by order."""
        import torch.distributed as dist
        L = self.layout
        ops = []
        if L.hi is not None:
            ops.append(dist.P2POp(dist.isend, send_hi, L.hi, self.group, tag=0))
        if L.lo is not None:
            ops.append(dist.P2POp(dist.irecv, recv_lo, L.lo, self.group, tag=0))
        if L.lo is not None:
            ops.append(dist.P2POp(dist.isend, send_lo, L.lo, self.group, tag=1))
        if L.hi is not None:
            ops.append(dist.P2POp(dist.irecv, recv_hi, L.hi, self.group, tag=1))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()

    def max(self, t):
        """In place: the largest value of t over the ranks."""
        if self.layout.world > 1:
            import torch.distributed as dist
            dist.all_reduce(t, op=dist.ReduceOp.MAX, group=self.group)
        return t

    def sum(self, t):
        """In place: the sum of t over the ranks."""
        if self.layout.world > 1:
            import torch.distributed as dist
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t


class SlabStepper:
    """The time loop of one rank over its slab (see the module docstring).

    The backend provides ``send_lo, send_hi, ghost_lo, ghost_hi`` (the
    packed boundary planes and the ghost buffers, None at a physical face),
    ``rate`` (a one-element float64 tensor), ``pack(U)``,
    ``stage(stage, U0, Ucur, out, with_rate)``, ``local_rate(U)`` and
    ``finalize(cfl, t_end)`` (dt of the next step from ``rate``, t
    advanced)."""

    def __init__(self, backend, exchange: HaloExchange):
        self.b = backend
        self.x = exchange

    def exchange(self, U):
        b = self.b
        b.pack(U)
        self.x.run(b.send_lo, b.send_hi, b.ghost_lo, b.ghost_hi)

    def advance(self, U, U1, nsteps: int, cfl: float, t_end: float = 0.0):
        """In place on U (U1: scratch of the same shape): nsteps steps, each
        with the dt of the whole mesh's signal rate at its start."""
        b = self.b
        if nsteps <= 0:
            return
        b.local_rate(U)
        self.x.max(b.rate)
        b.finalize(cfl, t_end)
        for step in range(nsteps):
            self.exchange(U)
            b.stage(1, U, U, U1, False)
            self.exchange(U1)
            b.stage(2, U, U1, U, True)
            self.x.max(b.rate)
            if step + 1 < nsteps:
                b.finalize(cfl, t_end)


class SlabAdjoint:
    """The adjoint of a step on one rank's slab (dt held constant): the
    forward ghost exchange, reversed for the cotangents.

    Each stage's VJP is split around an exchange: the face pass leaves the
    cotangent of the cells on the neighbours' planes in ``adj_send_lo`` /
    ``adj_send_hi``, which go to the rank below / above; what they send back
    arrives in ``adj_recv_lo`` / ``adj_recv_hi`` and is added before the cell
    pass.  The backend provides, besides the forward stepper's interface,
    ``set_dt(dt)``, ``vjp_faces(stage, Uc, G)``, ``vjp_add()``,
    ``vjp_cells(stage, Uc, G, gUc, accumulate, gU0)`` and ``g_gamma`` (a
    one-element float64 tensor the passes add to)."""

    def __init__(self, backend, exchange: HaloExchange):
        self.b = backend
        self.x = exchange
        self.fwd = SlabStepper(backend, exchange)

    def _reverse(self):
        b = self.b
        self.x.run(b.adj_send_lo, b.adj_send_hi, b.adj_recv_lo, b.adj_recv_hi)
        b.vjp_add()

    def backward_step(self, U, U1, G, gU, gU1, dt):
        """gU = (dU^{n+1}/dU^n)^T G for this slab's cells (U1, gU1: scratch of
        U's shape); the slab's d/dgamma is added to the backend's g_gamma
        (sum it over the ranks with ``exchange.sum``)."""
        b = self.b
        b.set_dt(dt)
        self.fwd.exchange(U)
        b.stage(1, U, U, U1, False)                    # recompute U1
        self.fwd.exchange(U1)
        b.vjp_faces(2, U1, G)
        self._reverse()
        b.vjp_cells(2, U1, G, gU1, False, gU)          # gU1 = G/2 + J^T, gU = G/2
        self.fwd.exchange(U)
        b.vjp_faces(1, U, gU1)
        self._reverse()
        b.vjp_cells(1, U, gU1, gU, True, None)         # gU += gU1 + J^T


def slab_handle(shape, layout: SlabLayout, gamma, bc6, dtype=None, kernel=0, tile=-1,
                extent=(1.0, 1.0, 1.0)) -> HardHydro:
    """A handle for rank `layout.rank`'s slab of the (nz, ny, nx) mesh: its
    planes, the mesh's x/y faces, HARD_BC_HALO towards neighbours, and the
    whole mesh's cell widths."""
    nz, ny, nx = (int(s) for s in shape)
    if nz != layout.nz:
        raise ValueError("the layout was made for another number of planes")
    bc = list(bc6)
    bc[4], bc[5] = layout.bc_z
    m = HardHydro((layout.planes, ny, nx), gamma, bc, dtype=dtype,
                  extent=(extent[0], extent[1], extent[2] * layout.planes / nz), kernel=kernel,
                  tile=tile)
    check(hard_hydro_set_cells(m.h, extent[0] / nx, extent[1] / ny, extent[2] / nz),
          "hard_hydro_set_cells")
    return m


class CudaSlabBackend:
    """Stage arithmetic on this library's kernels for a slab handle (made by
    `slab_handle`), on the current CUDA device and stream.  dt, t and the
    rate stay on the device."""

    def __init__(self, m: HardHydro, layout: SlabLayout):
        torch = m.torch
        self.m = m
        self.torch = torch
        _, ny, nx = m.shape
        dev = torch.device("cuda", torch.cuda.current_device())

        def buf(on):
            return torch.zeros((5, 2, ny, nx), dtype=m.dtype, device=dev) if on else None

        lo, hi = layout.lo is not None, layout.hi is not None
        self.send_lo, self.send_hi = buf(lo), buf(hi)
        self.ghost_lo, self.ghost_hi = buf(lo), buf(hi)
        check(hard_hydro_set_zghost(m.h, self._p(self.ghost_lo), self._p(self.ghost_hi)),
              "hard_hydro_set_zghost")
        self.rate = torch.zeros(1, dtype=torch.float64, device=dev)
        self.dt = torch.zeros((), dtype=torch.float64, device=dev)
        self.t = torch.zeros((), dtype=torch.float64, device=dev)

    @staticmethod
    def _p(t):
        return None if t is None else t.data_ptr()

    def _stream(self):
        return self.torch.cuda.current_stream().cuda_stream

    def pack(self, U):
        check(hard_hydro_pack_zhalo(self.m.h, self.m._check(U), self._p(self.send_lo),
                                    self._p(self.send_hi), self._stream()),
              "hard_hydro_pack_zhalo")

    def stage(self, stage, U0, Ucur, out, with_rate):
        m = self.m
        check(hard_hydro_stage_ex(m.h, stage, m._check(U0), m._check(Ucur), m._check(out), 0.0,
                                  self.dt.data_ptr(), self.rate.data_ptr() if with_rate else None,
                                  self._stream()), "hard_hydro_stage_ex")

    def local_rate(self, U):
        check(hard_hydro_local_rate(self.m.h, self.m._check(U), self.rate.data_ptr(),
                                    self._stream()), "hard_hydro_local_rate")

    def finalize(self, cfl, t_end):
        check(hard_hydro_finalize_dt(self.m.h, self.rate.data_ptr(), cfl, t_end, self.t.data_ptr(),
                                     self.dt.data_ptr(), self._stream()), "hard_hydro_finalize_dt")

    # ---- the adjoint (SlabAdjoint) ----

    def set_dt(self, dt):
        """Fix the step's dt (host value, also the forward stages' dt)."""
        if not hasattr(self, "g_gamma"):
            torch, m = self.torch, self.m
            _, ny, nx = m.shape
            dev = self.rate.device

            def acc(on):
                return torch.zeros((2, ny, nx, 8), dtype=m.dtype, device=dev) if on else None

            lo, hi = self.send_lo is not None, self.send_hi is not None
            self.adj_send_lo, self.adj_send_hi = acc(lo), acc(hi)
            self.adj_recv_lo, self.adj_recv_hi = acc(lo), acc(hi)
            check(hard_hydro_set_zghost_adjoint(m.h, self._p(self.adj_send_lo),
                                                self._p(self.adj_send_hi)),
                  "hard_hydro_set_zghost_adjoint")
            self.g_gamma = torch.zeros(1, dtype=torch.float64, device=dev)
        self.dt_host = float(dt)
        self.dt.fill_(self.dt_host)

    def vjp_faces(self, stage, Uc, G):
        m = self.m
        check(hard_hydro_stage_vjp_faces(m.h, stage, m._check(Uc), m._check(G), self.dt_host,
                                         self.g_gamma.data_ptr(), self._stream()),
              "hard_hydro_stage_vjp_faces")

    def vjp_add(self):
        check(hard_hydro_add_zghost_cotangent(self.m.h, self._p(self.adj_recv_lo),
                                              self._p(self.adj_recv_hi), self._stream()),
              "hard_hydro_add_zghost_cotangent")

    def vjp_cells(self, stage, Uc, G, gUc, accumulate, gU0):
        m = self.m
        check(hard_hydro_stage_vjp_cells(m.h, stage, m._check(Uc), m._check(G), m._check(gUc),
                                         accumulate, None if gU0 is None else m._check(gU0),
                                         self.g_gamma.data_ptr(), self._stream()),
              "hard_hydro_stage_vjp_cells")


# ---- independent problems (the batched configuration) ----

def lpt_partition(costs, world: int) -> list[list[int]]:
    """Split independent problems over `world` ranks with no exchange between
    them: longest processing time first (problems in decreasing cost, each to
    the rank with the least load so far; ties to the lower problem index and
    the lower rank), so that the most loaded rank carries at most the mean
    load plus one problem's cost.  Returns each rank's problem indices in
    increasing order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = [float(c) for c in costs]
    order = sorted(range(len(costs)), key=lambda p: (-costs[p], p))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for p in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(p)
        load[r] += costs[p]
    return [sorted(q) for q in parts]
