"""Checkpoint and resume of a time loop.

A checkpoint holds what a run needs to continue: the conserved state U, the
simulated time t, the number of steps taken, the dt of each of them, and the
mesh description of the handle that took them (shape, gamma, boundary kinds,
extents, element type, scheme).  The next step's dt depends only on the
state (the CFL rate of U), so a run resumed from a checkpoint takes the same
steps as the uninterrupted run, bit for bit.

The file is written with ``torch.save`` from host copies (to a temporary
name, then renamed, so an interrupted write leaves the previous checkpoint
in place) and read with ``torch.load(weights_only=True)``: tensors, numbers,
strings and lists only.
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import torch

FORMAT = 1
_DTYPES = {"float32": torch.float32, "float64": torch.float64}


@dataclass
class Checkpoint:
    U: torch.Tensor                 # (5, nz, ny, nx) on the requested device
    t: float
    step: int
    dts: list = field(default_factory=list)
    mesh: dict = field(default_factory=dict)

    def handle(self, **kw):
        """A HardHydro handle for the saved mesh (kernel and tile as given)."""
        from . import HardHydro
        m = self.mesh
        return HardHydro(tuple(m["shape"]), m["gamma"], list(m["bc6"]),
                         dtype=_DTYPES[m["dtype"]], extent=tuple(m["extent"]),
                         scheme=m["scheme"], **kw)


def _dtype_name(dtype):
    for k, v in _DTYPES.items():
        if v == dtype:
            return k
    raise ValueError(f"unsupported element type {dtype}")


def save(path, m, U, t, step, dts=None):
    """Write U (device or host tensor of handle m's shape and type), the time t
    (float or 0-d tensor), the step count and the dt list to `path`."""
    if tuple(U.shape) != (5,) + tuple(m.shape):
        raise ValueError(f"U has shape {tuple(U.shape)}, the mesh {(5,) + tuple(m.shape)}")
    if U.dtype != m.dtype:
        raise ValueError("U's element type differs from the handle's")
    if int(step) < 0:
        raise ValueError("step must be >= 0")
    if dts is not None and len(dts) != int(step):
        raise ValueError("one dt per step taken")
    payload = {
        "format": FORMAT,
        "U": U.detach().to("cpu").contiguous(),
        "t": float(t),
        "step": int(step),
        "dts": [float(d) for d in (dts if dts is not None else [])],
        "mesh": {"shape": list(m.shape), "gamma": float(m.gamma), "bc6": list(m.bc6),
                 "extent": list(m.extent), "dtype": _dtype_name(m.dtype),
                 "scheme": int(m.scheme)},
    }
    tmp = f"{path}.tmp"
    torch.save(payload, tmp)
    os.replace(tmp, path)


def load(path, device="cuda") -> Checkpoint:
    """Read a checkpoint written by `save`; U is placed on `device`."""
    p = torch.load(path, map_location="cpu", weights_only=True)
    if not isinstance(p, dict) or p.get("format") != FORMAT:
        raise ValueError(f"{path}: not a checkpoint of format {FORMAT}")
    mesh = p["mesh"]
    U = p["U"]
    if tuple(U.shape) != (5,) + tuple(mesh["shape"]) or U.dtype != _DTYPES[mesh["dtype"]]:
        raise ValueError(f"{path}: the state does not match the mesh description")
    if len(p["dts"]) not in (0, p["step"]):
        raise ValueError(f"{path}: the dt list does not match the step count")
    return Checkpoint(U=U.to(device), t=p["t"], step=p["step"], dts=list(p["dts"]), mesh=mesh)
