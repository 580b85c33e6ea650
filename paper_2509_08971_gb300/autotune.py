"""Tile autotuner for the stage kernel.

For a mesh, element type and kernel variant it times every tile
configuration the library offers (tile extents, threads per block, z-chunk
length; `hard_hydro_tile_info`) on the caller's own state: each candidate
runs a few untimed stage-1/stage-2 pairs, then a timed batch bracketed by
CUDA events on the current stream.  The fastest tile is set on the handle and
remembered in a JSON cache keyed by mesh shape, boundary kinds per face,
extents, element type, kernel, scheme and gamma (``HARD_HYDRO_TUNE_CACHE``
names the file; unset = in-memory only): the boundary kinds decide which tiles
take the generic ghost path, so a tile tuned on one kind is not reused for
another.

``tune_batch`` does the same for the persistent batched launch: it times each
batched tile set (`hard_batch_tile_count`) on a few steps of the caller's
packed batch and keeps the fastest, keyed by the batch's problem sizes,
boundary kinds and element type.
"""
from __future__ import annotations

import json
import os

import hashlib

from . import HardHydro, hard_batch_tile_count

_memory: dict[str, int] = {}


def _key(m: HardHydro, kernel: int) -> str:
    return (f"{m.shape}|bc{m.bc6}|ext{m.extent}|{m.dtype}|k{kernel}|s{m.scheme}|g{m.gamma}")


def _load_cache(path):
    if not path or not os.path.exists(path):
        return {}
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def tune(m: HardHydro, U, kernel: int = 0, reps: int = 10, warmup: int = 2,
         cache_path: str | None = None, verbose: bool = False) -> dict:
    """Pick the fastest tile for handle `m` on state `U` and set it.
    Returns {"tile": best, "info": (tx, ty, zc, threads), "ms": {tile: ms}}."""
    torch = m.torch
    cache_path = cache_path if cache_path is not None else os.environ.get("HARD_HYDRO_TUNE_CACHE")
    key = _key(m, kernel)
    disk = _load_cache(cache_path)
    if key in disk or key in _memory:
        best = int(disk.get(key, _memory.get(key)))
        m.set_kernel(kernel, best)
        return {"tile": best, "info": m.tile_info(best), "ms": {}, "cached": True}
    stream = torch.cuda.current_stream()
    U1 = torch.empty_like(U)
    U2 = torch.empty_like(U)
    dt = m.cfl_dt(U, 0.4)
    times = {}
    # two sweeps, the faster of each tile's two timings: a host-side stall in
    # one timed window (process start-up work, another process) cannot decide
    for sweep in range(2):
        for tile in range(m.tile_count()):
            m.set_kernel(kernel, tile)
            for _ in range(warmup):
                m.stage(1, None, U, dt, out=U1)
                m.stage(2, U, U1, dt, out=U2)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                m.stage(1, None, U, dt, out=U1)
                m.stage(2, U, U1, dt, out=U2)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / (2 * reps)
            times[tile] = min(ms, times.get(tile, ms))
            if verbose:
                print(f"tile {tile} {m.tile_info(tile)}: {ms:.4f} ms per stage")
    best = min(times, key=times.get)
    m.set_kernel(kernel, best)
    _memory[key] = best
    if cache_path:
        disk[key] = best
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(disk, fh, indent=1)
        os.replace(tmp, cache_path)
    return {"tile": best, "info": m.tile_info(best), "ms": times, "cached": False}


def _batch_key(B) -> str:
    h = hashlib.sha256()
    h.update(repr((B.nx, B.ny, B.bcs, B.gammas, str(B.dtype))).encode())
    return "batch|" + h.hexdigest()[:32]


def tune_batch(B, packed, cfl: float, steps: int = 5, cache_path: str | None = None) -> dict:
    """Time every batched tile set on `steps` steps of a copy of the packed
    batch (the caller's tensor is not changed), set the fastest on the batch
    and return {"tile": best, "ms": {tile: ms}}."""
    torch = B.torch
    cache_path = cache_path if cache_path is not None else os.environ.get("HARD_HYDRO_TUNE_CACHE")
    key = _batch_key(B)
    disk = _load_cache(cache_path)
    if key in disk or key in _memory:
        best = int(disk.get(key, _memory.get(key)))
        B.set_tile(best)
        return {"tile": best, "ms": {}, "cached": True}
    stream = torch.cuda.current_stream()
    times = {}
    for tile in range(hard_batch_tile_count()):
        B.set_tile(tile)
        P = packed.clone()
        B.step(P, 1, cfl)                       # warm-up (module load, first touch)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.step(P, steps, cfl)
        e1.record(stream)
        torch.cuda.synchronize()
        times[tile] = e0.elapsed_time(e1)
        del P
    best = min(times, key=times.get)
    B.set_tile(best)
    _memory[key] = best
    if cache_path:
        disk[key] = best
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(disk, fh, indent=1)
        os.replace(tmp, cache_path)
    return {"tile": best, "ms": times, "cached": False}
