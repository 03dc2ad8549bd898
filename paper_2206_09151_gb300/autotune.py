"""Autotuner for the run-time shape choices of the reconstruction.

The kernels' voxel tiles and FFT groups are fixed at compile time for sm_103a; what
varies per problem is how many directions share one block of layer stacks (``dir_block``
of a run: a larger block means fewer volume read-modify-writes but a larger workspace),
how a warp of the direct general backprojection covers its tile's voxel columns
(``bp_warp``: 8 x 4, 16 x 2 or 32 x 1, which sets how many detector rows and cache lines one
gather touches for the scan's view orientations), the voxel tile of the TMA-staged
backprojection (``bp_tile_z``: 16 x 16 x 8 or 16 x 16 x 16), and how many directions a
batch round holds.  Each ``tune_*`` times ``recon_run`` (or a batch run) for every
candidate with CUDA events after a warm-up run and returns the fastest; ``tune_dir_block``,
``tune_bp_warp`` and ``tune_bp_tile`` cache their result per problem shape in a JSON file
when ``cache`` is given."""
from __future__ import annotations

import json
import os

import torch

from .recon import Batch, Reconstructor


def _key(rot, nu, nv, grid, nz_layers, kw) -> str:
    return json.dumps([int(len(rot)), nu, nv, list(grid), nz_layers, kw.get("stack_dtype", "f32"),
                       kw.get("filter", "tikhonov"), kw.get("ramp", "single_axis"),
                       torch.cuda.get_device_name()])


def _time(fn, repeats: int) -> float:
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune_dir_block(rot, nu: int, nv: int, grid, images: torch.Tensor, *, nz_layers: int, candidates=None,
                   repeats: int = 3, cache: str | None = None, memory_fraction: float = 0.5, **plan_kw) -> dict:
    """Fastest direction block for this problem: {"dir_block": best, "ms": {candidate: ms}}.
    Candidates whose workspace exceeds ``memory_fraction`` of the free device memory are
    skipped."""
    key = _key(rot, nu, nv, grid, nz_layers, plan_kw)
    if cache and os.path.exists(cache):
        table = json.load(open(cache))
        if key in table:
            return table[key]
    D = len(rot)
    if candidates is None:
        candidates = sorted({c for c in (8, 16, 32, 60, 90, 120, 180, 360) if c <= D} | {D})
    free = torch.cuda.mem_get_info()[0]
    timings = {}
    vol = None
    for c in candidates:
        r = Reconstructor(rot, nu, nv, grid, nz_layers=nz_layers, dir_block=c, allocate=False, **plan_kw)
        if r.ws_bytes > memory_fraction * free:
            r.close()
            continue
        r.workspace = torch.empty(max(r.ws_bytes, 256), dtype=torch.uint8, device=images.device)
        if vol is None:
            vol = r.new_volume()
        timings[c] = _time(lambda: r.run(images, vol), repeats)
        r.close()
        del r
        torch.cuda.empty_cache()
    best = min(timings, key=timings.get)
    out = {"dir_block": best, "ms": {str(k): v for k, v in timings.items()}}
    if cache:
        table = json.load(open(cache)) if os.path.exists(cache) else {}
        table[key] = out
        with open(cache, "w") as f:
            json.dump(table, f, indent=1)
    return out


def tune_bp_warp(rot, nu: int, nv: int, grid, images: torch.Tensor, *, nz_layers: int, candidates=(8, 16, 32),
                 repeats: int = 3, cache: str | None = None, **plan_kw) -> dict:
    """Fastest warp patch of the general backprojection: {"bp_warp": best, "ms": {...}}.
    The shapes give the same volume bit for bit (they only move voxels between threads)."""
    key = _key(rot, nu, nv, grid, nz_layers, plan_kw) + "|bp_warp"
    if cache and os.path.exists(cache):
        table = json.load(open(cache))
        if key in table:
            return table[key]
    timings = {}
    vol = None
    for c in candidates:
        r = Reconstructor(rot, nu, nv, grid, nz_layers=nz_layers, bp_warp=c, **plan_kw)
        if vol is None:
            vol = r.new_volume()
        timings[c] = _time(lambda: r.run(images, vol), repeats)
        r.close()
        del r
        torch.cuda.empty_cache()
    best = min(timings, key=timings.get)
    out = {"bp_warp": best, "ms": {str(k): v for k, v in timings.items()}}
    if cache:
        table = json.load(open(cache)) if os.path.exists(cache) else {}
        table[key] = out
        with open(cache, "w") as f:
            json.dump(table, f, indent=1)
    return out


def tune_bp_tile(rot, nu: int, nv: int, grid, images: torch.Tensor, *, nz_layers: int, candidates=(8, 16),
                 repeats: int = 3, cache: str | None = None, **plan_kw) -> dict:
    """Fastest voxel-tile depth of the TMA-staged backprojection (16 x 16 x 8 or 16 x 16 x 16
    tiles): {"bp_tile_z": best, "ms": {...}}.  Timed with ``bp_kernel="tma"``; a deeper
    tile shares each direction's set-up over more voxels, a shallower one wastes less at
    the volume's z edge and stages smaller boxes."""
    plan_kw = dict(plan_kw, bp_kernel="tma")
    key = _key(rot, nu, nv, grid, nz_layers, plan_kw) + "|bp_tile_z"
    if cache and os.path.exists(cache):
        table = json.load(open(cache))
        if key in table:
            return table[key]
    timings = {}
    vol = None
    for c in candidates:
        r = Reconstructor(rot, nu, nv, grid, nz_layers=nz_layers, bp_tile_z=c, **plan_kw)
        if vol is None:
            vol = r.new_volume()
        timings[c] = _time(lambda: r.run(images, vol), repeats)
        r.close()
        del r
        torch.cuda.empty_cache()
    best = min(timings, key=timings.get)
    out = {"bp_tile_z": best, "ms": {str(k): v for k, v in timings.items()}}
    if cache:
        table = json.load(open(cache)) if os.path.exists(cache) else {}
        table[key] = out
        with open(cache, "w") as f:
            json.dump(table, f, indent=1)
    return out


def tune_batch_round(recons, images, *, candidates=(8, 16, 32, 64), repeats: int = 3) -> dict:
    """Fastest round size (directions per tomogram per persistent launch) for a batch."""
    timings = {}
    for c in candidates:
        b = Batch(recons, dir_block=c)
        vols = [r.new_volume() for r in recons]
        timings[c] = _time(lambda: b.run(images, vols), repeats)
        b.close()
        del b
        torch.cuda.empty_cache()
    best = min(timings, key=timings.get)
    return {"dir_block": best, "ms": {str(k): v for k, v in timings.items()}}
