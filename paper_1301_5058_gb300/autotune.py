"""Autotuner for the batched and single-grid steppers.

The knobs change no result bit (include/cx.h): the tile height of the step
kernel, the temporal blocking depth (explicit stages per pass), the number
of steps captured per CUDA graph, the size of the instance groups a batch
runs back to back (to keep a group resident in L2), and how many steps a
group advances per resident (cooperative) launch.
Each candidate is timed with CUDA events on the handle's stream after a
warm-up; the fastest is applied and cached in a JSON file keyed by
precision, scheme and the mix of grid sizes (CX_TUNE_CACHE, default
~/.cache/cx_tune.json).
"""
from __future__ import annotations

import json
import os
from collections import Counter

import paper_1301_5058_gb300 as cx

L2_BYTES = 126 * 2 ** 20   # GB300 L2 (about 126 MiB usable)

# (tile rows, graph steps, group bytes, resident steps, stages per pass):
# one launch per pass over every instance at either depth; L2-sized groups
# stepped by resident launches (one stage per pass) are searched only when
# asked for (RESIDENT_CANDIDATES: they have never won on GB300)
BATCH_CANDIDATES = [(rows, graph, 0, 0, depth) for depth in (1, 2) for rows in (16, 32, 64, 128)
                    for graph in (0, 64)]
RESIDENT_CANDIDATES = [(rows, 0, group, res, 1) for rows in (4, 8, 16)
                       for group in (L2_BYTES // 2, L2_BYTES // 4) for res in (50, 200)]
SINGLE_CANDIDATES = (2, 4, 8, 16, 32, 64, 128, 256)


def cache_path() -> str:
    return os.environ.get("CX_TUNE_CACHE", os.path.expanduser("~/.cache/cx_tune.json"))


def _load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, value) -> None:
    d = _load_cache()
    d[key] = value
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def batch_key(grids, params) -> str:
    mix = Counter((g.nx, g.ny) for g in grids)
    sizes = ",".join(f"{nx}x{ny}:{c}" for (nx, ny), c in sorted(mix.items()))
    return f"batch/p{params[0].precision}/s{params[0].scheme}/{sizes}"


def _time_steps(torch, stream, fn, steps: int, reps: int) -> float:
    """Median seconds per step of fn(steps), measured with CUDA events."""
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn(steps)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b) / 1e3 / steps)
    times.sort()
    return times[len(times) // 2]


def tune_batch(batch: "cx.Batch", steps: int = 128, reps: int = 3, candidates=None,
               use_cache: bool = True, verbose: bool = False):
    """Pick (tile_rows, graph_steps, group_bytes, resident_steps, stages per
    pass) for `batch`, apply it and return (choice, {candidate: seconds per
    step}).  The timed steps advance the batch's state."""
    import torch
    key = batch_key(batch.grids, batch.params)
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            choice = tuple(hit["choice"])
            batch.tune(*choice)
            return choice, {}
    stream = getattr(batch, "_stream", None)
    if stream is None:
        # graph capture needs a real stream, not the legacy default one; the
        # batch keeps a reference so the stream outlives this call
        stream = torch.cuda.Stream()
        cx.cx_batch_set_stream(batch.h, stream.cuda_stream)
        batch._stream = stream
    results = {}
    for cand in candidates or BATCH_CANDIDATES:
        batch.tune(*cand)
        batch.step(steps)                      # warm-up (and graph capture)
        results[cand] = _time_steps(torch, stream, batch.step, steps, reps)
        if verbose:
            print(f"  rows={cand[0]:3d} graph={cand[1]:3d} group={cand[2] >> 20:4d} MiB "
                  f"resident={cand[3]:4d} depth={cand[4]}: {results[cand] * 1e6:9.1f} us/step")
    choice = min(results, key=results.get)
    batch.tune(*choice)
    _store(key, {"choice": list(choice), "us_per_step": results[choice] * 1e6})
    return choice, results


def tune_single(sim: "cx.Sim", steps: int = 20, reps: int = 3, use_cache: bool = True):
    """Pick the temporal blocking depth and tile height of a single grid;
    applies the winner and returns ((time_block, rows), timings)."""
    import torch
    key = f"single/p{sim.params.precision}/s{sim.params.scheme}/n{sim.params.noise_mode}/" \
          f"{sim.grid.nx}x{sim.grid.ny}"
    if use_cache:
        hit = _load_cache().get(key)
        if hit and isinstance(hit.get("choice"), list):
            cx.cx_set_time_block(sim.h, hit["choice"][0])
            cx.cx_set_tile_rows(sim.h, hit["choice"][1])
            return tuple(hit["choice"]), {}
    stream = torch.cuda.current_stream()
    cx.cx_set_stream(sim.h, stream.cuda_stream)
    results = {}
    for depth in (1, 2):
        cx.cx_set_time_block(sim.h, depth)
        for rows in SINGLE_CANDIDATES:
            if (sim.grid.ny + rows - 1) // rows > 65535:
                continue
            cx.cx_set_tile_rows(sim.h, rows)
            sim.step(steps)
            results[(depth, rows)] = _time_steps(torch, stream, sim.step, steps, reps)
    choice = min(results, key=results.get)
    cx.cx_set_time_block(sim.h, choice[0])
    cx.cx_set_tile_rows(sim.h, choice[1])
    _store(key, {"choice": list(choice), "us_per_step": results[choice] * 1e6})
    return choice, results
