"""Autotuner of the batching form's evaluation tile.

For each class of runs -- (precision, d_in, hidden width, d_out, 128-sample
tiles per batch) -- it times the evaluation on the device with every
candidate tile and keeps the fastest.  The tile is the tensor-core MMA's
M x N: M is the 128-sample tile, N = group x hidden with `group` individuals
of the run per MMA in the group evaluation (the candidates: the most that fit
in N <= 256, and halvings), or, where that evaluation does not take the
shape, N = the hidden chunk of the chunked evaluation (the columns of the
TMEM accumulator next to the batch tile).  The pipeline's stage depth is not
a candidate: shared memory fixes it (four stages of BF16, three of FP8, at
N = 256).  Results are cached in a JSON file keyed by device name and class,
so a later process reuses them without timing.
"""
from __future__ import annotations

import dataclasses
import json
import os

from . import leea

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
TMEM_COLUMNS, MAX_CHUNK = 512, 128
MAX_N, MAX_GROUP = 256, 16


def max_group(hidden: int) -> int:
    """Most individuals of width `hidden` that share one MMA (N = group hidden <= 256)."""
    return max(1, min(MAX_GROUP, MAX_N // hidden))


def group_candidates(hidden: int, extra: int = 2) -> list[int]:
    """The widest group and up to `extra` halvings of it."""
    out = [max_group(hidden)]
    while len(out) <= extra and out[-1] > 1:
        out.append(max(1, out[-1] // 2))
    return out


def max_chunk(precision: int, d_in: int) -> int:
    """Widest hidden chunk the tensor memory holds next to the batch tile."""
    if precision == 1:
        a_cols = -(-(8 * -(-d_in // 16)) // 16) * 16
    else:
        a_cols = -(-(2 * 8 * -(-d_in // 32)) // 16) * 16
    return min(MAX_CHUNK, (TMEM_COLUMNS - a_cols) // 16 * 16)


def effective_chunk(hidden: int, chunk: int) -> int:
    """The chunk the kernel uses for a requested one: equal chunks of ceil(h / n) rounded up to 16."""
    cw = min(chunk, hidden)
    n = -(-hidden // cw)
    return -(-(-(-hidden // n)) // 16) * 16


def candidates(precision: int, d_in: int, hidden: int, extra: int = 2) -> list[int]:
    """Distinct effective chunks: the fewest chunks the tensor memory allows, and up to `extra` more."""
    cw_max = max_chunk(precision, d_in)
    n_min = -(-hidden // cw_max)
    out = []
    for n in range(n_min, n_min + extra + 1):
        cw = effective_chunk(hidden, -(-(-(-hidden // n)) // 16) * 16)
        if 16 <= cw <= cw_max and cw not in out:
            out.append(cw)
    return out


def _sm_count() -> int:
    try:
        import torch
        return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    except Exception:
        return 152


def _device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(torch.cuda.current_device())
    except Exception:
        return "unknown"


def _key(device: str, precision: int, d_in: int, hidden: int, d_out: int, tiles: int) -> str:
    return f"{device}|p{precision}|{d_in}-{hidden}-{d_out}|tiles{tiles}|v2"


def tune(specs, d_in: int, d_out: int, precision: int, cache_path: str | None = DEFAULT_CACHE,
         pop: int = 608, reps: int = 3):
    """Returns (specs with `group` -- or, where the group evaluation does not take a class, `chunk` --
    chosen, {class key: {candidate: ms}} of the timings taken now)."""
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
    device = _device_name()
    timings = {}
    out = []
    for sp in specs:
        tiles = -(-sp.batch // 128)
        key = _key(device, precision, d_in, sp.hidden, d_out, tiles)
        if key not in cache:
            batch = min(sp.batch, 128 * tiles)
            times, knob = {}, "group"
            # enough individuals for two units of the widest group per SM, so that
            # the timing measures throughput, not how many units there are
            pop_g = max(pop, 2 * _sm_count() * max_group(sp.hidden))
            try:
                for g in group_candidates(sp.hidden):
                    times[g] = leea.leea_tune_group_eval(precision, d_in, sp.hidden, d_out, batch, pop_g, g, reps)
            except leea.LeeaError:  # the group evaluation does not take this class
                times, knob = {}, "chunk"
                for cw in candidates(precision, d_in, sp.hidden):
                    times[cw] = leea.leea_tune_shadow_eval(precision, d_in, sp.hidden, d_out, batch, pop, cw, reps)
            best = min(times, key=times.get)
            cache[key] = {knob: best, "ms": {str(k): v for k, v in times.items()}}
            timings[key] = times
        entry = cache[key]
        out.append(dataclasses.replace(sp, group=int(entry["group"])) if "group" in entry
                   else dataclasses.replace(sp, chunk=int(entry["chunk"])))
    if cache_path and timings:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return out, timings
