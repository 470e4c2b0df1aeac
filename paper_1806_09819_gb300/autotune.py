"""Autotuner of the batching form's evaluation tile.

For each class of runs -- (precision, d_in, hidden width, d_out, 128-sample
tiles per batch) -- it times the shadow evaluation on the device with every
candidate hidden chunk (the N of the tensor-core MMA, the columns of the TMEM
accumulator) and keeps the fastest.  Results are cached in a JSON file keyed
by device name and class, so a later process reuses them without timing.
"""
from __future__ import annotations

import dataclasses
import json
import os

from . import leea

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
TMEM_COLUMNS, MAX_CHUNK = 512, 128


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


def _device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(torch.cuda.current_device())
    except Exception:
        return "unknown"


def _key(device: str, precision: int, d_in: int, hidden: int, d_out: int, tiles: int) -> str:
    return f"{device}|p{precision}|{d_in}-{hidden}-{d_out}|tiles{tiles}"


def tune(specs, d_in: int, d_out: int, precision: int, cache_path: str | None = DEFAULT_CACHE,
         pop: int = 608, reps: int = 3):
    """Returns (specs with `chunk` chosen, {class key: {chunk: ms}} of the timings taken now)."""
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
            times = {}
            for cw in candidates(precision, d_in, sp.hidden):
                times[cw] = leea.leea_tune_shadow_eval(precision, d_in, sp.hidden, d_out, min(sp.batch, 128 * tiles),
                                                       pop, cw, reps)
            best = min(times, key=times.get)
            cache[key] = {"chunk": best, "ms": {str(k): v for k, v in times.items()}}
            timings[key] = times
        out.append(dataclasses.replace(sp, chunk=int(cache[key]["chunk"])))
    if cache_path and timings:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return out, timings
