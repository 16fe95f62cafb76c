"""Autotuner of the MSD path: times candidate tunings (digit width, finish
threshold, merge threshold, chunk size in scatter tiles) for a dtype and size
on the current GPU and keeps the fastest per (dtype, size class) in a JSON
table; `autotune_segmented` does the same on a caller's segmented workload.
The tuning never changes a result, only the speed; `lookup` picks the entry of
the nearest size class.

Table format: {"<dtype>": {"<log2 n>": {"radix_bits": r, "unit_keys": u,
"merge_keys": m, "chunk_tiles": c, "ms": t}}} -- zero fields mean the library
default.
"""
from __future__ import annotations

import json
import math
import os

FIELDS = ("radix_bits", "unit_keys", "merge_keys", "chunk_tiles")

# digit width x finish threshold (0: default) x chunk of 2 or 1 scatter tiles;
# the merge threshold follows the finish threshold
CANDIDATES = [{"radix_bits": r, "unit_keys": u, "merge_keys": 0, "chunk_tiles": c}
              for r in (8, 11, 6, 4) for u in (0, 2048) for c in (0, 1)]


def _random_keys(dtype: str, n: int, device):
    """Uniform bit patterns over the whole key width, on the device (tuning
    input, not a test input)."""
    import torch
    tdt = getattr(torch, dtype)
    width = torch.empty(0, dtype=tdt).element_size()
    lo = torch.randint(0, 1 << 32, (n,), dtype=torch.int64, device=device)
    if width == 8:
        hi = torch.randint(0, 1 << 32, (n,), dtype=torch.int64, device=device)
        return ((hi << 32) | lo).view(tdt)
    small = {1: torch.uint8, 2: torch.int16, 4: torch.int32}[width]
    return lo.to(torch.int32).to(small).view(tdt) if width < 4 else (lo - (1 << 31)).to(torch.int32).view(tdt)


def time_tuning(dtype: str, n: int, tuning: dict, steps: int = 3, device=None) -> float:
    """Median milliseconds of one sort of n uniform keys with `tuning`."""
    import torch
    from . import Handle, bsort_keys_ws, workspace_bytes
    device = device or torch.device("cuda", torch.cuda.current_device())
    width = torch.empty(0, dtype=getattr(torch, dtype)).element_size()
    h = Handle()
    h.set_tuning(width, tuning)
    x = _random_keys(dtype, n, device)
    ws = torch.empty(workspace_bytes(n, dtype, tuning=tuning), dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream()
    times = []
    for i in range(steps + 1):
        y = x.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bsort_keys_ws(h, y, ws, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if i:
            times.append(e0.elapsed_time(e1))
    if h.get_error(stream) != 0:
        raise RuntimeError("device error word set while tuning")
    times.sort()
    return times[len(times) // 2]


def time_tuning_segmented(keys, offsets, tuning: dict, steps: int = 3) -> float:
    """Median milliseconds of one segmented sort of `keys` (a CUDA tensor,
    left unchanged) over `offsets` (int64 CUDA tensor, S + 1 entries) with
    `tuning`."""
    import torch
    from . import Handle, bsort_keys_segmented, segmented_workspace_bytes
    h = Handle()
    h.set_tuning(keys.element_size(), tuning)
    nseg = offsets.numel() - 1
    ws = torch.empty(segmented_workspace_bytes(keys.numel(), nseg, keys.dtype, tuning=tuning),
                     dtype=torch.uint8, device=keys.device)
    stream = torch.cuda.current_stream()
    times = []
    for i in range(steps + 1):
        y = keys.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bsort_keys_segmented(y, offsets, stream=stream, handle=h, workspace=ws)
        e1.record(stream)
        torch.cuda.synchronize()
        if i:
            times.append(e0.elapsed_time(e1))
    if h.get_error(stream) != 0:
        raise RuntimeError("device error word set while tuning")
    times.sort()
    return times[len(times) // 2]


def autotune_segmented(keys, offsets, candidates=None, steps: int = 3, log: list = None) -> dict:
    """The fastest candidate for this segmented workload, with its time in
    "ms"; `log` (a list) receives every (candidate, ms)."""
    best = None
    for c in candidates or CANDIDATES:
        ms = time_tuning_segmented(keys, offsets, c, steps)
        if log is not None:
            log.append((c, ms))
        if best is None or ms < best["ms"]:
            best = dict(c, ms=ms)
    return best


def autotune(dtype: str, n: int, candidates=None, steps: int = 3) -> dict:
    """The fastest candidate for (dtype, n), with its time in "ms"."""
    best = None
    for c in candidates or CANDIDATES:
        ms = time_tuning(dtype, n, c, steps)
        if best is None or ms < best["ms"]:
            best = dict(c, ms=ms)
    return best


def size_class(n: int) -> int:
    return max(0, int(round(math.log2(max(1, n)))))


def tune_table(dtypes, sizes, path: str = None, candidates=None, steps: int = 3) -> dict:
    table = load_table(path) if path and os.path.exists(path) else {}
    for dt in dtypes:
        for n in sizes:
            table.setdefault(dt, {})[str(size_class(n))] = autotune(dt, n, candidates, steps)
    if path:
        save_table(table, path)
    return table


def save_table(table: dict, path: str) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def load_table(path: str) -> dict:
    with open(path) as fh:
        return json.load(fh)


def lookup(table: dict, dtype: str, n: int) -> dict:
    """The tuning of the nearest size class of `dtype` (defaults if none)."""
    entries = table.get(dtype, {})
    if not entries:
        return {f: 0 for f in FIELDS}
    k = size_class(n)
    best = min(entries, key=lambda s: (abs(int(s) - k), int(s)))
    e = entries[best]
    return {f: int(e.get(f, 0)) for f in FIELDS}
