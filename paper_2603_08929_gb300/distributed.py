"""One array sorted by several ranks, one GPU each: the one-exchange scheme.

Every rank holds a shard of the array.  The sorted result is the
concatenation, in rank order, of the ranks' outputs:

1. each rank counts its keys by the top ``bits`` bits of their sort-order
   code (``bsort_top_digit_counts``: digit d's keys precede digit d + 1's in
   the sorted output);
2. the counts are summed over the ranks (one all-reduce of 2^bits words);
3. every rank derives the same plan: contiguous digit ranges, one per rank,
   cut where the global prefix of the counts is closest to r * N / P;
4. each rank partitions its shard by digit (the library's first MSD levels,
   ``bsort_keys_partial_ws``; for 1- and 2-byte keys the whole counting
   sort), so the keys bound for each rank are contiguous, and one
   all-to-all-v moves them into the receiving rank's own memory;
5. each rank sorts what it received (``bsort_keys``).

The digits are the method's first ``bits`` MSB partitions: a split on the top
bits followed by sorting inside each part gives the global order, because
binary MSB splits refine lexicographically (the induction of Thm. 3).  A digit
is never split between ranks, so a rank holds at most N / P plus twice the
largest digit's count; duplicates of one value all land on one rank.

Only argument marshalling and the collectives run here; the counting,
partitioning and sorting are the library's kernels.  With NCCL the exchange
moves device memory directly; with a backend that cannot exchange device
tensors (gloo) the shard is staged through host memory.
"""
from __future__ import annotations

import numpy as np


def plan_digit_ranges(global_counts, world: int) -> np.ndarray:
    """Boundaries b[0..world] (digit indices, b[0] = 0, b[world] = D): rank r
    takes digits [b[r], b[r+1]).  Each inner boundary is the digit boundary
    whose global prefix is closest to r * N / world (ties to the lower one),
    kept non-decreasing."""
    c = np.asarray(global_counts, dtype=np.int64)
    d = c.size
    prefix = np.concatenate(([0], np.cumsum(c)))
    total = int(prefix[-1])
    b = np.zeros(world + 1, dtype=np.int64)
    b[world] = d
    scaled = prefix * world  # prefix[i] against total * r / world, exactly
    for r in range(1, world):
        goal = total * r
        i = int(np.searchsorted(scaled, goal, side="left"))  # first i with prefix[i] >= goal / world
        if i > 0 and (i > d or goal - scaled[i - 1] <= scaled[i] - goal):
            i -= 1
        b[r] = min(max(i, b[r - 1]), d)
    return b


def send_counts(local_counts, bounds) -> np.ndarray:
    """Keys this rank sends to each rank: its keys of that rank's digits."""
    lp = np.concatenate(([0], np.cumsum(np.asarray(local_counts, dtype=np.int64))))
    return lp[bounds[1:]] - lp[bounds[:-1]]


def exchange(keys, send, group=None):
    """All-to-all-v of a digit-partitioned shard: the first send[0] keys go to
    rank 0, the next send[1] to rank 1, ...; returns the keys received, in
    source-rank order, on the keys' device.  Moves bytes, so any key dtype
    works with any backend."""
    import torch
    import torch.distributed as dist
    device = keys.device
    world = dist.get_world_size(group)
    on_device = dist.get_backend(group) == "nccl"
    cdev = device if on_device else torch.device("cpu")
    send_t = torch.as_tensor(np.asarray(send, dtype=np.int64), device=cdev)
    recv_t = torch.empty(world, dtype=torch.int64, device=cdev)
    dist.all_to_all_single(recv_t, send_t, group=group)
    recv = recv_t.cpu().numpy()
    item = keys.element_size()
    xdev = device if on_device else torch.device("cpu")
    if keys.numel():
        src = keys.contiguous().view(torch.uint8).to(xdev)
    else:
        src = torch.empty(0, dtype=torch.uint8, device=xdev)  # an empty shard has no byte view
    out = torch.empty(int(recv.sum()) * item, dtype=torch.uint8, device=xdev)
    dist.all_to_all_single(out, src, output_split_sizes=[int(v) * item for v in recv],
                           input_split_sizes=[int(v) * item for v in send], group=group)
    if out.numel() == 0:
        return torch.empty(0, dtype=keys.dtype, device=device)
    return out.to(device).view(keys.dtype)


class LibraryOps:
    """The device steps of the scheme, each one library call."""

    def __init__(self):
        from . import Handle
        self.handle = Handle()

    def digit_counts(self, keys, descending, bits):
        from . import top_digit_counts
        return top_digit_counts(keys, bits, descending).cpu().numpy()

    def partition(self, keys, descending, bits):
        import torch
        from . import bsort_keys, bsort_keys_partial_ws, workspace_bytes
        if keys.numel() <= 1:
            return
        if keys.element_size() <= 2:
            bsort_keys(keys, descending=descending)  # counting sort: cheaper than any partial form
            return
        ws = torch.empty(workspace_bytes(keys.numel(), str(keys.dtype).replace("torch.", "")), dtype=torch.uint8,
                         device=keys.device)
        bsort_keys_partial_ws(self.handle, keys, ws, (bits + 7) // 8, descending=descending)

    def sort(self, keys, descending):
        from . import bsort_keys
        if keys.numel() > 1:
            bsort_keys(keys, descending=descending)


def sort_distributed(keys, descending: bool = False, group=None, bits: int = 12, ops=None):
    """Sorts the array whose shards the ranks of ``group`` hold (this rank's
    shard: ``keys``, a contiguous tensor, reordered in place by the
    partition).  Returns (this rank's part of the sorted array, a new tensor;
    its global start position).  Every rank must call it with the same
    ``descending`` and ``bits``."""
    import torch
    import torch.distributed as dist
    ops = ops or LibraryOps()
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    local = np.asarray(ops.digit_counts(keys, descending, bits), dtype=np.int64)
    cdev = keys.device if dist.get_backend(group) == "nccl" else torch.device("cpu")
    glob_t = torch.as_tensor(local, device=cdev).clone()
    dist.all_reduce(glob_t, group=group)
    glob = glob_t.cpu().numpy()
    bounds = plan_digit_ranges(glob, world)
    ops.partition(keys, descending, bits)
    mine = exchange(keys, send_counts(local, bounds), group)
    ops.sort(mine, descending)
    start = int(np.sum(glob[: bounds[rank]]))
    return mine, start


# ---- batched form: independent segments spread over the ranks ----------------

def plan_segments(sizes, world: int) -> np.ndarray:
    """Boundaries s[0..world] in segment indices: rank r sorts segments
    [s[r], s[r+1]), a contiguous run whose keys are as close to r * N / world
    as a segment boundary allows (the same closest-prefix rule as the digit
    plan), so each rank's part is one slice of the batch buffer and no rank
    holds more than N / world plus twice the largest segment."""
    return plan_digit_ranges(np.asarray(sizes, dtype=np.int64), world)


class LibrarySegmentOps:
    """The device step of the batched form: one segmented sort."""

    def sort_segments(self, keys, offsets, descending):
        """``offsets``: the run's segment boundaries relative to ``keys`` (a
        numpy array or a tensor on any device)."""
        import torch
        from . import bsort_keys_segmented
        off = torch.as_tensor(np.asarray(offsets.cpu() if hasattr(offsets, "cpu") else offsets, dtype=np.int64),
                              device=keys.device)
        if keys.numel() > 1 and off.numel() > 1:
            bsort_keys_segmented(keys, off, descending=descending)


def sort_segments_distributed(keys, offsets, descending: bool = False, group=None, ops=None):
    """Sorts every segment [offsets[i], offsets[i+1]) of a batch that each rank
    of ``group`` holds in full (``keys``, ``offsets``: the same on every rank;
    the segments are independent, so no data moves between ranks).  This rank
    sorts its planned run of segments in place in ``keys`` and returns the
    run (first segment, end segment).  Whichever rank sorts a segment, its
    bytes are those of the segment sorted alone."""
    import torch.distributed as dist
    ops = ops or LibrarySegmentOps()
    off = np.asarray(offsets.cpu() if hasattr(offsets, "cpu") else offsets, dtype=np.int64)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    s = plan_segments(np.diff(off), world)
    a, b = int(s[rank]), int(s[rank + 1])
    if b > a:
        lo, hi = int(off[a]), int(off[b])
        ops.sort_segments(keys[lo:hi], off[a:b + 1] - lo, descending)
    return a, b
