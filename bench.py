"""Benchmark of the GB300 bsort library (one JSON line on rank 0).

Default workload: one array of 2^28 int32 keys, uniform over the full bit
range (every bit pattern equally likely), sorted ascending -- the 32-bit
plain-sort configuration the throughput target is quoted on.  A step is one
complete sort of one such array, already resident in HBM; each timed step
sorts its own unsorted copy (the 1 GiB input is larger than the 129 MB L2).

  value         Gkeys/s over the timed steps, all ranks (max-over-ranks time)
  e2e           the same metric through bsort_keys_host(): host array in,
                host array out, copies inside the timed region
  roofline      the kernel with the largest share of the step: algorithmic
                bytes of its launches / their CUDA-event time, against the
                measured HBM copy bandwidth
  cpu_baseline  the CPU oracle on a bounded sample of the same workload

``--impl reference`` times the oracle itself (the only reference this paper
has: it publishes no code) on the same workload, a bounded sample per step.
With torchrun (N > 1) every rank sorts its own array (independent replicas,
weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "Gkeys/s & % HBM roofline per dtype at 2^28 keys; batched vs plain; serve p99 ms"
UNIT = "Gkeys/s"
DTYPE_TAG = {"uint8": "u8", "int8": "i8", "uint16": "u16", "int16": "i16", "float16": "f16",
             "uint32": "u32", "int32": "i32", "float32": "f32", "uint64": "u64", "int64": "i64",
             "float64": "f64", "bfloat16": "bf16"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="bsort", choices=["bsort", "reference"])
    ap.add_argument("--mode", default="plain", choices=["plain", "segmented", "serve", "pairs"],
                    help="plain: one 2^log2n array; segmented: the batched workload (see run_segmented)")
    ap.add_argument("--segments", type=int, default=10000, help="segments per dtype (segmented mode)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="segmented mode: library default tuning instead of the autotuner's choice")
    ap.add_argument("--seg-max-log2", type=int, default=20, help="segment sizes floor(2^(k*u)), u uniform")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="Poisson arrivals per second (serve mode)")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="length of the arrival trace (serve mode)")
    ap.add_argument("--serve-budget-gb", type=float, default=64.0, help="HBM admission budget (serve mode)")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--no-fifo", action="store_true", help="serve mode: skip the one-slot FIFO arm")
    ap.add_argument("--dtype", default="int32")
    ap.add_argument("--dist", default="uniform")
    ap.add_argument("--log2n", type=int, default=28)
    ap.add_argument("--desc", action="store_true")
    ap.add_argument("--inplace", action="store_true", help="in-place mode (no alternate buffer); reports aux bytes")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--value-dtype", default="int32", help="pairs mode: dtype of the values ('none': argsort only)")
    ap.add_argument("--radix-bits", type=int, default=0,
                    help="plain / pairs mode: MSD digit width 4..11 (0: default 8; pairs: of the packed-word sort)")
    ap.add_argument("--unit-keys", type=int, default=0,
                    help="plain / pairs mode: shared-memory finish threshold (0: default)")
    ap.add_argument("--chunk-tiles", type=int, default=0, help="plain / pairs mode: chunk of 1 or 2 scatter tiles (0: 2)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample-log2", type=int, default=23)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def whole_job(ms_per_step_local, keys_per_rank, world, device):
    """Max step time over the ranks and the whole-job throughput (Gkeys/s):
    every rank sorts its own keys_per_rank keys per step (independent
    replicas), so the job does world * keys_per_rank keys per max step time."""
    ms = float(ms_per_step_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, keys_per_rank * world / (ms * 1e-3) / 1e9


def measured_traffic(kind, dtype, keys_per_launch):
    """DRAM bytes per launch of kernel `kind` from the committed ncu record
    (`dtype`: the key dtype, or key_value dtypes for a key-value sort), or
    None when there is no record for it or the kernel sources changed since."""
    import glob
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_%s_traffic_%s.json" % (kind, dtype))
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh)
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(ROOT, "paper_2603_08929_gb300", "csrc", "*")))
    files.append(os.path.join(ROOT, "include", "bsort.h"))
    for f in files:
        with open(f, "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != rec.get("sources_sha256"):
        return None
    return rec["dram_bytes_per_key"] * keys_per_launch


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def host_cpu() -> dict:
    """The host's CPU model and logical core count (for the baseline's record)."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:  # Arm hosts: /proc/cpuinfo has no model name, lscpu does
        try:
            import subprocess
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            model = next((ln.split(":", 1)[1].strip() for ln in out.splitlines()
                          if ln.lower().startswith("model name")), None)
        except (OSError, subprocess.SubprocessError):
            model = None
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"cpu_model": model, "nproc": os.cpu_count()}


def oracle_sort(O, x, descending, dtype):
    """The oracle's sort of x (bfloat16 arrives as uint16 bit patterns,
    128-bit keys as uint64 (n, 2) arrays)."""
    if dtype in ("uint128", "int128"):
        return O.bsort128(x, signed=dtype == "int128", descending=descending)
    if dtype == "bfloat16":
        w = x.astype(np.uint64)
        O.bsort_words(w, O.BF16, descending)
        return w.astype(np.uint16)
    return O.bsort(x, descending=descending)


def cpu_baseline(x, descending, sample_log2, dtype=None):
    """The oracle (literal partition, single thread) on the first 2^k keys."""
    import oracle as O
    O.build()
    m = min(x.shape[0], 1 << sample_log2)
    sample = np.ascontiguousarray(x[:m])
    t0 = time.perf_counter()
    oracle_sort(O, sample, descending, dtype)
    dt = time.perf_counter() - t0
    return dict({"value": m / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                 "sample": "first 2^%d keys of the same input (%d keys), literal partition, one thread, "
                           "%.1f s" % (sample_log2, m, dt)}, **host_cpu())


def run_reference(args, rank, world):
    """Reference arm: the oracle itself, timed on the host cores."""
    if rank != 0:
        return
    import oracle as O
    O.build()
    n = 1 << args.log2n
    m = min(n, 1 << args.cpu_sample_log2)
    x = W.make(args.dist, args.dtype, m, seed=args.seed)
    times = []
    for i in range(args.warmup + args.steps):
        y = x.copy()
        t0 = time.perf_counter()
        oracle_sort(O, y, args.desc, args.dtype)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = m * len(times) / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / len(times) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE_TAG.get(args.dtype, args.dtype), "data": "synthetic",
        "config": {"workload": "plain sort, %s %s, 2^%d keys, %s (each step: the oracle on a "
                                "2^%d-key sample)" % (args.dtype, args.dist, args.log2n,
                                                      "descending" if args.desc else "ascending",
                                                      args.cpu_sample_log2),
                   "n": n, "sample_keys": m},
        "cpu_baseline": dict({"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                              "sample": "2^%d keys per step, literal partition, one thread"
                                        % args.cpu_sample_log2}, **host_cpu()),
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_segmented(args, rank, world):
    """Batched workload: args.segments int32 segments and as many float32
    segments, sizes floor(2^(k*u)) with u uniform (log-uniform in [1, 2^k]),
    uniform bits, ascending.  Timed: the two segmented sorts, each one
    captured CUDA graph (value), against one plain bsort_keys_ws call per
    segment on the same stream (plain_per_segment)."""
    import torch
    import paper_2603_08929_gb300 as bs
    from paper_2603_08929_gb300 import build as B
    from paper_2603_08929_gb300 import tune
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    B.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    h = bs.Handle()
    stream = torch.cuda.current_stream()
    arms = []
    tuned = {}
    for k, dt in enumerate(("int32", "float32")):
        sizes = W.segment_sizes(args.seed + 17 * k + rank, args.segments, args.seg_max_log2)
        n = int(sizes.sum())
        x = W.make("uniform", dt, n, seed=args.seed + k + rank)
        off = torch.from_numpy(np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)).to(dev)
        pristine = torch.from_numpy(x).to(dev)
        keys = pristine.clone()
        # autotuned digit width, finish threshold and chunk for this workload (untimed)
        tuning = None
        if not args.no_autotune:
            log = []
            best = tune.autotune_segmented(pristine, off, steps=2, log=log)
            tuning = {f: best[f] for f in tune.FIELDS}
            tuned[dt] = {"chosen": tuning, "ms": best["ms"],
                         "candidates_ms": {"r%d T=%s chunk=%d" % (c["radix_bits"] or 8, c["unit_keys"] or "def",
                                                                   c["chunk_tiles"] or 2): round(ms, 3)
                                           for c, ms in log}}
        hk = bs.Handle()
        hk.set_tuning(4, tuning)
        ws = torch.empty(bs.segmented_workspace_bytes(n, len(sizes), dt, tuning=tuning), dtype=torch.uint8,
                         device=dev)
        g = bs.Graph(hk, keys, ws, offsets=off)
        arms.append((dt, sizes, n, pristine, keys, ws, g, off, hk))
    total = sum(a[2] for a in arms)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            for a in arms:
                a[4].copy_(a[3])
            fn()
        torch.cuda.synchronize()
        ms = 0.0
        for _ in range(steps):
            for a in arms:
                a[4].copy_(a[3])
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        return ms / steps

    def graphs():
        for a in arms:
            a[6].launch(stream)

    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
    ms_graph = timed(graphs, args.steps, args.warmup)
    clock_info = clocks.stop() if clocks else None
    for a in arms:
        if a[6].error(stream) != 0:
            raise RuntimeError("device error word set in the segmented sort")
    # correctness of the last run: every segment non-decreasing (int32 arm)
    dt, sizes, n, pristine, keys, ws, g, off, _ = arms[0]
    seg_id = torch.repeat_interleave(torch.arange(len(sizes), device=dev), torch.from_numpy(sizes).to(dev))
    same = seg_id[1:] == seg_id[:-1]
    ok = bool(torch.all((keys[1:] >= keys[:-1]) | ~same).item())

    # one plain launch per segment, same keys, one workspace of the largest segment's size
    big = max(int(a[1].max()) for a in arms)
    wsp = torch.empty(max(bs.workspace_bytes(big, "int32"), bs.workspace_bytes(big, "float32")), dtype=torch.uint8,
                      device=dev)
    views = []
    for a in arms:
        o = a[7].cpu().numpy()
        views += [a[4][o[i]:o[i + 1]] for i in range(len(a[1])) if o[i + 1] - o[i] > 1]

    def per_segment():
        for v in views:
            bs.bsort_keys_ws(h, v, wsp, stream=stream)

    ms_plain = timed(per_segment, max(1, min(args.steps, 2)), 1)
    value = total / (ms_graph * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i32+f32", "data": "synthetic",
        "config": {"workload": "batched segmented sort: %d int32 + %d float32 segments, sizes log-uniform in "
                               "[1, 2^%d], uniform bits, ascending; one captured graph per dtype"
                               % (args.segments, args.segments, args.seg_max_log2),
                   "keys": total, "segments": 2 * args.segments,
                   "tuning": tuned if tuned else "library defaults (--no-autotune)",
                   "l2": "inputs %.1f GB > L2; restored from a pristine copy before each step (untimed)"
                         % (sum(a[2] * 4 for a in arms) / 1e9)},
        "plain_per_segment": {"value": total / (ms_plain * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms_plain,
                              "calls": len(views)},
        "speedup_vs_plain_per_segment": ms_plain / ms_graph,
        "sorted_check": ok,
    }
    if clock_info:
        line["clocks"] = clock_info
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_serve(args, rank, world):
    """Served workload: an open-loop Poisson trace (args.serve_rate requests/s
    for args.serve_seconds; sizes log-uniform in [2^10, 2^24]; int16 25%,
    int32 35%, float32 30%, float64 10%; uniform or normal(0, 1) values) sent
    to the continuous-batching server under an HBM budget.  Each request's
    payload is copied from a device-resident pool into a fresh buffer just
    before submission (the request's arrival).  Latency is the server's
    submit-to-completion time.  The same trace then goes through a one-slot,
    one-request-at-a-time server (a plain FIFO queue) for comparison."""
    import torch
    import paper_2603_08929_gb300 as bs
    from paper_2603_08929_gb300 import build as B
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    B.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    tr = W.serve_trace(args.seed + rank, args.serve_rate, args.serve_seconds)
    count = len(tr["t"])
    pool_n = 1 << 24
    pool = {}
    for d, name in enumerate(W.SERVE_DTYPES):
        for k, dist in enumerate(("uniform", "normal01")):
            pool[d, k] = torch.from_numpy(W.make(dist, name, pool_n, seed=args.seed + 7)).to(dev)
    offs = (W.uniform01(args.seed + rank, 0xF11, count) * (pool_n - tr["n"] + 1)).astype(np.int64) & ~7
    producer = torch.cuda.Stream()
    torch.cuda.synchronize()

    smode = bs.MODE_INPLACE if args.inplace else bs.MODE_PINGPONG

    def serve(num_slots, max_batch, batch_keys, seconds):
        srv = bs.Server(num_slots=num_slots, hbm_budget_bytes=int(args.serve_budget_gb * (1 << 30)),
                        max_request_keys=pool_n, max_batch=max_batch, batch_keys=batch_keys, mode=smode)
        last = int(np.searchsorted(tr["t"], seconds))
        lat, wait, done_keys = [], [], 0
        first_submit, last_done = None, 0
        t0 = time.perf_counter()
        i = 0
        while i < last or len(lat) < last:
            now = time.perf_counter() - t0
            if i < last and now >= tr["t"][i]:
                n = int(tr["n"][i])
                src = pool[int(tr["dtype"][i]), int(tr["dist"][i])]
                with torch.cuda.stream(producer):
                    buf = torch.empty(n, dtype=src.dtype, device=dev)
                    buf.copy_(src[int(offs[i]):int(offs[i]) + n])
                producer.synchronize()
                srv.submit(buf, tag=i)
                i += 1
                continue
            comps = srv.poll()
            for c in comps:
                if c["status"] != 0:
                    raise RuntimeError("request %d failed with status %d" % (c["tag"], c["status"]))
                lat.append((c["t_done_ns"] - c["t_submit_ns"]) * 1e-6)
                wait.append((c["t_admit_ns"] - c["t_submit_ns"]) * 1e-6)
                done_keys += int(tr["n"][c["tag"]])
                first_submit = c["t_submit_ns"] if first_submit is None else min(first_submit, c["t_submit_ns"])
                last_done = max(last_done, c["t_done_ns"])
            if not comps:
                nxt = tr["t"][i] - (time.perf_counter() - t0) if i < last else 1e-4
                time.sleep(min(max(nxt, 0.0), 1e-4))
        st = srv.stats()
        srv.close()
        span = (last_done - first_submit) * 1e-9
        lat = np.array(lat)
        return {"requests": last, "keys": done_keys, "seconds": span, "value": done_keys / span / 1e9,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
                "queue_p99_ms": float(np.percentile(np.array(wait), 99)),
                "batches": st["batches"], "max_concurrent_slots": st["max_concurrent_slots"],
                "peak_in_flight_gb": st["peak_in_flight_bytes"] / 1e9, "launches": st["launches"],
                "slot_workspace_gb": st["slot_workspace_bytes"] / 1e9}

    serve(args.serve_slots, 16, 1 << 20, min(2.0, args.serve_seconds))  # warm-up
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    main_arm = serve(args.serve_slots, 16, 1 << 20, args.serve_seconds)
    clock_info = clocks.stop()
    fifo = None if args.no_fifo else serve(1, 1, 1, args.serve_seconds)
    line = {
        "metric": METRIC, "value": main_arm["value"], "unit": UNIT, "n_gpus": world, "steps": main_arm["requests"],
        "warmup": 1, "ms_per_step": main_arm["mean_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i16+i32+f32+f64", "data": "synthetic",
        "config": {"workload": "served sorting: Poisson %.0f requests/s for %.0f s, sizes log-uniform in "
                               "[2^10, 2^24], int16 25%% / int32 35%% / float32 30%% / float64 10%%, uniform "
                               "or normal(0, 1) values, %.0f GB HBM budget, %d slots, %s mode"
                               % (args.serve_rate, args.serve_seconds, args.serve_budget_gb, args.serve_slots,
                                  "in-place" if args.inplace else "ping-pong"),
                   "l2": "each request sorts a fresh copy of a window of a 2^24-key device pool"},
        "serve": main_arm,
        "fifo_one_slot": fifo,
        "gpu_launches": main_arm["launches"],
        "note": "value = keys completed / (last completion - first submission): under an open-loop trace "
                "it tracks the offered load; p50/p99 are submit-to-completion latencies",
    }
    if clock_info:
        line["clocks"] = clock_info
    print(json.dumps(line), flush=True)


def run_pairs_mode(args, rank, world):
    """Stable key-value sort of 2^log2n keys of --dtype (--dist) with
    --value-dtype values (or, with 'none', the int64 positions: an argsort).
    Every step sorts its own copy of keys and values (made before timing).
    The value: K bsort_pairs_ws calls between two CUDA events; then the same K
    calls on restored copies with the library's events around every launch
    group, for the per-kernel times and the roofline."""
    import torch
    import paper_2603_08929_gb300 as bs
    from paper_2603_08929_gb300 import build as B
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    B.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    n = 1 << args.log2n
    x = torch.from_numpy(W.make(args.dist, args.dtype, n, seed=args.seed + rank)).to(dev)
    argsort = args.value_dtype == "none"
    v0 = None if argsort else torch.from_numpy(W.make("uniform", args.value_dtype, n, seed=args.seed + 1)).to(dev)
    total_steps = args.warmup + args.steps
    keys = [x.clone() for _ in range(total_steps)]
    vals = [None if argsort else v0.clone() for _ in range(total_steps)]
    idx = torch.empty(n, dtype=torch.int64, device=dev) if argsort else None
    tuning8 = {"radix_bits": args.radix_bits, "unit_keys": args.unit_keys, "chunk_tiles": args.chunk_tiles}
    tuning8 = tuning8 if any(tuning8.values()) else None
    ws = torch.empty(bs.pairs_workspace_bytes(n, args.dtype, tuning8=tuning8), dtype=torch.uint8, device=dev)
    h = bs.Handle()
    if tuning8:
        h.set_tuning(8, tuning8)
    stream = torch.cuda.current_stream()
    for i in range(args.warmup):
        bs.bsort_pairs_ws(h, keys[i], ws, values=vals[i], indices=idx, descending=args.desc, stream=stream)
    torch.cuda.synchronize()
    if h.get_error(stream) != 0:
        raise RuntimeError("device error word set during warm-up")
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()

    def timed_region():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.warmup, total_steps):
            bs.bsort_pairs_ws(h, keys[i], ws, values=vals[i], indices=idx, descending=args.desc, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    elapsed_ms = timed_region()
    out_k = keys[-1].clone()
    for i in range(args.warmup, total_steps):
        keys[i].copy_(x)
        if not argsort:
            vals[i].copy_(v0)
    h.set_profiling(True)
    elapsed_prof_ms = timed_region()
    prof = h.profile()
    h.set_profiling(False)
    launches = prof["launches"]  # kernels of the K timed calls
    if world > 1:
        torch.distributed.barrier()
    clock_info = clocks.stop() if clocks else None
    if h.get_error(stream) != 0:
        raise RuntimeError("device error word set in the key-value sort")
    per_kind = {}
    for r in prof["records"]:
        k = per_kind.setdefault(r["kind"], {"ms": 0.0, "bytes": 0, "launches": 0})
        k["ms"] += r["ms"]
        k["bytes"] += r["counted_bytes"]
        k["launches"] += 1
    ms_per_step, value = whole_job(elapsed_ms / args.steps, n, world, dev)
    signed_ok = args.dtype in ("int8", "int16", "int32", "int64", "uint8")  # torch compares these on the device
    ok = (bool(torch.all(out_k[1:] <= out_k[:-1]).item()) if args.desc else
          bool(torch.all(out_k[1:] >= out_k[:-1]).item())) if signed_ok else None
    esize = x.element_size()
    vsize = 8 if argsort else v0.element_size()
    peak, peak_src = load_peaks()
    floor_bytes = n * (2 * esize + (vsize if argsort else 2 * vsize))  # read keys (+values), write keys + values/positions
    dom_kind = max(per_kind.items(), key=lambda kv: kv[1]["ms"])[0]
    dk = per_kind[dom_kind]
    achieved = dk["bytes"] / (dk["ms"] * 1e-3) / 1e9 if dk["ms"] > 0 else 0.0
    sort_ms = sum(k["ms"] for k in per_kind.values()) / args.steps
    total_bytes = sum(k["bytes"] for k in per_kind.values()) / args.steps
    sort_gbs = total_bytes / (ms_per_step * 1e-3) / 1e9
    tag = "%s_%s" % (args.dtype, args.value_dtype)
    carried = 4 if argsort else vsize  # bytes travelling with each key through the levels
    line = {
        "metric": METRIC, "value": value, "unit": "Gpairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_TAG.get(args.dtype, args.dtype), "data": "synthetic",
        "config": {"workload": "stable key-value sort, %s %s keys, 2^%d, %s, %s" % (
            args.dtype, args.dist, args.log2n, "argsort (int64 positions)" if argsort else
            "%s values" % args.value_dtype, "descending" if args.desc else "ascending"),
            "n": n, "l2": "inputs > L2 at this size; each step sorts its own copy",
            "timing": "value: K calls between two CUDA events, nothing between their launches; kernel times "
                      "and the roofline: the same K calls on restored copies with the library's events around "
                      "every launch group (ms_per_step_instrumented)",
            "tuning_of_the_word_sort": tuning8 or "library defaults"},
        "gpu_launches": launches,
        "ms_per_step_instrumented": elapsed_prof_ms / args.steps,
        "roofline": {"bound": "hbm", "kernel": dom_kind, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_src,
                     "traffic": measured_traffic(
                         dom_kind, tag, dk["bytes"] / (2 * (esize + carried)) / max(dk["launches"], 1))
                     if dom_kind in ("finish", "scatter") and not tuning8 else None},
        "sort_roofline": {"counted_bytes_per_step": total_bytes, "achieved": sort_gbs, "frac": sort_gbs / peak,
                          "peak": peak},
        "kernels": {k: {"ms_per_step": v["ms"] / args.steps, "share": v["ms"] / (sort_ms * args.steps),
                        "gbs": v["bytes"] / (v["ms"] * 1e-3) / 1e9 if v["ms"] > 0 else 0.0,
                        "launches_per_step": v["launches"] / args.steps}
                    for k, v in sorted(per_kind.items())},
        "min_bytes_frac": floor_bytes / (ms_per_step * 1e-3) / 1e9 / peak,
        "min_bytes_note": "bytes any key-value sort must move (read keys%s, write keys and %s) / time / %s HBM "
                          "copy bandwidth" % ("" if argsort else " and values", "positions" if argsort else "values",
                                              peak_src),
        "sorted_check": ok,
    }
    if clock_info:
        line["clocks"] = clock_info
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.mode == "segmented":
        run_segmented(args, rank, world)
        return
    if args.mode == "serve":
        run_serve(args, rank, world)
        return
    if args.mode == "pairs":
        run_pairs_mode(args, rank, world)
        return
    import torch
    import paper_2603_08929_gb300 as bs
    from paper_2603_08929_gb300 import build as B

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    B.build()
    dev = torch.device("cuda", torch.cuda.current_device())

    n = 1 << args.log2n
    x = W.make(args.dist, args.dtype, n, seed=args.seed + rank)
    wide = args.dtype in W.WIDE_DTYPES  # 16-byte keys: uint64 (n, 2) arrays, passed with a dtype override
    kdt = args.dtype if wide else None
    esize = 16 if wide else x.dtype.itemsize
    total_steps = args.warmup + args.steps
    base = torch.from_numpy(x.view(np.int64) if wide else x).to(dev)
    if args.dtype == "bfloat16":  # the generator gives bfloat16 as uint16 bit patterns
        base = base.view(torch.bfloat16)
    bufs = [base.clone() for _ in range(total_steps)]
    pristine_dev = base
    mode = bs.MODE_INPLACE if args.inplace else bs.MODE_PINGPONG
    tuning = {"radix_bits": args.radix_bits, "unit_keys": args.unit_keys, "chunk_tiles": args.chunk_tiles}
    tuning = tuning if any(tuning.values()) and esize >= 4 else None
    ws = torch.empty(bs.workspace_bytes(n, args.dtype, mode=mode, tuning=tuning), dtype=torch.uint8, device=dev)
    h = bs.Handle()
    if tuning:
        h.set_tuning(esize, tuning)
    stream = torch.cuda.current_stream()

    for i in range(args.warmup):
        bs.bsort_keys_ws(h, bufs[i], ws, descending=args.desc, stream=stream, mode=mode, dtype=kdt)
    torch.cuda.synchronize()
    if h.get_error(stream) != 0:
        raise RuntimeError("device error word set during warm-up")

    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()

    def timed_region():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.warmup, total_steps):
            bs.bsort_keys_ws(h, bufs[i], ws, descending=args.desc, stream=stream, mode=mode, dtype=kdt)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # (1) the value: K sorts with no event between their launches
    elapsed_ms = timed_region()
    # (2) the same K sorts again, on restored copies, with the library's CUDA
    # events around every launch group on the same stream (per-kernel times
    # for the roofline; the events themselves lengthen the step a little)
    for i in range(args.warmup, total_steps):
        bufs[i].copy_(pristine_dev)
    del pristine_dev
    h.set_profiling(True)
    elapsed_prof_ms = timed_region()
    prof = h.profile()
    h.set_profiling(False)
    launches = prof["launches"]
    per_kind = {}
    for r in prof["records"]:
        k = per_kind.setdefault(r["kind"], {"ms": 0.0, "bytes": 0, "launches": 0})
        k["ms"] += r["ms"]
        k["bytes"] += r["counted_bytes"]
        k["launches"] += 1
    if world > 1:
        torch.distributed.barrier()
    clock_info = clocks.stop() if clocks else None
    if h.get_error(stream) != 0:
        raise RuntimeError("device error word set during the timed steps")
    aux_bytes = h.last_aux_bytes()

    # step time: sum of each step's sort (events around every launch group)
    sort_ms = sum(k["ms"] for k in per_kind.values()) / args.steps
    ms_per_step, value = whole_job(elapsed_ms / args.steps, n, world, dev)

    # correctness of the last timed step (cheap properties at full size)
    out = bufs[-1]
    ok_sorted = bool(torch.all(out[:-1] <= out[1:]).item()) if (
        args.dist == "uniform" and args.dtype in ("int8", "int16", "int32", "int64", "uint8")
        and not args.desc) else None

    peak, peak_src = load_peaks()
    dom_kind = max(per_kind.items(), key=lambda kv: kv[1]["ms"])[0]
    dk = per_kind[dom_kind]
    achieved = dk["bytes"] / (dk["ms"] * 1e-3) / 1e9 if dk["ms"] > 0 else 0.0
    total_bytes = sum(k["bytes"] for k in per_kind.values()) / args.steps
    sort_gbs = total_bytes / (ms_per_step * 1e-3) / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_TAG.get(args.dtype, args.dtype),
        "data": "synthetic",
        "config": {"workload": "plain sort, %s %s, 2^%d keys, %s%s" % (
            args.dtype, args.dist, args.log2n, "descending" if args.desc else "ascending",
            ", in-place mode" if args.inplace else ""),
            "n": n, "per_gpu_keys": n, "l2": "input 2^%d x %d B > L2; each step sorts its own copy"
                                            % (args.log2n, esize),
            "parallelism": "replicas%d" % world,
            "tuning": tuning or "library defaults",
            "timing": "value: K sorts between two CUDA events, nothing between their launches; kernel "
                      "times and the roofline: the same K sorts on restored copies with the library's "
                      "events around every launch group (ms_per_step_instrumented)"},
        "gpu_launches": launches,
        "ms_per_step_instrumented": elapsed_prof_ms / args.steps,
        "roofline": {"bound": "hbm", "kernel": dom_kind, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                     "traffic": measured_traffic(
                         dom_kind, args.dtype,
                         dk["bytes"] / (2 * esize) / max(dk["launches"], 1)) if dom_kind in (
                             "finish", "scatter") and not tuning else None},
        "sort_roofline": {"counted_bytes_per_step": total_bytes, "achieved": sort_gbs,
                          "frac": sort_gbs / peak, "peak": peak,
                          "fixed_2nb_frac": 2 * n * esize / (ms_per_step * 1e-3) / 1e9 / peak},
        "kernels": {k: {"ms_per_step": v["ms"] / args.steps, "share": v["ms"] / (sort_ms * args.steps),
                        "gbs": v["bytes"] / (v["ms"] * 1e-3) / 1e9 if v["ms"] > 0 else 0.0,
                        "launches_per_step": v["launches"] / args.steps}
                    for k, v in sorted(per_kind.items())},
        "finish_units_per_step": {k: v / args.steps for k, v in prof["finish_units"].items()},
        "mode": "inplace" if args.inplace else "pingpong",
        "aux": {"bytes": aux_bytes, "frac_of_keys": aux_bytes / (n * esize),
                "workspace_reserved": ws.numel(),
                "paper_bound": "O(w): the sequential in-place partition keeps only its recursion (Sec. III)"},
        "sorted_check": ok_sorted,
    }
    if clock_info:
        line["clocks"] = clock_info

    if not args.no_e2e:
        host = torch.from_numpy(x.view(np.int64).copy() if wide else x.copy()).pin_memory()
        if args.dtype == "bfloat16":
            host = host.view(torch.bfloat16)
        pristine = host.clone()
        for _ in range(2):
            host.copy_(pristine)
            bs.bsort_keys_host(host, descending=args.desc, dtype=kdt)
        ts = []
        for _ in range(max(3, min(args.steps, 5))):
            host.copy_(pristine)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bs.bsort_keys_host(host, descending=args.desc, dtype=kdt)
            ts.append(time.perf_counter() - t0)
        e2e_s = statistics.median(ts)
        line["e2e"] = {"value": n / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": n * esize,
                       "d2h_bytes_per_step": n * esize, "ms_per_step": e2e_s * 1e3,
                       "api": "bsort_keys_host (pinned host array in and out; library default tuning)"}
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(x, args.desc, args.cpu_sample_log2, args.dtype)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
