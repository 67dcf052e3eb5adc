#!/usr/bin/env python3
"""Benchmark of the batched RAMBO query path (arXiv 1910.02611) on one or more
GB300s.

A step (default workload, "uneven") is one batch of 10^6 DNA query sequences
with lognormal lengths (median 300 bases, sigma 1, clipped to [31, 10^4];
substrings of 10^4 synthetic genomes with 0-2% base substitutions) answered
against a resident index of 10^4 genomes x ~2*10^5 31-mers (B=128, R=8,
m=2^26, eta=2, 8 GiB): 2-bit packing, k-mer hashing, row probes, AND across
tables' cells and across the sequence's k-mers, set-level intersection and
compaction of the set-ID lists, all in the library's kernels, as one replay of
a CUDA graph captured once (the persistent query kernel with its device work
queue inside), with the kernel tiling picked by the library's autotuner on the
first batch before the timed region.  --config genome / document / tiny /
serving select the other workloads, --api call the direct C-ABI call.  The
index is built once per run with the construction kernel (timed and reported
beside the query numbers).

  value   k-mers (query keys submitted) per second, inputs already in device
          memory, summed over ranks, time = max over ranks of the CUDA-event
          time of the K timed steps (L2 flushed before every step);
  e2e     the same metric through the same C-ABI call with host (pinned)
          inputs and outputs: host-to-device copy of the batch, the kernels,
          device-to-host copy of the results, all inside the timed region.

--impl reference times the CPU oracle (plain C, Algorithms 1 and 2 of the
paper on B*R separate Bloom filters) on a bounded sample of the same
workload on the host cores.  Multi-GPU: every rank holds a replica of the
index and answers its own batches (no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "k-mer queries/s and achieved HBM GB/s vs roofline; p50/p99 query latency"
UNIT = "k-mers/s"
SECTOR = 32
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="uneven", choices=["genome", "uneven", "document", "tiny", "serving"])
    ap.add_argument("--rates", default="1000,10000,100000,1000000",
                    help="serving: Poisson arrival rates (requests/s) to sweep")
    ap.add_argument("--requests-per-rate", type=int, default=20000)
    ap.add_argument("--scale", type=float, default=1.0, help="workload scale (1.0 = the full configuration)")
    ap.add_argument("--batches", type=int, default=6, help="distinct query batches rotated over the steps")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--m-log2", type=int, default=None, help="override the Bloom filter size m = 2^L")
    ap.add_argument("--queries", type=int, default=None,
                    help="queries per step instead of the workload's own count (profiling cases)")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the query steps only (no e2e, random-row or CPU legs): the profiling case")
    ap.add_argument("--per-query-baseline", type=int, default=2000,
                    help="queries timed through the one-query-per-launch kernel (0 = skip)")
    ap.add_argument("--autotune", action=argparse.BooleanOptionalAction, default=True,
                    help="pick the kernel configuration with the library's autotuner on batch 0 first")
    ap.add_argument("--query-config", default=None,
                    help="set the query kernel configuration, e.g. lanes_per_key=1,words_per_lane=4,warps_per_block=8 "
                         "(profiling runs: the autotuner's timings under a profiler are not the run's)")
    ap.add_argument("--api", choices=["call", "plan"], default="plan",
                    help="timed step through rambo_query_*_into (call) or a replayed CUDA-graph plan (plan)")
    ap.add_argument("--plan-timing", action=argparse.BooleanOptionalAction, default=True,
                    help="replay the plan graph with its event-record nodes around the query kernel (the kernel's "
                         "time live in the timed region); without them a replay finishes a few microseconds "
                         "sooner and the kernel is timed by direct calls after the timed region")
    ap.add_argument("--json-out", default=None)
    return ap.parse_args()


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_workload(config: str, scale: float, m_log2=None, queries=None):
    kw = {} if m_log2 is None else {"m": 1 << m_log2}
    if queries:
        # the generators scale their query count with the workload; ask for
        # the count that leaves `queries` after scaling
        kw["n_queries"] = int(queries) if scale == 1.0 else max(1, int(round(queries / scale)))
    return synth.make(config, scale, **kw)


def extra_batches(w, n_batches: int, rank: int):
    """Distinct query batches of the workload's shape (the first is the
    workload's own when rank == 0)."""
    out = [w.queries] if rank == 0 else []
    b = 0
    while len(out) < n_batches:
        rng = np.random.default_rng(10_000 + 97 * rank + b)
        b += 1
        n = len(w.queries)
        if w.name == "genome":
            lengths = rng.integers(100, 1001, n)
            out.append(synth.substring_queries(rng, w.sets, lengths))
        elif w.name == "uneven":
            lengths = np.clip(np.round(rng.lognormal(np.log(300), 1.0, n)), 31, 10_000).astype(np.int64)
            out.append(synth.substring_queries(rng, w.sets, lengths))
        else:
            idx = rng.permutation(n)
            out.append(w.queries.subset(idx))
    return out


def reduce_over_ranks(dist, maxes, sums, device):
    """Whole-job figures: the max over ranks of the times (the job ends when the
    slowest rank ends) and the sum over ranks of the work.  dist is
    torch.distributed or None for one process; no data-path collective."""
    if dist is None or not dist.is_initialized():
        return [float(x) for x in maxes], [float(x) for x in sums]
    import torch

    t = torch.tensor([float(x) for x in maxes], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(x) for x in sums], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.tolist()], [float(x) for x in c.tolist()]


def keys_in(q, k: int) -> int:
    if q.kind == "keys":
        return int(q.offsets[-1] - q.offsets[0])
    return int(q.offsets[-1] - q.offsets[0]) - len(q) * (k - 1)


# ---------------------------------------------------------------------------
# measurement helpers
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max((num(r[3]) or 0) for r in rows)}


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def _code_only(text: str) -> str:
    """C++ source with comments and blank lines removed (comment edits leave
    the compiled kernel, and so its profile, unchanged)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(l.rstrip() for l in text.splitlines() if l.strip())


def kernel_source_hash() -> str:
    """Hash of the query kernel's device code, comments removed: k_query.cuh,
    its instantiation header, and the device helpers of rambo_impl.cuh (up to
    the launcher declarations)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1910_02611_gb300", "csrc")
    for name in ("k_query.cuh", "k_query_inst.cuh"):
        with open(os.path.join(csrc, name)) as f:
            h.update(_code_only(f.read()).encode())
    with open(os.path.join(csrc, "rambo_impl.cuh")) as f:
        text = f.read()
    h.update(_code_only(text.split("// launchers (defined in the .cu files)")[0]).encode())
    return h.hexdigest()[:16]


def ncu_traffic(config: str):
    """Per-launch DRAM bytes of the query kernel from the committed ncu summary,
    valid only while the kernel source is the one that was profiled."""
    p = os.path.join(ROOT, "profiles", f"query_kernel_{config}_traffic.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    with open(p) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------

def oracle_index(w, nthreads: int):
    from oracle.oracle import Oracle

    o = Oracle(w.K, w.B, w.R, w.m, w.eta, w.seed)
    t0 = time.perf_counter()
    if w.sets.kind == "keys":
        o.insert_keys_batch(w.sets.ids, w.sets.data, w.sets.offsets, nthreads=nthreads)
    else:
        o.insert_seq_batch(w.sets.ids, w.sets.data, w.sets.offsets, w.k, nthreads=nthreads)
    return o, time.perf_counter() - t0


def oracle_rate(o, q, k: int, nthreads: int, target_s: float):
    """keys/s of the oracle on a prefix of batch q sized to ~target_s seconds."""
    n = min(len(q), 64)
    while True:
        sub = q.subset(np.arange(n))
        t0 = time.perf_counter()
        o.query_batch_counts(sub.kind, sub.data, sub.offsets, k=k, nthreads=nthreads)
        dt = time.perf_counter() - t0
        if dt >= target_s or n >= len(q):
            return keys_in(sub, k) / dt, n, dt
        n = min(len(q), max(n * 2, int(n * target_s / max(dt, 1e-3) * 1.05)))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    nthreads = os.cpu_count() or 1
    w = make_workload("document" if args.config == "serving" else args.config, args.scale, args.m_log2, args.queries)
    o, build_s = oracle_index(w, nthreads)
    q = w.queries
    # size one step to a bounded sample so the whole run stays within minutes
    rate, n, dt = oracle_rate(o, q, w.k, nthreads, target_s=min(5.0, args.cpu_seconds))
    per_step_n = max(1, int(n * 2.0 / max(dt, 1e-3)))  # about 2 s of oracle work per step
    per_step_n = min(per_step_n, len(q))
    times, keys = [], 0
    for s in range(args.warmup + args.steps):
        idx = (np.arange(per_step_n) + s * per_step_n) % len(q)
        sub = q.subset(idx)
        t0 = time.perf_counter()
        o.query_batch_counts(sub.kind, sub.data, sub.offsets, k=w.k, nthreads=nthreads)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            keys += keys_in(sub, w.k)
    total = sum(times)
    value = keys / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"{w.name}: K={w.K} B={w.B} R={w.R} m=2^{int(np.log2(w.m))} eta={w.eta}, "
                               f"{len(q)} query sequences (scale {args.scale})",
                   "step": f"{per_step_n} queries of the workload per step (bounded sample)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                         "sample": f"{per_step_n} queries per step x {args.steps} steps; oracle index built in "
                                   f"{build_s:.1f} s"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch

    from paper_1910_02611_gb300 import Rambo

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    t_gen = time.perf_counter()
    w = make_workload(args.config, args.scale, args.m_log2, args.queries)
    batches = extra_batches(w, args.batches, rank)
    t_gen = time.perf_counter() - t_gen

    # ---- construction (Algorithm 1) ----
    g = Rambo(w.K, w.B, w.R, w.m, w.eta, w.seed)
    sets = w.sets
    d_ids = torch.from_numpy(sets.ids.view(np.int64)).to(dev)
    d_data = torch.from_numpy(sets.data.view(np.int64) if sets.kind == "keys" else sets.data).to(dev)
    d_off = torch.from_numpy(sets.offsets.view(np.int64)).to(dev)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.insert(d_ids, d_data, d_off, kind=sets.kind, k=w.k)
    e1.record(stream)
    e1.synchronize()
    build_ms = e0.elapsed_time(e1)
    build_keys = keys_in(sets, w.k)
    del d_ids, d_data, d_off
    torch.cuda.empty_cache()

    # ---- query batches resident in device memory ----
    dev_batches = []
    for q in batches:
        qd = torch.from_numpy(q.data.view(np.int64) if q.kind == "keys" else q.data).to(dev)
        qo = torch.from_numpy(q.offsets.view(np.int64)).to(dev)
        dev_batches.append((qd, qo, keys_in(q, w.k), len(q)))
    tuned = None
    if args.autotune and not args.query_config:
        qd0, qo0, _, _ = dev_batches[0]
        tuned = g.autotune(qd0, qo0, kind=batches[0].kind, k=w.k, reps=2)
    if args.query_config:
        g.set_config(**{kv.split("=")[0]: int(kv.split("=")[1]) for kv in args.query_config.split(",")})
    # size the caller-owned result buffer: a call with no room reports the IDs needed
    from paper_1910_02611_gb300 import ENOSPC, RamboError

    need = 0
    probe_ids = torch.empty(1, dtype=torch.int32, device=dev)
    probe_off = torch.empty(max(len(q) for q in batches) + 1, dtype=torch.int64, device=dev)
    for qd, qo, _, nq in dev_batches:
        try:
            n_ids = g.query_into(qd, qo, probe_ids[:0], probe_off[: nq + 1], kind=batches[0].kind, k=w.k)
        except RamboError as ex:
            if ex.code != ENOSPC:
                raise
            n_ids = ex.item
        need = max(need, n_ids)
    del probe_ids, probe_off
    out_cap = max(1 << 20, int(need * 1.02) + 1024)
    out_off = torch.empty(max(len(q) for q in batches) + 1, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    out = {}  # the direct call's result buffer, allocated when first needed

    def one_step(i):
        qd, qo, nk, nq = dev_batches[i % len(dev_batches)]
        if "ids" not in out:
            out["ids"] = torch.empty(out_cap, dtype=torch.int32, device=dev)
        g.query_into(qd, qo, out["ids"], out_off[: nq + 1], kind=batches[0].kind, k=w.k)
        return nk

    plans = []
    n_plans = 0
    if args.api == "plan":
        from paper_1910_02611_gb300 import Plan
        from paper_1910_02611_gb300.rambo import _CudaArray

        # graph-captured plans, one per batch with its inputs copied into the
        # plan's device buffers before the timed region -- as many as memory
        # holds (a plan owns its result and staging buffers, device and pinned
        # host); with fewer plans than batches, each step first copies its
        # batch's inputs into the plan's device buffers (inside the step)
        elem = 8 if batches[0].kind == "keys" else 1
        max_nq = max(len(q) for q in batches)
        max_items = max(max(int(q.offsets[-1] - q.offsets[0]) for q in batches), 1)
        stage_words = min(out_cap, max_nq * ((w.K + 31) // 32))
        dev_per_plan = 4 * (stage_words + out_cap) + max_items * (elem + 1) + 40 * max_nq
        host_per_plan = 4 * out_cap + max_items * elem + 16 * max_nq
        free_dev = torch.cuda.mem_get_info(dev)[0]
        host_avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        n_plans = max(1, min(len(batches), int(0.5 * free_dev // dev_per_plan), int(0.4 * host_avail // host_per_plan)))
        for j in range(n_plans):
            plan = Plan(g, batches[0].kind, max_queries=max_nq, max_items=max_items, max_ids=out_cap, k=w.k)
            plan.set_timing(args.plan_timing)
            dst = torch.as_tensor(_CudaArray(plan.dev_data_ptr, max_items * elem, "|u1"), device=dev)
            dst_off = torch.as_tensor(_CudaArray(plan.dev_offsets_ptr, max_nq + 1, "<i8"), device=dev)
            plans.append((plan, dst, dst_off))

        def load_batch(j, i):
            qd, qo, nk, nq = dev_batches[i % len(dev_batches)]
            items = int(batches[i % len(batches)].offsets[-1] - batches[i % len(batches)].offsets[0])
            _, dst, dst_off = plans[j]
            dst[: items * elem].copy_(qd.view(torch.uint8)[: items * elem])
            dst_off[: nq + 1].copy_(qo - qo[0])
            return nq, max(items, 1), nk

        resident = [load_batch(j, j) for j in range(n_plans)]
        torch.cuda.synchronize()

        def plan_step(i):
            j = i % n_plans
            nq, items, nk = load_batch(j, i) if n_plans < len(batches) else resident[j]
            plan = plans[j][0]
            plan.launch_device(nq, items, stream=stream)
            plan.wait(to_host=False, copy=False, stream=stream)
            return nk

    step = plan_step if plans else one_step
    for i in range(args.warmup):
        flush.zero_()
        step(i)
    torch.cuda.synchronize()

    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, keys, probed, rows_read, qk_ms, launches, n_ids, staged = [], 0, 0, 0, [], 0, 0, 0
    stages = [0, 0, 0, 0]  # surviving queries by set stage: staged dense, dense, sparse, union
    for i in range(args.steps):
        flush.zero_()
        e0.record(stream)
        nk = step(i)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        keys += nk
        # counters of this step's batch, and the query kernel's time from CUDA
        # events recorded on the launching stream around it (inside the graph
        # for a plan replay)
        st = plans[i % n_plans][0].last_stats() if plans else g.last_query_stats()
        probed += st["keys_probed"]
        rows_read += st["rows_read"]
        qk_ms.append(st["query_kernel_ms"])
        launches += st["kernel_launches"]
        n_ids += st["n_results"]
        staged += st["staged_words"]
        stages = [a + b for a, b in zip(stages, st["stage_queries"])]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    qk_timing = "CUDA events recorded by nodes of the replayed graph around the query kernel" if plans else \
        "CUDA events recorded by the library on the call's stream around the query kernel"
    used_plans = len(plans)
    for pl in plans:  # their buffers are not needed past the timed region
        pl[0].close()
    plans = []
    if used_plans and not all(x > 0 for x in qk_ms):
        # the graph was captured without its timing nodes: time the same kernel
        # on the same batches through direct calls, after the timed region
        qk_timing = ("direct calls of the same batches after the timed region (graph replayed without timing "
                     "nodes)")
        qk_ms, probed, rows_read, n_ids, staged = [], 0, 0, 0, 0
        for i in range(args.steps):
            flush.zero_()
            one_step(i)
            st = g.last_query_stats()
            probed += st["keys_probed"]
            rows_read += st["rows_read"]
            qk_ms.append(st["query_kernel_ms"])
            n_ids += st["n_results"]
            staged += st["staged_words"]
    total_ms = sum(step_ms)

    # ---- end to end through the same call with host buffers ----
    host_batches = []
    for q in batches:
        hd = torch.from_numpy(q.data.view(np.int64) if q.kind == "keys" else q.data).pin_memory().numpy()
        ho = torch.from_numpy(q.offsets.view(np.int64)).pin_memory().numpy().view(np.uint64)
        host_batches.append((hd.view(np.uint64) if q.kind == "keys" else hd, ho, keys_in(q, w.k), len(q)))
    e2e_s, e2e_keys, h2d, d2h = 0.0, 0, 0, 0
    e2e_dev_ms, e2e_launch = [], set()
    n_e2e = 0 if args.no_extras else max(1, min(args.e2e_steps, args.steps))
    # untimed warm-up over every batch: the handle's pinned result arena and
    # input buffers reach their largest size before the timed calls
    for i in range(min(n_e2e, len(host_batches)) if n_e2e else 0):
        hd, ho, _, _ = host_batches[i]
        g.query(hd, ho, kind=batches[0].kind, k=w.k, copy=False)
    e2e_wall0 = time.perf_counter()
    for i in range(n_e2e):
        if i >= 2 and time.perf_counter() - e2e_wall0 > 20.0:  # bound the end-to-end leg's wall time
            n_e2e = i
            break
        hd, ho, nk, nq = host_batches[i % len(host_batches)]
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ids, offs = g.query(hd, ho, kind=batches[0].kind, k=w.k, copy=False)
        e2e_s += time.perf_counter() - t0
        e2e_keys += nk
        st = g.last_query_stats()
        e2e_dev_ms.append(st["device_ms"])
        e2e_launch.add(st["kernel_launches"])
        h2d += hd.nbytes + ho.nbytes
        d2h += offs.nbytes + ids.nbytes

    # ---- the plain one-query-per-launch kernel on the same GPU (identical results) ----
    per_launch = None
    if args.per_query_baseline and not args.no_extras:
        q0 = batches[0]
        nq = min(args.per_query_baseline, len(q0))
        sub = q0.subset(np.arange(nq))
        sd = torch.from_numpy(sub.data.view(np.int64) if sub.kind == "keys" else sub.data).to(dev)
        torch.cuda.synchronize()
        pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pe0.record(stream)
        pids, poff = g.query_one_per_launch(sd, sub.offsets, kind=sub.kind, k=w.k)
        pe1.record(stream)
        pe1.synchronize()
        p_ms = pe0.elapsed_time(pe1)
        bids, boff = g.query(sd, torch.from_numpy(sub.offsets.view(np.int64)).to(dev), kind=sub.kind, k=w.k)
        same = bool(np.array_equal(poff, boff.cpu().numpy().view(np.uint64)) and
                    np.array_equal(pids, bids.cpu().numpy().view(np.uint32)))
        per_launch = {"value": keys_in(sub, w.k) / (p_ms / 1000), "unit": UNIT, "queries": nq,
                      "launches": nq, "identical_results": same,
                      "note": "one thread block launched per query, same GPU, first queries of batch 0 "
                              "(includes the per-launch host loop; host offsets)"}

    # ---- reduce over ranks ----
    (total_ms_max, e2e_s_max), (keys_all, e2e_keys_all) = reduce_over_ranks(
        dist, [total_ms, e2e_s], [keys, e2e_keys], dev)

    # ---- roofline of the query kernel ----
    peaks = load_peaks()
    rows_per_key = w.R * w.eta
    row_bytes = g.row_stride * 4
    sectors_per_row = (row_bytes + SECTOR - 1) // SECTOR if row_bytes <= SECTOR else -(-row_bytes // SECTOR)
    # rows read (whole sectors) plus the 4-byte write of every result ID the kernel stages
    alg_bytes = rows_read * sectors_per_row * SECTOR + staged * 4
    qk_total = sum(qk_ms)
    achieved = alg_bytes / (qk_total / 1000) / 1e9
    # random-row ceiling on a buffer the size of the index
    rr = None
    try:
        if args.no_extras:
            raise RuntimeError("skipped (--no-extras)")
        from paper_1910_02611_gb300 import random_row_probe

        n_rows = w.R * w.m
        buf = torch.empty(n_rows * g.row_stride, dtype=torch.int32, device=dev)
        buf.zero_()
        reads = 1024
        blocks = torch.cuda.get_device_properties(dev).multi_processor_count * 8
        random_row_probe(buf, n_rows, g.row_stride, reads, blocks, 256)
        ms = random_row_probe(buf, n_rows, g.row_stride, reads, blocks, 256, seed=7)
        rr_reads_s = blocks * 256 * reads / (ms / 1000)
        rr_gbs = rr_reads_s * SECTOR * sectors_per_row / 1e9
        # the kernel's row reads per second against the ceiling's (row traffic only)
        kernel_reads_s = rows_read / (qk_total / 1000)
        rr = {"gbs": rr_gbs, "reads_per_s": rr_reads_s, "row_bytes": row_bytes, "buffer_bytes": n_rows * row_bytes,
              "kernel_reads_per_s": kernel_reads_s, "frac_of_roofline": kernel_reads_s / rr_reads_s}
        del buf
    except Exception as ex:  # measurement helper only
        rr = {"error": str(ex)}

    # ---- CPU oracle baseline (rank 0, N=1) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.no_extras:
        nthreads = os.cpu_count() or 1
        o, ob_s = oracle_index(w, nthreads)
        rate, n, dt = oracle_rate(o, batches[0], w.k, nthreads, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": nthreads, "kind": "oracle",
               "sample": f"first {n} queries of the timed batch ({dt:.1f} s, {nthreads} threads); oracle index "
                         f"built from the same sets in {ob_s:.1f} s"}
        del o

    if rank != 0:
        return 0
    lat = sorted(step_ms)
    line = {
        "metric": METRIC,
        "value": keys_all / (total_ms_max / 1000),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u64",
        "data": "synthetic",
        "config": {
            "workload": f"{w.name}: K={w.K} sets, B={w.B}, R={w.R}, m=2^{int(np.log2(w.m))}, eta={w.eta}, k={w.k}; "
                        f"{len(batches[0])} {'query sequences' if batches[0].kind == 'seq' else 'key queries'} "
                        f"per step (scale {args.scale})",
            "parallelism": f"replicas x{world} (one index per GPU, disjoint batches)",
            "api": "CUDA-graph plan replay" if used_plans else "rambo_query_*_into call",
            "autotuned": bool(tuned),
            "l2": f"flushed before every step (256 MiB write); index {g.info().index_bytes / 2**30:.1f} GiB",
            "batches": len(batches),
            "plans": used_plans,
            "plan_timing_nodes": bool(used_plans and args.plan_timing),
        },
        "batch_latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
        "keys_probed_frac": probed / max(keys, 1),
        "results_per_step": n_ids / args.steps,
        "result_bytes_per_s": n_ids * 4 / (total_ms_max / 1000),
        "e2e": ({"value": e2e_keys_all / e2e_s_max, "unit": UNIT, "h2d_bytes_per_step": h2d // n_e2e,
                 "d2h_bytes_per_step": d2h // n_e2e, "steps": n_e2e, "ms_per_step": 1000 * e2e_s / n_e2e,
                 "device_ms_per_step": statistics.mean(e2e_dev_ms),
                 "kernel_launches_per_call": sorted(e2e_launch)} if n_e2e else None),
        "gpu_launches": launches,
        "roofline": {
            "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": ncu_traffic(w.name),
            "kernel": "k_query", "peak_source": peaks["source"],
            "bytes_model": f"rows read (device counter) x {sectors_per_row} sector(s) x 32 B + 4 B per staged word "
                           "(an ID of a list-staged answer or a word of a bitmap-staged one; device counter)",
            "staged_words_per_step": staged / args.steps,
            "rows_read_per_step": rows_read / args.steps,
            "rows_per_submitted_key": rows_read / max(keys, 1),
            "query_kernel_ms_per_step": qk_total / args.steps,
            "kernel_timing": qk_timing,
            "set_stage_queries_per_step": {name: v / args.steps for name, v in
                                           zip(("staged_dense", "dense", "sparse", "union"), stages)},
        },
        "random_row_roofline": rr,
        "construction": {"keys": build_keys, "ms": build_ms, "keys_per_s": build_keys / (build_ms / 1000)},
        "clocks": clocks,
        "cpu_baseline": cpu,
        "per_query_launch_baseline": per_launch,
        "query_config": tuned or g.get_config(),
        "setup_s": {"workload_generation": t_gen},
    }
    print(json.dumps(line), flush=True)
    if args.json_out:
        with open(args.json_out, "w") as f:
            json.dump(line, f, indent=1)
    if dist:
        dist.destroy_process_group()
    g.close()
    return 0


# ---------------------------------------------------------------------------
# serving (continuous batching with streaming inserts)
# ---------------------------------------------------------------------------

def serving_workload(scale: float, rng):
    """Document index (K docs over a Zipf(1.0) vocabulary, B=320, R=8, m=2^25,
    eta=3) plus genome-like sets for the DNA queries, and new documents to
    stream in, 100 per insert batch."""
    docs = synth.make("document", scale)
    gen = synth.make("genome", 0.1 * max(scale, 0.05))
    vocab = docs.meta["vocab_keys"]
    df = docs.meta["df"]
    p = df / df.sum()
    mu = np.log(500.0) - 0.5
    new_docs = []
    for _ in range(400):
        L = int(np.clip(np.round(rng.lognormal(mu, 1.0)), 1, vocab.size))
        new_docs.append(np.unique(vocab[rng.choice(vocab.size, L, p=p)]))
    return docs, gen, new_docs, p


def serving_requests(rng, docs, gen, p, n):
    """A third each: 1-term and 5-term key queries by corpus term frequency,
    and DNA substrings of U{31..2000} bases of the genome-like sets."""
    vocab = docs.meta["vocab_keys"]
    kinds = np.zeros(n, np.uint8)
    payload = []
    r = rng.random(n)
    for i in range(n):
        if r[i] < 1 / 3:
            payload.append(vocab[rng.choice(vocab.size, 1, p=p)].astype(np.uint64).view(np.uint8))
        elif r[i] < 2 / 3:
            payload.append(vocab[rng.choice(vocab.size, 5, replace=False, p=p)].astype(np.uint64).view(np.uint8))
        else:
            kinds[i] = 1
            gi = int(rng.integers(0, len(gen.sets)))
            s = gen.sets.item(gi)
            L = int(min(s.size, rng.integers(31, 2001)))
            a = int(rng.integers(0, s.size - L + 1))
            payload.append(s[a: a + L])
    boff = np.zeros(n + 1, np.uint64)
    np.cumsum([x.size for x in payload], out=boff[1:])
    return kinds, np.concatenate(payload), boff, payload


def run_serving(args):
    import torch

    from paper_1910_02611_gb300 import Rambo, Server

    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rng = np.random.default_rng(1005)
    t_gen = time.perf_counter()
    docs, gen, new_docs, p = serving_workload(args.scale, rng)
    rates = [float(x) for x in args.rates.split(",")]
    n_req = args.requests_per_rate
    phases = [serving_requests(rng, docs, gen, p, n_req) for _ in rates]
    t_gen = time.perf_counter() - t_gen
    n_docs, n_gen = len(docs.sets), len(gen.sets)
    K = n_docs + n_gen + len(new_docs)
    g = Rambo(K, docs.B, docs.R, docs.m, docs.eta, 42)
    g.insert(docs.sets.ids, docs.sets.data, docs.sets.offsets, kind="keys")
    g.insert(gen.sets.ids + np.uint64(n_docs), gen.sets.data, gen.sets.offsets, kind="seq")
    srv = Server(g, slots=4, max_batch_queries=1024, max_batch_bases=1024 * 2000, max_batch_keys=1024 * 5,
                 max_batch_ids=1 << 25)
    sweep = []
    next_doc = 0
    check_sample = []
    clocks = None
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    time.sleep(0.3)
    for (kinds, payload, boff, items), rate in zip(phases, rates):
        # a streamed insert batch of 100 new documents before every phase
        batch = new_docs[next_doc: next_doc + 100]
        ids = np.arange(n_docs + n_gen + next_doc, n_docs + n_gen + next_doc + len(batch), dtype=np.uint64)
        off = np.zeros(len(batch) + 1, np.uint64)
        np.cumsum([b.size for b in batch], out=off[1:])
        t_ins = srv.submit_insert(ids, np.concatenate(batch), off, kind="keys")
        next_doc += len(batch)
        srv.drain()
        srv.result(t_ins)
        srv.reset_stats()
        arrivals = np.cumsum(rng.exponential(1e9 / rate, len(kinds))).astype(np.uint64)
        # a client thread collects answers as they complete (tickets are issued
        # in submission order, right after the insert's), as a serving client
        # would, so finished batches' buffers return to the server's pool
        results = [None] * len(kinds)

        def collect(first=int(t_ins) + 1, out=results):
            for i in range(len(out)):
                out[i] = srv.result(first + i)[0]

        collector = threading.Thread(target=collect)
        collector.start()
        t0 = time.perf_counter()
        tickets = srv.replay(kinds, payload, boff, arrivals)
        srv.drain()
        wall = time.perf_counter() - t0
        collector.join()
        st = srv.stats()
        assert int(tickets[0]) == int(t_ins) + 1 and int(tickets[-1]) == int(t_ins) + len(kinds)
        keys = st["keys"]
        sweep.append({"rate_per_s": rate, "offered_s": float(arrivals[-1]) / 1e9, "wall_s": wall,
                      "queries": st["queries"], "batches": st["batches"],
                      "mean_batch": st["queries"] / max(st["batches"], 1),
                      "keys_per_s": keys / wall, "queries_per_s": st["queries"] / wall,
                      "p50_ms": st["p50_ns"] / 1e6, "p99_ms": st["p99_ns"] / 1e6, "max_ms": st["max_ns"] / 1e6,
                      "worker_s": {k: st[k + "_ns"] / 1e9 for k in ("admit", "finish", "insert", "idle")}})
        sel = rng.choice(len(kinds), 64, replace=False)
        check_sample.append((sel, kinds, items, results))
    clocks = sampler.stop()
    srv.close()
    # served answers equal the plain query call at the same (final) index state
    # for the last phase (no insert happened after it)
    sel, kinds, items, results = check_sample[-1]
    same = True
    for i in sel:
        kind = "keys" if kinds[i] == 0 else "seq"
        data = items[i].view(np.uint64) if kind == "keys" else items[i]
        ids_plain, _ = g.query(data, np.array([0, data.size], np.uint64), kind=kind)
        same &= bool(np.array_equal(ids_plain, results[i]))
    best = max(sweep, key=lambda x: x["keys_per_s"])
    line = {
        "metric": METRIC, "value": best["keys_per_s"], "unit": UNIT, "n_gpus": 1, "steps": len(rates),
        "warmup": 0, "ms_per_step": 1000 * sum(x["wall_s"] for x in sweep) / len(sweep),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"serving: document index K={n_docs} (+{n_gen} genome sets, +{len(new_docs)} "
                               f"streamed docs capacity), B={docs.B}, R={docs.R}, m=2^{int(np.log2(docs.m))}, "
                               f"eta={docs.eta}; Poisson arrivals, 1/3 1-term, 1/3 5-term, 1/3 DNA 31-2000 bases; "
                               f"100-document insert batch before every rate phase",
                   "step": f"one rate phase of {n_req} requests", "slots": 4},
        "latency": {"p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"]},
        "sweep": sweep,
        "served_equals_plain_call": same,
        "e2e": {"value": best["keys_per_s"], "unit": UNIT,
                "h2d_bytes_per_step": int(sum(x.size for x in phases[-1][3])),
                "d2h_bytes_per_step": None, "note": "requests enter from host memory and results return to host "
                                                    "memory inside the measured latency"},
        "clocks": clocks,
        "setup_s": {"workload_generation": t_gen},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                json.dump(line, f, indent=1)
    g.close()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "serving":
        return run_serving(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
