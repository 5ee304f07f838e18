"""Benchmark: exact 100-NN queries/s on 1B x 128-bit codes, multi-index
hashing vs linear scan, on GB300.

A step is one batch of 10,000 queries through mih_knn (Algorithm 3) on an
index built once over n = 10^9 LSH-style 128-bit codes (m = 4 substrings of
32 bits).  Inputs are resident in HBM when the timed region starts; the
codes (16 GB) and the tables are far larger than L2, so no flush is needed.
The same batch through linscan_knn is timed once as the comparator, the
end-to-end figure adds the host<->device copies through the C-ABI, and the
CPU oracle is timed on a bounded sample of queries (the reported baseline).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload H|1|2|3|4] [--n N] [--nq NQ] [--k K] [--m M]

Multi-GPU: one process per GPU (torchrun), every rank holds the whole
database (replicas) and answers its own 10,000 queries; value = all queries
of all ranks / the slowest rank's time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "exact 100-NN queries/s on 1B×128-bit codes, MIH vs linear scan on GB300; p99 ms"

# mih_params.executor values (include/mih.h)
EXECUTORS = {"graph": 2, "host": 1}
# candidate m for the autotuner (substrings of at most 32 bits)
AUTOTUNE_M = {"H": [4, 5], "1": [3, 4, 5], "2": [5, 6, 7], "3": [2, 3, 4], "4": [8, 9, 10]}
# workload name -> (kind, n, q, nq, k, m); "kper" = per-query log-uniform k
WORKLOADS = {
    "H": ("lsh", 1_000_000_000, 128, 10_000, 100, 4),
    "1": ("uniform", 100_000, 64, 1_000, 100, 4),
    "2": ("lsh", 10_000_000, 128, 10_000, 100, 6),
    "3": ("uniform", 1_000_000_000, 64, 10_000, "kper", 2),
    "4": ("lsh", 1_000_000_000, 256, 10_000, "kper", 9),
    "5": ("serve", 1_000_000_000, 128, 0, "kper", 4),
}
WORKLOAD_NAMES = {
    "H": "1B x 128-bit LSH-style codes, 10k queries, k=100",
    "1": "100k x 64-bit uniform codes, 1k queries, k=100",
    "2": "10M x 128-bit LSH-style codes, 10k queries, k=100",
    "3": "1B x 64-bit uniform codes, 10k queries, k log-uniform [1,1000]",
    "4": "1B x 256-bit LSH-style codes, 10k queries, k log-uniform [1,1000]",
    "5": "serving: 1M x 64 uniform + 100M x 128 LSH + 1B x 128 LSH, Poisson, k log-uniform [1,1000]",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="H", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--nq", type=int, default=None)
    ap.add_argument("--k", type=int, default=None)
    ap.add_argument("--m", type=int, default=None)
    ap.add_argument("--cpu-sample", type=int, default=32, help="queries timed on the CPU oracle")
    ap.add_argument("--no-linscan", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--probe", type=int, default=0, help="bound-probe entries per bucket (0 default, <0 off)")
    ap.add_argument("--no-autotune", action="store_true", help="use the workload's default m")
    ap.add_argument("--serve-qps", type=float, default=200_000.0, help="offered load of the serving check")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--tail-from", type=int, default=0,
                    help="step from which k-NN queries run two steps per wave (0: chosen by mih_tune_search, "
                         "or never with --no-autotune; <0 never)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads (1e9 x 64, 1e9 x 256, three-database serving) after the headline")
    ap.add_argument("--opt-substrings", action="store_true",
                    help="optimised substrings (Sec. 5.5): greedy bit order from a 10M-code sample")
    ap.add_argument("--executor", default="graph", choices=["graph", "host"],
                    help="k-NN wave loop: one CUDA graph (while node) or a host loop (per-kernel profiling)")
    a = ap.parse_args()
    if a.warmup < 3:
        ap.error("--warmup must be at least 3")
    return a


def workload_name(a):
    kind, n, q, nq, k, m = workload(a)
    if (n, nq, k) == WORKLOADS[a.workload][1:2] + WORKLOADS[a.workload][3:5]:
        return WORKLOAD_NAMES[a.workload]
    ks = "k log-uniform [1,1000]" if k == "kper" else f"k={k}"
    return f"{n:.0e} x {q}-bit {'LSH-style' if kind == 'lsh' else 'uniform'} codes, {nq} queries, {ks}"


def workload(a):
    kind, n, q, nq, k, m = WORKLOADS[a.workload]
    n = a.n or n
    nq = a.nq or nq
    k = a.k or k
    m = a.m or m
    return kind, n, q, nq, k, m


# ------------------------------------------------------------------ helpers
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        # raw samples: a temporary file unless MIH_BENCH_CLOCKS_CSV names one to keep
        self.path = os.environ.get("MIH_BENCH_CLOCKS_CSV") or os.path.join(
            tempfile.gettempdir(), f"mih_clocks_rank{gpu_index}_{os.getpid()}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def make_codes(kind, n, q, seed, device):
    from paper_1307_2982_gb300 import synth

    if kind == "uniform":
        return synth.uniform_codes_torch(n, q, seed, device=device)
    return synth.lsh_codes_torch(n, q, seed, device=device)


def per_query_k(nq, k, seed_shift=0):
    from paper_1307_2982_gb300 import synth

    if k == "kper":
        return synth.per_query_k(nq, seed=3 + seed_shift, kmax=1000)
    return None


# The files the slice kernel's translation unit and the tables it streams are
# compiled from: a DRAM capture stays valid while these hash the same.
SLICE_SOURCES = ("search.cu", "search.h", "index.h", "launch.h", "mih_internal.cuh", "substrings.h",
                 "build.cu", "util_kernels.cu")


def source_sha256() -> str:
    """Hash of the slice kernel's sources (SLICE_SOURCES and include/mih.h), as in profiles/."""
    import hashlib

    files = [os.path.join(ROOT, "paper_1307_2982_gb300", "csrc", f) for f in SLICE_SOURCES]
    files.append(os.path.join(ROOT, "include", "mih.h"))
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def slice_traffic(info, slice_launches, bstats, steps, q, kind, n, m):
    """DRAM bytes per launch of the slice kernel from the committed ncu
    summary (dram__bytes_read.sum + dram__bytes_write.sum over the slice
    kernel's launches of one batch on the same workload), if the kernel
    sources still hash as they did when it was captured; else (None, None)."""
    path = os.path.join(ROOT, "profiles", "search_stream_1Bx128_k100_dram.txt")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if "=" in line:
                    k, v = line.split("=", 1)
                    kv[k.strip()] = v.strip()
        same = (kv.get("source_sha256") == source_sha256() and int(kv.get("n", -1)) == n and
                int(kv.get("q", -1)) == q and int(kv.get("m", -1)) == m and kv.get("codes") == kind)
        if same:
            return float(kv["dram_bytes_per_launch"]), os.path.relpath(path, ROOT)
    except (OSError, ValueError, KeyError):
        pass
    return None, None


# -------------------------------------------------------------- CPU oracle
def cpu_oracle_time(db_host, qs_host, k, sample: int):
    """Time the oracle on `sample` queries with all host cores; (q/s, cores, results)."""
    import oracle

    oracle.build()
    qs = np.ascontiguousarray(qs_host[:sample])
    cores = min(oracle.default_threads(), len(qs))
    t0 = time.perf_counter()
    res = oracle.knn(db_host, qs, k if isinstance(k, int) else k[:sample], nthreads=cores)
    dt = time.perf_counter() - t0
    return len(qs) / dt, cores, dt, res


# ------------------------------------------------------------------- arms
def run_reference(a):
    """The oracle (plain CPU linear scan) on a bounded sample of the same workload."""
    world, rank, local = dist_env()
    if rank != 0:
        return
    import torch

    import oracle

    kind, n, q, nq, k, m = workload(a)
    dev = torch.device("cuda", local) if torch.cuda.is_available() else torch.device("cpu")
    codes = make_codes(kind, n, q, 0, dev)
    queries = make_codes(kind, nq, q, 1, dev)
    db = codes.cpu().numpy().view(np.uint64)
    qs = queries.cpu().numpy().view(np.uint64)
    del codes, queries
    kq = per_query_k(nq, k)
    kk = k if kq is None else kq
    oracle.build()
    cores = oracle.default_threads()
    # per step: a bounded sample sized for a few seconds of CPU work
    sample = max(1, min(a.cpu_sample, nq))
    for _ in range(a.warmup):
        oracle.knn(db, qs[:min(sample, cores)], kk if isinstance(kk, int) else kk[:min(sample, cores)],
                   nthreads=cores)
    t0 = time.perf_counter()
    done = 0
    for s in range(a.steps):
        lo = (s * sample) % nq
        sl = slice(lo, min(nq, lo + sample))
        oracle.knn(db, qs[sl], kk if isinstance(kk, int) else kk[sl], nthreads=cores)
        done += sl.stop - sl.start
    dt = time.perf_counter() - t0
    value = done / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000 * dt / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": workload_name(a), "n": n, "q": q, "nq": nq, "k": k if k != "kper" else
                   "log-uniform[1,1000]", "codes": kind},
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample} queries per step over all {n} codes"},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(a):
    import torch

    import paper_1307_2982_gb300 as mih

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    mih.load()
    kind, n, q, nq, k, m = workload(a)
    W = q // 64

    # inputs: the whole database on every rank, this rank's own queries
    t0 = time.perf_counter()
    codes = make_codes(kind, n, q, 0, dev)
    from paper_1307_2982_gb300 import replicas

    all_q = make_codes(kind, nq * world, q, 1, dev)
    lo, hi = replicas.shard(nq * world, world, rank)      # this rank's queries (weak scaling)
    queries = all_q[lo:hi].contiguous()
    del all_q
    kq_np = per_query_k(nq, k, seed_shift=rank)
    kt = torch.from_numpy(kq_np.astype(np.int32)).to(dev) if kq_np is not None else None
    karg = kt if kt is not None else k
    torch.cuda.synchronize()
    torch.cuda.empty_cache()      # hand the generator's cached blocks back before the build
    gen_s = time.perf_counter() - t0

    # m by the library's autotuner on 1000 hold-out queries (Sec. 6), unless --m is given
    tune = None
    if not a.no_autotune and a.m is None:
        hold = make_codes(kind, 1000, q, 5, dev)
        kk_tune = k if k != "kper" else 100
        t0 = time.perf_counter()
        m, tune_ms = mih.mih_autotune(codes, q, hold, kk_tune, candidates=AUTOTUNE_M[a.workload], probe=a.probe,
                                      executor=EXECUTORS[a.executor])
        tune = {"candidates": AUTOTUNE_M[a.workload], "ms_per_query": {str(kq): v for kq, v in tune_ms.items()},
                "chosen_m": m, "holdout_queries": 1000, "k": kk_tune, "seconds": time.perf_counter() - t0}
        del hold
        torch.cuda.empty_cache()

    # optimised substrings (Sec. 5.5): bit correlation over 10M codes, greedy order
    order, substrings = None, "consecutive (Sec. 2.1)"
    if a.opt_substrings:
        t0 = time.perf_counter()
        sample = codes[: min(n, 10_000_000)]
        order = mih.optimize_substrings(sample, q, m, seed=0)
        substrings = {"method": "greedy on bit correlation (Sec. 5.5)", "sample_codes": int(sample.shape[0]),
                      "seconds": time.perf_counter() - t0}
        del sample

    # index build (Algorithm 1), timed on the device
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    index = mih.mih_build(codes, q, m, probe=a.probe, executor=EXECUTORS[a.executor], bit_order=order,
                          tail_from=a.tail_from)
    ev1.record()
    torch.cuda.synchronize()
    build_ms = ev0.elapsed_time(ev1)
    info = index.info()
    # launch choices of the k-NN waves (slice-kernel shape, two-step start),
    # timed on the hold-out queries and kept in the index
    # (hold-out batch of the benchmark's size: the per-wave overheads that
    # two-step waves save weigh differently in smaller batches)
    search_tuning = None
    if not a.no_autotune and a.tail_from == 0:
        hold = make_codes(kind, nq, q, 5, dev)
        t0 = time.perf_counter()
        best, table = mih.mih_tune_search(index, hold, k if k != "kper" else 100)
        search_tuning = {"chosen": best, "ms_per_query": table, "holdout_queries": nq,
                         "seconds": time.perf_counter() - t0}
        del hold
        torch.cuda.empty_cache()

    # outputs preallocated (the call writes into caller buffers)
    if kt is None:
        out_ids = torch.empty((nq, k), dtype=torch.int32, device=dev)
        out_dist = torch.empty((nq, k), dtype=torch.int32, device=dev)
    else:
        tot = int(kt.sum().item())
        out_ids = torch.empty(tot, dtype=torch.int32, device=dev)
        out_dist = torch.empty(tot, dtype=torch.int32, device=dev)

    def step():
        return mih.mih_knn(index, queries, karg, out=(out_ids, out_dist))

    sampler = ClockSampler(local)
    sampler.start()                       # clocks sampled from the warm-up through the timed region
    for _ in range(a.warmup):
        r = step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, device time, max over ranks
    mih.mih_set_timing(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats_acc = {"lookups": 0, "candidates_raw": 0, "candidates_unique": 0, "steps": 0, "phase2_queries": 0,
                 "waves": 0, "candidates_sliced": 0}
    main_ms, main_launches, launches = 0.0, 0, 0
    e0.record()
    for _ in range(a.steps):
        r = step()
        prof = mih.mih_last_profile()
        main_ms += prof["main_ms"]
        main_launches += prof["main_launches"]
        launches += prof["launches"]
        for key in stats_acc:
            stats_acc[key] += r["stats"][key]
    e1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    mih.mih_set_timing(False)
    ms = replicas.max_over_ranks(e0.elapsed_time(e1), device=dev)
    ms_per_step = ms / a.steps
    value = world * nq * a.steps / (ms / 1000.0)

    # ---- per-kernel breakdown: a few more batches with an event pair around
    # every launch (the waves then run from a host loop: same kernels and
    # results, no graph), outside the timed region
    breakdown_steps = 3
    mih.mih_set_timing(2)
    kern_ms = {kk: 0.0 for kk in mih.PROF_KINDS}
    kern_n = {kk: 0 for kk in mih.PROF_KINDS}
    bstats = {"candidates_raw": 0, "candidates_sliced": 0, "lookups": 0}
    for _ in range(breakdown_steps):
        r = step()
        prof = mih.mih_last_profile()
        for kk in mih.PROF_KINDS:
            kern_ms[kk] += prof["kernel_ms"][kk]
            kern_n[kk] += prof["kernel_launches"][kk]
        for kk in bstats:
            bstats[kk] += r["stats"][kk]
    mih.mih_set_timing(False)
    torch.cuda.synchronize()
    kernels = {kk: {"ms_per_step": kern_ms[kk] / breakdown_steps, "launches_per_step": kern_n[kk] / breakdown_steps}
               for kk in mih.PROF_KINDS if kern_n[kk]}

    # ---- roofline of the dominant kernel, algorithmic bytes
    sparse = [kd == mih.MIH_TABLE_SPARSE for kd in info["table_kind"]]
    bytes_per_lookup = 8 + (8 if all(sparse) else 0)       # bucket bounds (+ one {key, rank} slot)
    # full code per candidate; the id too unless the tables keep codes inline.
    # When every substring is one 32-bit word (m = q/32) the inline records
    # leave out the table's own word (its distance is the ring radius).
    if info["inline_codes"]:
        bytes_per_cand = q // 8 - (4 if m == q // 32 else 0)
    else:
        bytes_per_cand = q // 8 + 4
    alg_bytes = stats_acc["lookups"] * bytes_per_lookup + stats_acc["candidates_raw"] * bytes_per_cand
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    # The whole search (both search kernels, every wave): bytes over the span of
    # the wave-loop graph in the timed batches (the span also holds each wave's
    # planning and stopping test, so this rate slightly understates the kernels).
    span_rate = (alg_bytes / max(main_launches, 1)) / ((main_ms / max(main_launches, 1)) / 1000.0) / 1e9 \
        if main_ms > 0 else None
    # The dominant kernel alone: the slice kernel (big buckets), its candidates'
    # bytes over its own event time in the breakdown batches.
    slice_ms = kern_ms["slice"] / breakdown_steps
    slice_launches = kern_n["slice"] / breakdown_steps
    slice_bytes = (bstats["candidates_sliced"] / breakdown_steps) * bytes_per_cand
    achieved = slice_bytes / (slice_ms / 1000.0) / 1e9 if slice_ms > 0 else None
    traffic, traffic_src = slice_traffic(info, slice_launches, bstats, breakdown_steps, q, kind, n, m)
    roofline = {"bound": "hbm",
                "kernel": ("search_stream_kernel (big-bucket slices of inline codes or records, streamed by bulk "
                           "copies)" if info["inline_codes"] else "search_big_kernel (big-bucket slices, by id)"),
                "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": (achieved / hbm_peak) if achieved else None, "traffic": traffic,
                "traffic_source": traffic_src,
                "peak_source": "measured (burst copy)" if "hbm_gbs" in peaks else "fallback",
                "alg_bytes_per_launch": slice_bytes / max(slice_launches, 1e-9),
                "ms_per_launch": slice_ms / max(slice_launches, 1e-9), "launches_per_step": slice_launches,
                "bytes_model": f"{bytes_per_cand} B per streamed candidate",
                "timing": "CUDA events around each launch, host-loop waves, 3 batches after the timed region",
                "search_span": {"kernels": "search_kernel + slice kernel, every wave (graph span, timed batches)",
                                "achieved": span_rate, "frac": (span_rate / hbm_peak) if span_rate else None,
                                "alg_bytes_per_step": alg_bytes / a.steps,
                                "ms_per_step": main_ms / a.steps,
                                "bytes_model": f"{bytes_per_lookup} B/lookup + {bytes_per_cand} B/raw candidate",
                                "share_of_step": main_ms / ms if ms > 0 else None},
                "kernels_ms_per_step": kernels}

    # ---- end to end through the C-ABI with host buffers (pinned), K steps
    qh = queries.cpu().pin_memory()
    ids_h = torch.empty(out_ids.shape, dtype=torch.int32).pin_memory()
    dist_h = torch.empty(out_dist.shape, dtype=torch.int32).pin_memory()
    qd = torch.empty_like(queries)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    for _ in range(a.steps):
        qd.copy_(qh, non_blocking=True)
        mih.mih_knn(index, qd, karg, out=(out_ids, out_dist))
        ids_h.copy_(out_ids, non_blocking=True)
        dist_h.copy_(out_dist, non_blocking=True)
    f1.record()
    torch.cuda.synchronize()
    e2e_ms = replicas.max_over_ranks(f0.elapsed_time(f1), device=dev)
    e2e = {"value": world * nq * a.steps / (e2e_ms / 1000.0), "unit": "queries/s",
           "h2d_bytes_per_step": int(qh.numel() * 8),
           "d2h_bytes_per_step": int((ids_h.numel() + dist_h.numel()) * 4)}

    # ---- linear scan comparator on the same batch (one timed pass)
    linscan = None
    if not a.no_linscan:
        ls_q = queries[:min(nq, 256)]
        mih.linscan_knn(codes, q, ls_q, karg if kt is None else kt[:ls_q.shape[0]])   # warm-up
        torch.cuda.synchronize()
        mih.mih_set_timing(True)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record()
        ls = mih.linscan_knn(codes, q, queries, karg)
        g1.record()
        torch.cuda.synchronize()
        lprof = mih.mih_last_profile()
        mih.mih_set_timing(False)
        ls_ms = g0.elapsed_time(g1)
        same = bool(torch.equal(ls["ids"], out_ids) and torch.equal(ls["dist"], out_dist))
        pairs = float(n) * nq
        linscan = {"value": nq / (ls_ms / 1000.0), "unit": "queries/s", "ms_per_batch": ls_ms,
                   "mih_speedup": (value / world) / (nq / (ls_ms / 1000.0)),
                   "identical_to_mih": same, "pairs_per_s": pairs / (ls_ms / 1000.0),
                   "scan_kernel_ms": lprof["main_ms"]}

    # ---- the other form of the scan on the first 1000 queries (fp8 tensor-core
    # products; the timed pass above is the default form, xor + popcount)
    if linscan:
        pq = queries[:1000].contiguous()
        pk = karg if kt is None else kt[:1000].contiguous()
        mih.mih_set_scan_kernel(mih.MIH_SCAN_TENSOR)
        mih.linscan_knn(codes, q, pq[:64], karg if kt is None else kt[:64].contiguous())
        torch.cuda.synchronize()
        g0.record()
        pls = mih.linscan_knn(codes, q, pq, pk)
        g1.record()
        torch.cuda.synchronize()
        mih.mih_set_scan_kernel(mih.MIH_SCAN_AUTO)
        p_ms = g0.elapsed_time(g1)
        nrow = pq.shape[0]
        same_p = bool(torch.equal(pls["ids"], ls["ids"][:nrow]) and torch.equal(pls["dist"], ls["dist"][:nrow])) \
            if kt is None else None
        linscan["kernel"] = "xor + popcount with an OR lower bound"
        linscan["tensor_form"] = {"kernel": "fp8 tensor-core products (mma.sync m16n8k32 e4m3, +-1 codes)",
                                  "queries": nrow, "pairs_per_s": float(n) * nrow / (p_ms / 1000.0),
                                  "ms": p_ms, "identical": same_p}

    # ---- measured ceilings of this GPU (POPC, tensor-core Hamming forms,
    # random 32-byte reads), after the timed regions
    ceilings = mih.mih_measure_ceilings(gather_bytes=8 << 30)
    if linscan:
        # the tensor-core scan against the measured fp8 mma.sync rate (a pair
        # of q-bit codes is q multiply-adds); the popcount form against the
        # measured POPC rate at one POPC per pair (the OR lower bound settles
        # most pairs in one)
        fp8_pairs = ceilings["fp8_mma_tflops"] * 1e12 / (2.0 * q)
        linscan["roofline"] = {"bound": "alu", "achieved": linscan["pairs_per_s"], "unit": "pairs/s",
                               "peak": ceilings["popc_per_s"], "frac": linscan["pairs_per_s"] / ceilings["popc_per_s"],
                               "peak_source": "measured POPC rate (mih_measure_ceilings)",
                               "model": "one 32-bit POPC per (query, code) pair"}
        tf = linscan["tensor_form"]
        tf["roofline"] = {"bound": "tensor", "achieved": tf["pairs_per_s"], "unit": "pairs/s",
                          "peak": fp8_pairs, "frac": tf["pairs_per_s"] / fp8_pairs,
                          "peak_source": "measured fp8 mma.sync rate (mih_measure_ceilings)",
                          "model": f"{q} e4m3 multiply-adds per (query, code) pair"}

    # ---- re-ranking phase (Sec. 5.1): the batch's Hamming 100-NN lists
    # re-ranked to 10 by the asymmetric distance to the queries' real
    # projections (mih_rerank_asym), L2 flushed before every timed launch
    rerank = None
    if kind == "lsh" and kt is None and k >= 10:
        from paper_1307_2982_gb300 import synth

        _, proj_all = synth.lsh_projections_torch(nq * world, q, 1, device=dev)
        proj = proj_all[lo:hi].contiguous()
        del proj_all
        ko, reps = 10, 10
        rr_out = (torch.empty((nq, ko), dtype=torch.int32, device=dev),
                  torch.empty((nq, ko), dtype=torch.float64, device=dev))
        flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
        for _ in range(3):
            mih.mih_rerank_asym(codes, q, proj, out_ids, ko, out=rr_out)
        mih.mih_set_timing(True)
        r_ms, r_call = 0.0, 0.0
        for i in range(reps):
            flush.fill_(i)
            mih.mih_rerank_asym(codes, q, proj, out_ids, ko, out=rr_out)
            rp = mih.mih_last_profile()
            r_ms += rp["main_ms"]
            r_call += rp["call_ms"]
        mih.mih_set_timing(False)
        del flush
        r_ms /= reps
        cands = int((out_ids != -1).sum().item())
        sectors_gbs = cands * 32 / (r_ms / 1e3) / 1e9
        rerank = {"k_in": k, "k": ko, "queries": nq, "kernel": "rerank_warp_kernel (one warp per row, exact integer sums on the "
                  "query's fixed-point grid, bitonic sort by shuffles)", "kernel_ms": r_ms, "call_ms": r_call / reps,
                  "candidates_per_s": cands / (r_ms / 1e3),
                  "roofline": {"bound": "gather", "achieved": sectors_gbs, "unit": "GB/s",
                               "peak": ceilings["gather32_gbs"], "frac": sectors_gbs / ceilings["gather32_gbs"],
                               "peak_source": "measured random 32-byte read rate (mih_measure_ceilings)",
                               "model": "one random 32-byte sector per candidate code"},
                  "share_of_search": r_ms / ms_per_step,
                  "timing": f"CUDA events around the kernel, {reps} launches, 512 MB L2 flush before each"}
        del proj, rr_out

    # ---- serving: Poisson k=100 requests against the resident index (p50/p99)
    serve = None
    if not a.no_serve and kq_np is None:
        from paper_1307_2982_gb300 import serving, synth

        nreq = int(a.serve_qps * 1.0)
        gen = (lambda d, c, sd: synth.lsh_codes(c, q, sd)) if kind == "lsh" else \
            (lambda d, c, sd: synth.uniform_codes(c, q, sd))
        req = serving.poisson_requests(nreq, a.serve_qps, [q], k_max=1, seed=4, query_gen=gen)
        req.k[:] = k
        srv = serving.MihServer([index], result_budget=256 << 20, max_batch=8192)
        srv.run(serving.Requests(req.arrival[:2000] * 0.01, req.db[:2000], req.k[:2000], req.codes[:2000]))  # warm
        res = srv.run(req)
        serve = res.summary()
        serve.update({"offered_qps": a.serve_qps, "k": k, "db": workload_name(a).split(",")[0],
                      "latency": "arrival to results in host memory, continuous batching"})

    # ---- CPU oracle on a bounded sample (rank 0, N = 1) + sampled parity
    cpu = None
    parity = None
    if rank == 0 and world == 1 and not a.no_cpu:
        db_host = codes.cpu().numpy().view(np.uint64)
        qs_host = queries.cpu().numpy().view(np.uint64)
        sample = min(a.cpu_sample, nq)
        qps, cores, dt, res = cpu_oracle_time(db_host, qs_host, kq_np if kq_np is not None else k, sample)
        cpu = {"value": qps, "unit": "queries/s", "cores": cores, "kind": "oracle",
               "sample": f"first {sample} queries of the batch over all {n} codes ({dt:.1f} s)"}
        if kq_np is None:
            got_ids = out_ids[:sample].cpu().numpy().view(np.uint32)
            got_d = out_dist[:sample].cpu().numpy()
            mism = int(np.sum(np.any(got_ids != res[0], axis=1) | np.any(got_d != res[1], axis=1)))
        else:
            offs = np.concatenate([[0], np.cumsum(kq_np[:sample].astype(np.int64))])
            got_ids = out_ids[:offs[-1]].cpu().numpy().view(np.uint32)
            got_d = out_dist[:offs[-1]].cpu().numpy()
            mism = int(not (np.array_equal(got_ids, res[1]) and np.array_equal(got_d, res[2])))
        parity = {"sampled_queries": sample, "mismatched_queries": mism}
        del db_host

    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": workload_name(a), "n": n, "q": q, "nq_per_gpu": nq,
                   "k": k if k != "kper" else "log-uniform[1,1000]", "m": m, "codes": kind,
                   "parallelism": f"replicas{world}", "l2": "inputs larger than L2 (codes + tables, no flush)",
                   "substring_bits": info["substring_length"], "table_kind": info["table_kind"],
                   "index_bytes": info["index_bytes"], "build_ms": build_ms, "gen_s": gen_s,
                   "inline_codes": info["inline_codes"], "executor": a.executor, "substrings": substrings,
                   "tail_from": (search_tuning["chosen"]["tail_from"] if search_tuning else
                                 (a.tail_from if a.tail_from > 0 else "never")),
                   "search_tuning": search_tuning,
                   "autotune": tune},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": launches, "mih_stats_per_step": {kk: v / a.steps for kk, v in stats_acc.items()},
        "linscan": linscan, "parity": parity, "serving": serve, "ceilings": ceilings,
        "asym_rerank": rerank,
    }
    index.free()
    del codes, queries, out_ids, out_dist
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and a.workload == "H" and not a.no_extra and a.n is None:
        # the other configurations at reduced repeats (the headline above is the line's value)
        extra = {}
        for wl, wm in (("3", 3), ("4", 8)):   # the m the autotuner chose for these workloads
            extra[wl] = batch_workload(wl, wm, dev)
        # the by-id gather against the measured random 32-byte read ceiling
        bb = extra["4"]["big_bucket_kernel"]
        if bb["gbs"]:
            bb["ceiling_gbs"] = ceilings["gather32_gbs"]
            bb["frac_of_ceiling"] = bb["gbs"] / ceilings["gather32_gbs"]
        dbs, loads = serving_loads(a, dev)
        extra["5"] = {"workload": WORKLOAD_NAMES["5"], "databases": dbs, "loads": loads,
                      "k": "log-uniform[1,1000]", "latency": "arrival to results in host memory"}
        extra["layouts"] = layout_effect(dev)
        from paper_1307_2982_gb300 import diagnostics

        extra["asym_rerank_recall"] = diagnostics.rerank_recall(device=dev)
        line["extra_workloads"] = extra
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def serving_loads(a, dev, rates=(10_000.0, 100_000.0, 1_000_000.0)):
    """Three resident databases, Poisson requests at the offered loads; returns
    (databases, loads).  The indexes and codes are freed before returning."""
    import torch

    import paper_1307_2982_gb300 as mih
    from paper_1307_2982_gb300 import serving, synth

    specs = [("uniform", 1_000_000, 64), ("lsh", 100_000_000, 128), ("lsh", a.n or 1_000_000_000, 128)]
    dbs, idx, keep = [], [], []
    for kind, n, q in specs:
        codes = make_codes(kind, n, q, 0, dev)
        torch.cuda.empty_cache()
        m = mih.mih_suggest_m(q, n)
        idx.append(mih.mih_build(codes, q, m, probe=a.probe, executor=EXECUTORS[a.executor]))
        keep.append(codes)
        dbs.append({"codes": kind, "n": n, "q": q, "m": m, "index_bytes": idx[-1].info()["index_bytes"]})

    def gen(d, c, sd):
        kind, n, q = specs[d]
        return synth.uniform_codes(c, q, sd) if kind == "uniform" else synth.lsh_codes(c, q, sd)

    loads = []
    srv = serving.MihServer(idx, result_budget=512 << 20, max_batch=8192)
    warm = serving.poisson_requests(3000, 100_000.0, [q for _, _, q in specs], seed=9, query_gen=gen)
    srv.run(warm)
    for rate in rates:
        nreq = int(min(rate * 2.0, 2_000_000))
        req = serving.poisson_requests(nreq, rate, [q for _, _, q in specs], seed=4, query_gen=gen)
        res = srv.run(req)
        summ = res.summary()
        summ["offered_qps"] = rate
        loads.append(summ)
    for ix in idx:
        ix.free()
    del keep, idx
    torch.cuda.empty_cache()
    return dbs, loads


def run_serving(a):
    """Three resident databases, Poisson requests at three offered loads."""
    import torch

    import paper_1307_2982_gb300 as mih

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mih.load()
    dbs, loads = serving_loads(a, dev)
    best = max(l["throughput_qps"] for l in loads)
    line = {"metric": "served exact k-NN queries/s (three resident databases); p99 ms", "value": best,
            "unit": "queries/s", "n_gpus": 1, "steps": len(loads), "warmup": 1, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": WORKLOAD_NAMES["5"], "databases": dbs,
                                            "k": "log-uniform[1,1000]", "result_budget_bytes": 512 << 20,
                                            "max_batch": 8192, "workers_per_db": 2},
            "loads": loads}
    print(json.dumps(line), flush=True)


def layout_effect(dev, m=5):
    """Per-table substring lengths at 1e9 x 128-bit, k = 100: the Sec. 2.1 layout
    against the cost-model layout for the measured stop steps (m = 4 leaves no
    freedom: four 32-bit substrings), timed by mih_autotune_layout on 10^4
    hold-out queries."""
    import torch

    import paper_1307_2982_gb300 as mih

    codes = make_codes("lsh", 1_000_000_000, 128, 0, dev)
    hold = make_codes("lsh", 10_000, 128, 5, dev)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    lengths, times = mih.mih_autotune_layout(codes, 128, hold, 100, m)
    out = {"workload": "1B x 128-bit LSH-style codes, 10k hold-out queries, k=100", "m": m,
           "uniform_lengths": mih.mih_substring_layout(128, m)[1], "chosen_lengths": lengths,
           "ms_per_query": times, "seconds": time.perf_counter() - t0}
    del codes, hold
    torch.cuda.empty_cache()
    return out


def batch_workload(wl, m, dev, steps=3, warmup=3, parity_sample=6, ls_queries=1000):
    """One of the batched 1e9-code workloads at reduced repeats: queries/s of
    mih_knn over 10^4 queries (CUDA events), the linear scan on the first
    ls_queries queries, and sampled parity against the oracle over every code."""
    import torch

    import oracle
    import paper_1307_2982_gb300 as mih

    kind, n, q, nq, k, _ = WORKLOADS[wl]
    t0 = time.perf_counter()
    codes = make_codes(kind, n, q, 0, dev)
    queries = make_codes(kind, nq, q, 1, dev)
    kq = per_query_k(nq, k)
    kt = torch.from_numpy(kq.astype(np.int32)).to(dev) if kq is not None else None
    karg = kt if kt is not None else k
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    gen_s = time.perf_counter() - t0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    index = mih.mih_build(codes, q, m)
    ev1.record()
    torch.cuda.synchronize()
    build_ms = ev0.elapsed_time(ev1)
    info = index.info()
    hold = make_codes(kind, nq, q, 5, dev)
    best, _ = mih.mih_tune_search(index, hold, 100)
    del hold
    tot = int(kt.sum().item()) if kt is not None else nq * k
    out_ids = torch.empty(tot, dtype=torch.int32, device=dev)
    out_dist = torch.empty(tot, dtype=torch.int32, device=dev)
    for _ in range(warmup):
        r = mih.mih_knn(index, queries, karg, out=(out_ids, out_dist))
    torch.cuda.synchronize()
    stats = {}
    ev0.record()
    for _ in range(steps):
        r = mih.mih_knn(index, queries, karg, out=(out_ids, out_dist))
        for key, v in r["stats"].items():
            stats[key] = stats.get(key, 0) + v
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    # one more batch with an event pair around every kernel (host-loop waves)
    mih.mih_set_timing(2)
    rb = mih.mih_knn(index, queries, karg, out=(out_ids, out_dist))
    prof = mih.mih_last_profile()
    mih.mih_set_timing(0)
    kernels_ms = {kk: v for kk, v in prof["kernel_ms"].items() if prof["kernel_launches"][kk]}
    bstats = rb["stats"]
    off = r.get("offsets")
    off_h = off.cpu().numpy() if off is not None else np.arange(nq + 1, dtype=np.int64) * k
    ids_h = out_ids.cpu().numpy().view(np.uint32)
    dist_h = out_dist.cpu().numpy()
    # the linear scan on the first ls_queries queries
    lq = queries[:ls_queries].contiguous()
    lk = kt[:ls_queries].contiguous() if kt is not None else k
    mih.linscan_knn(codes, q, lq[:64], kt[:64].contiguous() if kt is not None else k)
    torch.cuda.synchronize()
    ev0.record()
    ls = mih.linscan_knn(codes, q, lq, lk)
    ev1.record()
    torch.cuda.synchronize()
    ls_ms = ev0.elapsed_time(ev1)
    ls_ids = ls["ids"].cpu().numpy().view(np.uint32)
    ls_same = bool(np.array_equal(ls_ids, ids_h[:int(off_h[ls_queries])]) and
                   np.array_equal(ls["dist"].cpu().numpy(), dist_h[:int(off_h[ls_queries])]))
    index.free()
    # sampled parity: the oracle over all n codes on a few queries spread over the batch
    rows = np.linspace(0, nq - 1, parity_sample).astype(np.int64)
    db_h = codes.cpu().numpy().view(np.uint64)
    qs_h = queries.cpu().numpy().view(np.uint64)[rows]
    del codes, queries, out_ids, out_dist, ls
    torch.cuda.empty_cache()
    ks = kq[rows] if kq is not None else k
    res = oracle.knn(db_h, qs_h, ks, nthreads=min(oracle.default_threads(), parity_sample))
    mism = 0
    for i, rrow in enumerate(rows):
        got_i = ids_h[off_h[rrow]:off_h[rrow + 1]]
        got_d = dist_h[off_h[rrow]:off_h[rrow + 1]]
        if kq is not None:
            woff, wid, wd = res
            want_i, want_d = wid[woff[i]:woff[i + 1]], wd[woff[i]:woff[i + 1]]
        else:
            want_i, want_d = res[0][i], res[1][i]
        mism += int(not (np.array_equal(got_i, want_i) and np.array_equal(got_d, want_d)))
    del db_h
    value = nq / (ms / 1000.0)
    ls_qps = ls_queries / (ls_ms / 1000.0)
    # the big-bucket kernel's bytes over its own time: whole codes by id (q/8 B
    # of code + 4 B of id per candidate) without inline codes, else inline
    if info["inline_codes"]:
        cand_b = q // 8 - (4 if m == q // 32 else 0)
    else:
        cand_b = q // 8 + 4
    slice_gbs = (bstats["candidates_sliced"] * cand_b / (kernels_ms["slice"] / 1000.0) / 1e9
                 if kernels_ms.get("slice") else None)
    return {"workload": WORKLOAD_NAMES[wl], "m": m, "search_tuning": best, "value": value, "unit": "queries/s",
            "ms_per_step": ms,
            "steps": steps, "warmup": warmup, "timing": "CUDA events around the batches",
            "build_ms": build_ms, "gen_s": gen_s, "inline_codes": info["inline_codes"],
            "index_bytes": info["index_bytes"], "mih_stats_per_step": {key: v / steps for key, v in stats.items()},
            "kernels_ms_per_step": kernels_ms,
            "big_bucket_kernel": {"gbs": slice_gbs, "bytes_model": f"{cand_b} B per candidate of a big bucket",
                                  "kind": "inline codes, streamed" if info["inline_codes"] else
                                  "codes gathered by id (random 32-byte sectors)"},
            "linscan": {"queries": ls_queries, "value": ls_qps, "unit": "queries/s", "mih_speedup": value / ls_qps,
                        "identical_to_mih": ls_same, "pairs_per_s": float(n) * ls_queries / (ls_ms / 1000.0)},
            "parity": {"sampled_queries": parity_sample, "mismatched_queries": mism, "reference": "oracle"}}


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "5":
        run_serving(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
