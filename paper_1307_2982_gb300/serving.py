"""Serving: continuous batching of exact k-NN requests over resident indexes.

Databases and their multi-index hashing tables stay resident in HBM.  A
stream of requests (arrival time, database, query code, k) is replayed on the
wall clock.  The admission thread admits an arrived request while its result
buffer (k ids + k distances) fits the result-memory budget.  For each
database, worker threads (one CUDA stream each) take every admitted request
not yet taken, up to a batch cap, and answer them with one mih_knn call with
per-query k.  Requests that arrive while a batch is on the GPU join the next
batch of a free worker, so batches of one database follow each other without
gaps, and batches of different databases overlap on the device.  Latency is
measured from arrival to the moment the results are back in host memory.

The results do not depend on how requests are batched (each query's answer is
a function of the query alone), which tests/test_serving.py checks against
one-query calls.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import mih_knn


@dataclass
class Requests:
    """A request stream: arrival[s], db[i] index, k[i], codes[i] (uint64 words, zero padded)."""

    arrival: np.ndarray   # float64, seconds from the start, non-decreasing
    db: np.ndarray        # int32 database index
    k: np.ndarray         # uint32
    codes: np.ndarray     # (N, Wmax) uint64

    def __len__(self):
        return len(self.arrival)


@dataclass
class ServeResult:
    latency_s: np.ndarray                 # per request
    done_s: np.ndarray                    # completion time per request (from start)
    batches: list = field(default_factory=list)   # (db, size, start_s, end_s)
    kept: dict = field(default_factory=dict)      # request index -> (ids, dist) for the kept sample
    elapsed_s: float = 0.0

    def summary(self) -> dict:
        lat = self.latency_s * 1e3
        n = len(lat)
        sizes = [b[1] for b in self.batches]
        return {
            "requests": n,
            "throughput_qps": n / self.elapsed_s if self.elapsed_s > 0 else None,
            "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)),
            "p999_ms": float(np.percentile(lat, 99.9)),
            "max_ms": float(lat.max()),
            "batches": len(self.batches),
            "mean_batch": float(np.mean(sizes)) if sizes else 0.0,
            "max_batch": int(max(sizes)) if sizes else 0,
        }


class MihServer:
    """Continuous batching over resident indexes (see the module docstring).

    indexes:       list of MihIndex (one per database; codes stay on the GPU)
    result_budget: bytes of result buffers that may be reserved at once
    max_batch:     largest batch one mih_knn call takes
    workers_per_db: CUDA streams (and host threads) per database
    keep:          request indices whose results are returned for checking
    """

    def __init__(self, indexes, result_budget: int = 256 << 20, max_batch: int = 8192,
                 workers_per_db: int = 2):
        self.indexes = list(indexes)
        self.result_budget = int(result_budget)
        self.max_batch = int(max_batch)
        self.workers_per_db = int(workers_per_db)

    def run(self, req: Requests, keep=()) -> ServeResult:
        import torch

        n = len(req)
        ndb = len(self.indexes)
        order = [np.nonzero(req.db == d)[0] for d in range(ndb)]     # arrival order per database
        adm = [0] * ndb        # admitted prefix of order[d]
        take = [0] * ndb       # taken prefix of order[d]
        res_bytes = req.k.astype(np.int64) * 8
        reserved = [0]
        lat = np.full(n, np.nan)
        done = np.full(n, np.nan)
        batches = []
        kept = {}
        keep = set(int(i) for i in keep)
        cv = threading.Condition()
        stop = [False]
        errors = []
        dev = torch.device("cuda", torch.cuda.current_device())
        t0 = time.perf_counter()

        def worker(d: int):
            torch.cuda.set_device(dev)
            ix = self.indexes[d]
            W = ix.q // 64
            stream = torch.cuda.Stream(device=dev)
            try:
                while True:
                    with cv:
                        while take[d] >= adm[d] and not stop[0]:
                            cv.wait(0.002)
                        if take[d] >= adm[d] and stop[0]:
                            return
                        lo = take[d]
                        hi = min(adm[d], lo + self.max_batch)
                        take[d] = hi
                    idx = order[d][lo:hi]
                    tb = time.perf_counter() - t0
                    with torch.cuda.stream(stream):
                        qh = torch.from_numpy(np.ascontiguousarray(req.codes[idx, :W]).view(np.int64)).pin_memory()
                        kh = torch.from_numpy(req.k[idx].astype(np.int32)).pin_memory()
                        qd = qh.to(dev, non_blocking=True)
                        # host k: the binding takes the CSR offsets from the host
                        # values, with no device synchronisation
                        r = mih_knn(ix, qd, kh, stream=stream)
                        ids = r["ids"].to("cpu", non_blocking=True)
                        dist = r["dist"].to("cpu", non_blocking=True)
                        off = r["offsets"].to("cpu", non_blocking=True)
                    stream.synchronize()
                    te = time.perf_counter() - t0
                    lat[idx] = te - req.arrival[idx]
                    done[idx] = te
                    if keep:
                        offn = off.numpy()
                        for j, i in enumerate(idx):
                            if int(i) in keep:
                                kept[int(i)] = (ids[offn[j]:offn[j + 1]].numpy().view(np.uint32).copy(),
                                                dist[offn[j]:offn[j + 1]].numpy().copy())
                    with cv:
                        reserved[0] -= int(res_bytes[idx].sum())
                        batches.append((d, len(idx), tb, te))
                        cv.notify_all()
            except Exception as e:  # surfaced after the run
                errors.append(e)
                with cv:
                    stop[0] = True
                    cv.notify_all()

        threads = [threading.Thread(target=worker, args=(d,), daemon=True)
                   for d in range(ndb) for _ in range(self.workers_per_db)]
        for t in threads:
            t.start()
        # admission: replay arrivals on the wall clock; per database, admit the
        # longest prefix that has arrived and whose result bytes fit the budget
        arr = [req.arrival[o] for o in order]
        cum = [np.concatenate([[0], np.cumsum(res_bytes[o])]) for o in order]
        while True:
            now = time.perf_counter() - t0
            with cv:
                progressed = False
                for d in range(ndb):
                    a0 = adm[d]
                    if a0 >= len(order[d]):
                        continue
                    arrived = int(np.searchsorted(arr[d], now, side="right"))
                    if arrived <= a0:
                        continue
                    room = self.result_budget - reserved[0]
                    fit = int(np.searchsorted(cum[d], cum[d][a0] + room, side="right")) - 1
                    if fit <= a0 and reserved[0] == 0:
                        fit = a0 + 1          # a single request larger than the budget still runs
                    a1 = min(arrived, fit)
                    if a1 > a0:
                        reserved[0] += int(cum[d][a1] - cum[d][a0])
                        adm[d] = a1
                        progressed = True
                if progressed:
                    cv.notify_all()
                if errors or all(adm[d] >= len(order[d]) for d in range(ndb)):
                    stop[0] = True
                    cv.notify_all()
                    break
            nxt = min((arr[d][adm[d]] for d in range(ndb) if adm[d] < len(order[d])), default=None)
            wait = (nxt - (time.perf_counter() - t0)) if nxt is not None else 0.0
            if wait > 0 or not progressed:
                time.sleep(min(max(wait, 0.0002), 0.0005))   # let the workers take the GIL
        for t in threads:
            t.join()
        if errors:
            raise errors[0]
        elapsed = float(np.nanmax(done)) if n else 0.0
        return ServeResult(latency_s=lat, done_s=done, batches=batches, kept=kept, elapsed_s=elapsed)


def poisson_requests(n: int, rate_qps: float, db_q: list, k_max: int = 1000, seed: int = 4,
                     query_gen=None) -> Requests:
    """n requests, Poisson arrivals at rate_qps, database uniform over len(db_q),
    k log-uniform in [1, k_max].  query_gen(d, count, seed) -> (count, q/64) uint64."""
    from . import synth

    rng = np.random.default_rng(seed)
    arrival = np.cumsum(rng.exponential(1.0 / rate_qps, size=n))
    db = rng.integers(0, len(db_q), size=n).astype(np.int32)
    u = rng.random(n)
    k = np.clip(np.floor(np.exp(u * np.log(k_max + 1.0))), 1, k_max).astype(np.uint32)
    wmax = max(q // 64 for q in db_q)
    codes = np.zeros((n, wmax), dtype=np.uint64)
    for d, q in enumerate(db_q):
        sel = np.nonzero(db == d)[0]
        if len(sel):
            codes[sel, : q // 64] = query_gen(d, len(sel), seed + 10 + d)
    return Requests(arrival=arrival, db=db, k=k, codes=codes)
