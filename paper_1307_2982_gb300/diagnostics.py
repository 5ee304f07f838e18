"""Search-radius and lookup diagnostics: the analogues of Fig. 3 (histograms of
the search radius k-NN needs) and Fig. 9 (lookups of multi-index hashing
against a single hash table and linear scan) on resident codes.

The search radius of a query for k-NN is d_k, the distance of its k-th
nearest neighbour: Algorithm 3 stops after step d_k.  Per-query counters
come from ``mih_knn(..., query_stats=True)`` (lookups, raw and unique
candidates, last step).  A single hash table over the whole q-bit code
(SHT, Sec. 5.4) probes every key within d_k bits, sum_{d <= d_k} C(q, d)
lookups (Eq. 1); linear scan compares all n codes.

    python -m paper_1307_2982_gb300.diagnostics --n 100000000 --q 128 --ks 10 1000
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import mih_build, mih_knn, mih_suggest_m


def sht_lookups_log10(q: int, radius: np.ndarray) -> np.ndarray:
    """log10 of sum_{d <= r} C(q, d) for every radius r (Eq. 1 with s = q)."""
    cum = np.cumsum([math.comb(q, d) for d in range(q + 1)], dtype=object)
    table = np.array([math.log10(int(c)) for c in cum])
    return table[np.asarray(radius, dtype=np.int64)]


def search_profile(index, queries, ks, stream=None) -> dict:
    """Per k: histogram of search radii, their moments, and the mean work per query."""
    q, n = index.q, index.info()["n"]
    out = {"q": q, "n": int(n), "m": index.m, "queries": int(queries.shape[0]), "per_k": {}}
    for k in ks:
        r = mih_knn(index, queries, int(k), query_stats=True, stream=stream)
        kk = min(int(k), int(n))
        radius = r["dist"].cpu().numpy()[:, kk - 1].astype(np.int64)
        st = r["query_stats"].cpu().numpy().astype(np.float64)
        hist = np.bincount(radius, minlength=q + 1)
        sht = sht_lookups_log10(q, radius)
        out["per_k"][str(k)] = {
            "radius_hist": {str(d): int(c) for d, c in enumerate(hist) if c},
            "radius_mean": float(radius.mean()),
            "radius_std": float(radius.std()),
            "radius_p10_p50_p90": [float(v) for v in np.percentile(radius, [10, 50, 90])],
            "mih_lookups_mean": float(st[:, 0].mean()),
            "mih_candidates_raw_mean": float(st[:, 1].mean()),
            "mih_candidates_unique_mean": float(st[:, 2].mean()),
            "mih_last_step_mean": float(st[:, 3].mean()),
            "sht_lookups_log10_mean": float(math.log10(np.mean(10.0 ** (sht - sht.max()))) + sht.max()),
            "linear_scan_comparisons": int(n),
        }
    return out


def main(argv=None):
    import torch

    from . import synth

    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=100_000_000)
    ap.add_argument("--q", type=int, default=128, choices=[64, 128, 256])
    ap.add_argument("--m", type=int, default=None)
    ap.add_argument("--nq", type=int, default=1000)
    ap.add_argument("--codes", default="lsh", choices=["lsh", "uniform"])
    ap.add_argument("--ks", type=int, nargs="+", default=[10, 1000])
    a = ap.parse_args(argv)
    dev = torch.device("cuda", torch.cuda.current_device())
    gen = synth.lsh_codes_torch if a.codes == "lsh" else synth.uniform_codes_torch
    codes = gen(a.n, a.q, 0, dev)
    queries = gen(a.nq, a.q, 1, dev)
    m = a.m or mih_suggest_m(a.q, a.n)
    index = mih_build(codes, a.q, m)
    prof = search_profile(index, queries, a.ks)
    prof["codes"] = a.codes
    print(json.dumps(prof))
    index.free()


if __name__ == "__main__":
    main()
