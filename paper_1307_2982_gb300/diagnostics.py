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

``rerank_recall`` measures what the re-ranking phase of Sec. 5.1 buys: the
recall of the Euclidean k-NN of the vectors behind LSH-style codes, for the
Hamming k-NN and for longer Hamming lists re-ranked by the asymmetric
distance (``mih_rerank_asym``) to k.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import mih_build, mih_knn, mih_rerank_asym, mih_suggest_m


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


def rerank_recall(n: int = 1_000_000, nq: int = 1000, q: int = 128, m: int = 4, k: int = 10,
                  candidates=(10, 100, 1000), tops=(1, 10, 100), seed: int = 60, device="cuda") -> dict:
    """What the re-ranking phase buys, against the Euclidean neighbours of the
    LSH generator's vectors (ground truth by an exhaustive fp32 search,
    evaluation only):

    - ``nn1_in_top``: the fraction of queries whose Euclidean nearest
      neighbour is among the first t results, for t in `tops`, in the
      Hamming order (the first t of mih_knn's max(candidates)-NN) and after
      re-ranking that list by the asymmetric distance (the measure of Fig. 5,
      recall of the nearest neighbour against the number retrieved);
    - ``recall_knn``: recall@k of the Euclidean k-NN for the Hamming c-NN of
      each c in `candidates`, re-ranked to k (c = k is the Hamming k-NN: the
      re-ranking reorders it but keeps its set)."""
    import torch

    from . import synth

    dev = torch.device(device)
    codes, _, x = synth.lsh_vectors_torch(n, q, seed, device=dev)
    qc, qproj, qx = synth.lsh_vectors_torch(nq, q, seed + 1, device=dev)
    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    xn = (x * x).sum(dim=1)
    truth = []
    for s in range(0, nq, 100):
        d2 = xn[None, :] - 2.0 * (qx[s:s + 100] @ x.T)
        truth.append(torch.topk(d2, k, dim=1, largest=False, sorted=True).indices)
        del d2
    torch.backends.cuda.matmul.allow_tf32 = tf32
    truth = torch.cat(truth).cpu().numpy()
    del x, xn, qx
    index = mih_build(codes, q, m)
    out = {"n": n, "queries": nq, "q": q, "m": m, "codes": "lsh-style (synthetic Gaussian mixture)",
           "truth": "Euclidean neighbours of the 128-d vectors", "nn1_in_top": {}, "recall_knn": {"k": k}}
    cmax = max(candidates)
    r = mih_knn(index, qc, cmax)
    ham = r["ids"].cpu().numpy()
    asym = mih_rerank_asym(codes, q, qproj, r["ids"], max(tops))["ids"].cpu().numpy()
    nn1 = truth[:, 0]
    for t in tops:
        out["nn1_in_top"][str(t)] = {
            "hamming": float(np.mean([nn1[i] in ham[i, :t] for i in range(nq)])),
            "asymmetric": float(np.mean([nn1[i] in asym[i, :t] for i in range(nq)])),
            "list": cmax}
    for c in candidates:
        rc = mih_knn(index, qc, int(c))
        got = mih_rerank_asym(codes, q, qproj, rc["ids"], k)["ids"].cpu().numpy()
        hits = [len(set(got[i].tolist()) & set(truth[i].tolist())) for i in range(nq)]
        out["recall_knn"][str(c)] = float(np.mean(hits)) / k
    index.free()
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
