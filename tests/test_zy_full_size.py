"""Full-size sampled parity: the benchmark's configurations (10^4 queries in
one call, the default graph executor) checked against the oracle on queries
spread over the batch, which the oracle answers over every code of the
database.  The linear scan is checked on the same queries.  Collected after
the other GPU tests (a minute or two per case: generation, build, and the
oracle's pass over up to 32 GB of codes).

Configurations:
- 1e9 x 128-bit LSH-style codes, k = 100, m = 4 (inline records); the
  batch's 100-NN lists are also re-ranked to 10 by the asymmetric distance
  (mih_rerank_asym) and checked against the oracle's re-ranking;
- 1e9 x 64-bit uniform codes, per-query k log-uniform in [1, 1000], m = 3;
- 1e9 x 256-bit LSH-style codes, per-query k log-uniform in [1, 1000], m = 9:
  the index keeps no inline codes (they would need 9 x 32 GB), so every
  candidate is gathered by id;
- 1e7 x 128-bit LSH-style codes, k = 100, m = 6 (21/21/21/21/22/22-bit
  substrings), 1000 of the 10^4 queries compared.
"""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NQ = 10_000
CASES = [
    # kind, q, n, m, k, sampled queries, expected inline codes
    ("lsh", 128, 1_000_000_000, 4, 100, 6, 1),
    ("uniform", 64, 1_000_000_000, 3, "kper", 6, None),
    ("lsh", 256, 1_000_000_000, 9, "kper", 6, 0),
    ("lsh", 128, 10_000_000, 6, 100, 1000, 1),
]


@pytest.mark.parametrize("kind,q,n,m,k,sample,inline", CASES)
def test_full_size_sampled_parity(gpu_lib, orc, kind, q, n, m, k, sample, inline):
    import torch

    from paper_1307_2982_gb300 import synth

    mih = gpu_lib
    dev = torch.device("cuda", 0)
    gen = synth.lsh_codes_torch if kind == "lsh" else synth.uniform_codes_torch
    codes = gen(n, q, 0, device=dev)
    queries = gen(NQ, q, 1, device=dev)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    ix = mih.mih_build(codes, q, m)
    if inline is not None:
        assert ix.info()["inline_codes"] == inline
    rows = np.linspace(0, NQ - 1, sample).astype(np.int64)
    if k == "kper":
        kq = synth.per_query_k(NQ, seed=3, kmax=1000).astype(np.uint32)
        r = mih.mih_knn(ix, queries, torch.from_numpy(kq.astype(np.int32)).to(dev))
        off = r["offsets"].cpu().numpy()
        ids_all, dist_all = r["ids"].cpu().numpy().view(np.uint32), r["dist"].cpu().numpy()
        got = [(ids_all[off[i]:off[i + 1]], dist_all[off[i]:off[i + 1]]) for i in rows]
        ksample = kq[rows]
    else:
        r = mih.mih_knn(ix, queries, k)
        ids_all, dist_all = r["ids"].cpu().numpy().view(np.uint32), r["dist"].cpu().numpy()
        got = [(ids_all[i], dist_all[i]) for i in rows]
        ksample = k
    rerank = None
    if kind == "lsh" and q == 128 and k == 100:
        # the re-ranking phase on the whole batch: 100 Hamming neighbours of
        # every query re-ranked to 10 by the asymmetric distance
        _, proj = synth.lsh_projections_torch(NQ, q, 1, device=dev)
        rr = mih.mih_rerank_asym(codes, q, proj, r["ids"], 10)
        rerank = (proj[torch.from_numpy(rows).to(dev)].cpu().numpy(),
                  rr["ids"].cpu().numpy().view(np.uint32)[rows], rr["a"].cpu().numpy()[rows])
        del proj, rr
    qsel = queries[torch.from_numpy(rows).to(dev)].contiguous()
    ls = mih.linscan_knn(codes, q, qsel, torch.from_numpy(np.asarray(ksample, dtype=np.int32)).to(dev)
                         if k == "kper" else k)
    torch.cuda.synchronize()
    ix.free()
    db = codes.cpu().numpy().view(np.uint64)
    qs = qsel.cpu().numpy().view(np.uint64)
    del codes, queries
    torch.cuda.empty_cache()
    res = orc.knn(db, qs, ksample, nthreads=min(orc.default_threads(), sample))
    if k == "kper":
        woff, wids, wdist = res
        lsoff = ls["offsets"].cpu().numpy()
        ls_ids, ls_dist = ls["ids"].cpu().numpy().view(np.uint32), ls["dist"].cpu().numpy()
        for s in range(sample):
            want = (wids[woff[s]:woff[s + 1]], wdist[woff[s]:woff[s + 1]])
            assert np.array_equal(got[s][0], want[0]) and np.array_equal(got[s][1], want[1]), s
            assert np.array_equal(ls_ids[lsoff[s]:lsoff[s + 1]], want[0]), s
            assert np.array_equal(ls_dist[lsoff[s]:lsoff[s + 1]], want[1]), s
    else:
        wids, wdist = res
        bad = [s for s in range(sample)
               if not (np.array_equal(got[s][0], wids[s]) and np.array_equal(got[s][1], wdist[s]))]
        assert not bad, bad[:10]
        assert np.array_equal(ls["ids"].cpu().numpy().view(np.uint32), wids)
        assert np.array_equal(ls["dist"].cpu().numpy(), wdist)
        if rerank is not None:
            want_ids, want_a = orc.rerank_asym(db, rerank[0], wids, 10)
            assert np.array_equal(rerank[1], want_ids) and np.array_equal(rerank[2], want_a)
    del db
