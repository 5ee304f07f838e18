"""Full-size sampled parity: the benchmark's configurations (1e9 codes, 10^4
queries in one call, the default graph executor) checked against the oracle
on a few queries spread over the batch, which the oracle answers over all 1e9
codes.  The linear scan is checked on the same queries.  Collected after the
other GPU tests (a minute or two per case: generation, build, and the oracle's
pass over 16 GB of codes)."""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N, NQ, SAMPLE = 1_000_000_000, 10_000, 6


@pytest.mark.parametrize("kind,q,m,k", [("lsh", 128, 4, 100), ("uniform", 64, 3, "kper")])
def test_full_size_sampled_parity(gpu_lib, orc, kind, q, m, k):
    import torch

    from paper_1307_2982_gb300 import synth

    mih = gpu_lib
    dev = torch.device("cuda", 0)
    gen = synth.lsh_codes_torch if kind == "lsh" else synth.uniform_codes_torch
    codes = gen(N, q, 0, device=dev)
    queries = gen(NQ, q, 1, device=dev)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    ix = mih.mih_build(codes, q, m)
    rows = np.linspace(0, NQ - 1, SAMPLE).astype(np.int64)
    if k == "kper":
        kq = synth.per_query_k(NQ, seed=3, kmax=1000).astype(np.uint32)
        r = mih.mih_knn(ix, queries, torch.from_numpy(kq.astype(np.int32)).to(dev))
        off = r["offsets"].cpu().numpy()
        got = [(r["ids"][off[i]:off[i + 1]].cpu().numpy().view(np.uint32),
                r["dist"][off[i]:off[i + 1]].cpu().numpy()) for i in rows]
        ksample = kq[rows]
    else:
        r = mih.mih_knn(ix, queries, k)
        got = [(r["ids"][i].cpu().numpy().view(np.uint32), r["dist"][i].cpu().numpy()) for i in rows]
        ksample = k
    qsel = queries[torch.from_numpy(rows).to(dev)].contiguous()
    ls = mih.linscan_knn(codes, q, qsel, torch.from_numpy(np.asarray(ksample, dtype=np.int32)).to(dev)
                         if k == "kper" else k)
    torch.cuda.synchronize()
    ix.free()
    db = codes.cpu().numpy().view(np.uint64)
    qs = qsel.cpu().numpy().view(np.uint64)
    del codes, queries
    torch.cuda.empty_cache()
    res = orc.knn(db, qs, ksample, nthreads=min(orc.default_threads(), SAMPLE))
    if k == "kper":
        woff, wids, wdist = res
        lsoff = ls["offsets"].cpu().numpy()
        for s in range(SAMPLE):
            want = (wids[woff[s]:woff[s + 1]], wdist[woff[s]:woff[s + 1]])
            assert np.array_equal(got[s][0], want[0]) and np.array_equal(got[s][1], want[1]), s
            assert np.array_equal(ls["ids"][lsoff[s]:lsoff[s + 1]].cpu().numpy().view(np.uint32), want[0]), s
    else:
        wids, wdist = res
        for s in range(SAMPLE):
            assert np.array_equal(got[s][0], wids[s]) and np.array_equal(got[s][1], wdist[s]), s
        assert np.array_equal(ls["ids"].cpu().numpy().view(np.uint32), wids)
        assert np.array_equal(ls["dist"].cpu().numpy(), wdist)
    del db
