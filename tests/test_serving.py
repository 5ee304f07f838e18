"""Continuous batching: each served result equals the same query answered alone.

Three resident databases of different code lengths receive a Poisson stream
of requests with log-uniform k; requests that arrive while batches run join
later batches.  Every kept result must equal a one-query mih_knn call and the
CPU oracle.
"""
import numpy as np
import pytest

from paper_1307_2982_gb300 import synth

pytestmark = pytest.mark.gpu


def test_served_results_equal_single_calls(gpu_lib, orc):
    mih = gpu_lib
    import torch

    from paper_1307_2982_gb300 import serving

    dbs = [(64, synth.uniform_codes(50_000, 64, 0)), (128, synth.lsh_codes(100_000, 128, 0)),
           (256, synth.lsh_codes(30_000, 256, 0))]
    idx = []
    for q, db in dbs:
        t = torch.from_numpy(db.view(np.int64)).cuda()
        idx.append(mih.mih_build(t, q, mih.mih_suggest_m(q, len(db))))

    def gen(d, count, seed):
        q = dbs[d][0]
        return synth.uniform_codes(count, q, seed) if q == 64 else synth.lsh_codes(count, q, seed)

    req = serving.poisson_requests(3000, 30_000.0, [q for q, _ in dbs], k_max=300, seed=4, query_gen=gen)
    keep = list(range(0, 3000, 7))
    server = serving.MihServer(idx, result_budget=1 << 20, max_batch=512)
    res = server.run(req, keep=keep)
    s = res.summary()
    assert s["requests"] == 3000 and np.all(np.isfinite(res.latency_s)) and np.all(res.latency_s > 0)
    assert s["batches"] > 3 and s["mean_batch"] > 1          # requests were batched
    for i in keep:
        d, k = int(req.db[i]), int(req.k[i])
        q = dbs[d][0]
        g = np.ascontiguousarray(req.codes[i:i + 1, : q // 64])
        alone = mih.mih_knn(idx[d], torch.from_numpy(g.view(np.int64)).cuda(), k)
        ids, dist = res.kept[i]
        assert np.array_equal(ids, alone["ids"].cpu().numpy().view(np.uint32)[0])
        assert np.array_equal(dist, alone["dist"].cpu().numpy()[0])
        if i % 49 == 0:
            wi, wd = orc.knn(dbs[d][1], g, k)
            assert np.array_equal(ids, wi[0]) and np.array_equal(dist, wd[0])
