"""Radius / lookup diagnostics (Fig. 3 and Fig. 9 analogues): the single-table
lookup count is Eq. 1, and the radii are the oracle's k-th distances."""
import math

import numpy as np
import pytest

from paper_1307_2982_gb300 import synth


def test_sht_lookups_is_the_hamming_ball():
    from paper_1307_2982_gb300.diagnostics import sht_lookups_log10

    for q in (64, 128, 256):
        for r in (0, 1, 5, 20, q):
            want = math.log10(sum(math.comb(q, d) for d in range(r + 1)))
            assert abs(sht_lookups_log10(q, np.array([r]))[0] - want) < 1e-12
        assert abs(sht_lookups_log10(q, np.array([q]))[0] - q * math.log10(2)) < 1e-9


@pytest.mark.gpu
def test_profile_radii_are_oracle_kth_distances(gpu_lib, orc):
    import torch

    from paper_1307_2982_gb300.diagnostics import search_profile

    mih = gpu_lib
    q, n = 128, 50_000
    db, qs = synth.lsh_codes(n, q, 0), synth.lsh_codes(64, q, 1)
    codes = torch.from_numpy(db.view(np.int64)).cuda()
    queries = torch.from_numpy(qs.view(np.int64)).cuda()
    ix = mih.mih_build(codes, q, 4)
    prof = search_profile(ix, queries, [1, 10, 100])
    for k in (1, 10, 100):
        _, want_dist = orc.knn(db, qs, k)
        radius = want_dist[:, k - 1]
        hist = np.bincount(radius, minlength=q + 1)
        got = prof["per_k"][str(k)]
        assert got["radius_hist"] == {str(d): int(c) for d, c in enumerate(hist) if c}
        assert abs(got["radius_mean"] - radius.mean()) < 1e-9
        assert got["linear_scan_comparisons"] == n
        assert got["mih_lookups_mean"] > 0
    ix.free()


@pytest.mark.gpu
def test_rerank_recall_matches_oracle_lists(gpu_lib, orc):
    """rerank_recall's recall figures equal those of the oracle's Hamming
    lists and the oracle's re-ranking of them, scored against the same
    Euclidean ground truth (fp32 exhaustive search of the generator's
    vectors)."""
    import torch

    from paper_1307_2982_gb300.diagnostics import rerank_recall

    n, nq, q, k, seed = 20_000, 40, 128, 10, 90
    out = rerank_recall(n=n, nq=nq, q=q, m=4, k=k, candidates=(10, 50), tops=(1, 10), seed=seed)
    dev = torch.device("cuda", 0)
    codes, _, x = synth.lsh_vectors_torch(n, q, seed, device=dev)
    qc, qproj, qx = synth.lsh_vectors_torch(nq, q, seed + 1, device=dev)
    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    d2 = (x * x).sum(dim=1)[None, :] - 2.0 * (qx @ x.T)
    torch.backends.cuda.matmul.allow_tf32 = tf32
    truth = torch.topk(d2, k, dim=1, largest=False, sorted=True).indices.cpu().numpy()
    db = codes.cpu().numpy().view(np.uint64)
    qs = qc.cpu().numpy().view(np.uint64)
    proj = qproj.cpu().numpy()
    ham50, _ = orc.knn(db, qs, 50)
    asym10, _ = orc.rerank_asym(db, proj, ham50, 10)
    for t in (1, 10):
        want_h = np.mean([truth[i, 0] in ham50[i, :t] for i in range(nq)])
        want_a = np.mean([truth[i, 0] in asym10[i, :t] for i in range(nq)])
        assert out["nn1_in_top"][str(t)]["hamming"] == pytest.approx(want_h)
        assert out["nn1_in_top"][str(t)]["asymmetric"] == pytest.approx(want_a)
    for c in (10, 50):
        hc, _ = orc.knn(db, qs, c)
        rc, _ = orc.rerank_asym(db, proj, hc, k)
        want = np.mean([len(set(rc[i].tolist()) & set(truth[i].tolist())) for i in range(nq)]) / k
        assert out["recall_knn"][str(c)] == pytest.approx(want)
