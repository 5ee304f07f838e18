"""Re-ranking by the asymmetric Hamming distance (Sec. 5.1 re-ranking phase,
Conclusion): the CUDA kernel against the oracle, bit for bit on ids and on
the distances (both sides sum the same fixed-point weights exactly and round
once), on ragged rows, every code length, rows sorted by one warp (up to 256
candidates) and by a CTA (up to 8192), k below and above the row length, and
after a real mih_knn.
"""
import numpy as np
import pytest

from paper_1307_2982_gb300 import synth

pytestmark = pytest.mark.gpu
PAD = 0xFFFFFFFF


def _run(mih, codes_np, proj_np, ids_np, q, k):
    import torch

    dev = torch.device("cuda", 0)
    codes = torch.from_numpy(codes_np.view(np.int64)).to(dev)
    proj = torch.from_numpy(proj_np).to(dev)
    ids = torch.from_numpy(ids_np.view(np.int32)).to(dev)
    r = mih.mih_rerank_asym(codes, q, proj, ids, k)
    return r["ids"].cpu().numpy().view(np.uint32), r["a"].cpu().numpy()


@pytest.mark.parametrize("q,n,nq,k_in,k", [
    (64, 3000, 37, 1, 1),
    (64, 3000, 37, 100, 10),
    (128, 5000, 41, 100, 100),
    (128, 5000, 9, 1000, 1005),
    (256, 5000, 23, 300, 64),
    (128, 20000, 3, 8192, 8192),
    (64, 3000, 11, 32, 40),      # one slot per lane, k past the row
    (128, 5000, 29, 33, 7),      # 64 slots
    (256, 5000, 19, 256, 300),   # 256 slots (the widest warp-per-row case), k past the row
    (128, 5000, 5, 257, 20),     # the first width sorted by a CTA
])
def test_rerank_matches_oracle(gpu_lib, orc, q, n, nq, k_in, k):
    codes, _ = synth.lsh_projections(n, q, 40 + q)
    _, proj = synth.lsh_projections(nq, q, 41 + q)
    rng = np.random.default_rng(k_in + q)
    ids = np.stack([rng.choice(n, size=k_in, replace=False) for _ in range(nq)]).astype(np.uint32)
    # ragged rows: padding at the end of some rows, in the middle of others
    for i in range(0, nq, 3):
        cut = int(rng.integers(0, k_in + 1))
        ids[i, cut:] = PAD
    for i in range(1, nq, 5):
        ids[i, rng.random(k_in) < 0.3] = PAD
    want_ids, want_a = orc.rerank_asym(codes, proj, ids, k)
    got_ids, got_a = _run(gpu_lib, codes, proj, ids, q, k)
    assert np.array_equal(got_ids, want_ids)
    assert np.array_equal(got_a, want_a)


def test_rerank_ties_and_zero_weights(gpu_lib, orc):
    """Many equal sums: a database of 8 distinct codes repeated, and a query
    with small-integer and zero weights; equal (a) are ordered by id."""
    q = 128
    base = synth.uniform_codes(8, q, 5)
    codes = np.ascontiguousarray(np.tile(base, (250, 1)))
    rng = np.random.default_rng(6)
    proj = (rng.integers(-3, 4, size=(7, q))).astype(np.float32)
    ids = np.stack([rng.permutation(2000)[:700] for _ in range(7)]).astype(np.uint32)
    want = orc.rerank_asym(codes, proj, ids, 500)
    got = _run(gpu_lib, codes, proj, ids, q, 500)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_rerank_grid_extremes(gpu_lib, orc):
    """The per-row grid at the ends of the fp32 range: an all-zero row, rows
    scaled by 1e30 and 1e-30, one with subnormal values beside normal ones,
    one with a single nonzero value, one with values far below its largest."""
    q, n = 128, 4000
    codes, _ = synth.lsh_projections(n, q, 70)
    _, base = synth.lsh_projections(6, q, 71)
    proj = base.astype(np.float64)
    proj[0] = 0.0
    proj[1] *= 1e30
    proj[2] *= 1e-30
    proj[3, ::2] *= 1e-40        # subnormal in fp32
    proj[4] = 0.0
    proj[4, 77] = -3.25
    proj[5, 1::2] *= 2.0 ** -70   # below the grid of the row's largest value
    proj = proj.astype(np.float32)
    rng = np.random.default_rng(72)
    ids = np.stack([rng.choice(n, size=500, replace=False) for _ in range(6)]).astype(np.uint32)
    want_ids, want_a = orc.rerank_asym(codes, proj, ids, 200)
    got_ids, got_a = _run(gpu_lib, codes, proj, ids, q, 200)
    assert np.array_equal(got_ids, want_ids)
    assert np.array_equal(got_a, want_a)
    assert (got_a[0] == 0.0).all()


def test_rerank_after_mih_knn(gpu_lib, orc):
    """The two calls in sequence (mih_knn_asym): the Hamming 100-NN of real
    LSH-style queries, re-ranked to 10, equals the oracle's k-NN re-ranked by
    the oracle."""
    import torch

    mih = gpu_lib
    q, n, nq = 128, 200_000, 300
    dev = torch.device("cuda", 0)
    db, _ = synth.lsh_projections(n, q, 50)
    qc, proj = synth.lsh_projections(nq, q, 51)
    codes = torch.from_numpy(db.view(np.int64)).to(dev)
    queries = torch.from_numpy(qc.view(np.int64)).to(dev)
    ix = mih.mih_build(codes, q, 4)
    r = mih.mih_knn_asym(ix, codes, queries, torch.from_numpy(proj).to(dev), 10, 100)
    ix.free()
    want_knn, _ = orc.knn(db, qc, 100)
    want_ids, want_a = orc.rerank_asym(db, proj, want_knn, 10)
    assert np.array_equal(r["ids"].cpu().numpy().view(np.uint32), want_ids)
    assert np.array_equal(r["a"].cpu().numpy(), want_a)


def test_rerank_errors(gpu_lib):
    import torch

    mih = gpu_lib
    dev = torch.device("cuda", 0)
    codes = torch.from_numpy(synth.uniform_codes(100, 64, 1).view(np.int64)).to(dev)
    proj = torch.ones((2, 64), dtype=torch.float32, device=dev)
    ok = torch.tensor([[1, 2], [3, -1]], dtype=torch.int32, device=dev)
    r = mih.mih_rerank_asym(codes, 64, proj, ok, 3)
    assert r["ids"].cpu().numpy().view(np.uint32)[1].tolist() == [3, PAD, PAD]
    assert r["a"].cpu().numpy()[1, 1:].tolist() == [-1.0, -1.0]
    bad = torch.tensor([[1, 100], [3, 4]], dtype=torch.int32, device=dev)
    with pytest.raises(mih.MihError):
        mih.mih_rerank_asym(codes, 64, proj, bad, 2)
    # the library stays usable after the rejected call
    r = mih.mih_rerank_asym(codes, 64, proj, ok, 2)
    assert r["ids"].cpu().numpy().view(np.uint32)[0].tolist() in ([1, 2], [2, 1])
    with pytest.raises(mih.MihError):
        mih.mih_rerank_asym(codes, 64, proj, ok, 0)
    empty = mih.mih_rerank_asym(codes, 64, proj[:0], ok[:0], 4)
    assert empty["ids"].shape == (0, 4)


@pytest.mark.parametrize("kmax", [100, 300])
def test_rerank_csr_after_per_query_k(gpu_lib, orc, kmax):
    """Per-query k: mih_knn's CSR answers (k log-uniform in [1, kmax]) re-ranked
    to ceil(k_i / 2) per row by mih_rerank_asym_csr, against the oracle row by
    row (kmax 100: rows sorted by one warp; 300: by a CTA)."""
    import torch

    mih = gpu_lib
    q, n, nq = 128, 100_000, 200
    dev = torch.device("cuda", 0)
    db, _ = synth.lsh_projections(n, q, 80)
    qc, proj = synth.lsh_projections(nq, q, 81)
    codes = torch.from_numpy(db.view(np.int64)).to(dev)
    queries = torch.from_numpy(qc.view(np.int64)).to(dev)
    kq = synth.per_query_k(nq, seed=5, kmax=kmax)
    ix = mih.mih_build(codes, q, 4)
    r = mih.mih_knn(ix, queries, torch.from_numpy(kq.astype(np.int32)).to(dev))
    ix.free()
    kout = (kq.astype(np.int64) + 1) // 2
    ooff = np.concatenate([[0], np.cumsum(kout)]).astype(np.int64)
    rr = mih.mih_rerank_asym_csr(codes, q, torch.from_numpy(proj).to(dev), r["ids"], r["offsets"],
                                 torch.from_numpy(ooff).to(dev))
    got_ids, got_a = rr["ids"].cpu().numpy().view(np.uint32), rr["a"].cpu().numpy()
    off = r["offsets"].cpu().numpy().astype(np.int64)
    cand = r["ids"].cpu().numpy().view(np.uint32)
    for i in range(nq):
        want_ids, want_a = orc.rerank_asym(db, proj[i:i + 1], cand[off[i]:off[i + 1]][None, :], int(kout[i]))
        assert np.array_equal(got_ids[ooff[i]:ooff[i + 1]], want_ids[0]), i
        assert np.array_equal(got_a[ooff[i]:ooff[i + 1]], want_a[0]), i
    # a row longer than the stated maximum is an error
    with pytest.raises(mih.MihError):
        mih.mih_rerank_asym_csr(codes, q, torch.from_numpy(proj).to(dev), r["ids"], r["offsets"],
                                torch.from_numpy(ooff).to(dev), k_in_max=int(kq.max()) - 1)
