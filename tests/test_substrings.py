"""Substring optimisation (Sec. 5.5): the greedy bit assignment on the host,
the GPU bit correlation against numpy, and search results that the bit
order leaves unchanged (against the oracle, and Alg. 3's counters on the
permuted codes)."""
import numpy as np
import pytest

from paper_1307_2982_gb300 import synth


@pytest.fixture(scope="module")
def lib():
    import paper_1307_2982_gb300 as mih

    mih.build()
    mih.load()
    return mih


def unpack(codes, q):
    by = np.ascontiguousarray(codes).view(np.uint8).reshape(len(codes), -1)
    return np.unpackbits(by, axis=1, bitorder="little")[:, :q]


def permute_host(codes, order, q):
    bits = np.ascontiguousarray(unpack(codes, q)[:, order])
    packed = np.ascontiguousarray(np.packbits(bits, axis=1, bitorder="little"))
    return packed.view(np.uint64).reshape(len(codes), -1)


def substrings_of(lib, order, q, m):
    off, ln = lib.mih_substring_layout(q, m)
    return [order[o:o + l].tolist() for o, l in zip(off, ln)]


# ------------------------------------------------------------------ host
@pytest.mark.parametrize("q,m", [(64, 2), (64, 3), (128, 4), (128, 6), (256, 8), (256, 12)])
def test_greedy_is_a_layout_permutation(lib, q, m):
    rng = np.random.default_rng(q + m)
    x = rng.standard_normal((q, 3 * q))
    corr = np.corrcoef(x)
    order = lib.mih_greedy_substrings(corr, m, seed=5)
    assert sorted(order.tolist()) == list(range(q))
    subs = substrings_of(lib, order, q, m)
    assert [len(s) for s in subs] == lib.mih_substring_layout(q, m)[1]
    assert order[0] == 5 % q
    # the first bit of substring j is the unused bit most correlated with the
    # first bit of substring j - 1 (ties to the lower index)
    used = {subs[0][0]}
    for j in range(1, m):
        prev = subs[j - 1][0]
        cand = [b for b in range(q) if b not in used]
        best = max(cand, key=lambda b: (abs(corr[prev, b]), -b))
        assert subs[j][0] == best
        used.add(best)


def test_greedy_later_bits_minimise_max_correlation(lib):
    """Replays the round-robin phase on a small case from the definition."""
    q, m = 64, 4
    rng = np.random.default_rng(11)
    corr = np.corrcoef(rng.standard_normal((q, 200)))
    order = lib.mih_greedy_substrings(corr, m, seed=9)
    subs = substrings_of(lib, order, q, m)
    c = np.abs(corr)
    held = [[s[0]] for s in subs]
    used = {s[0] for s in subs}
    j = 0
    while len(used) < q:
        if len(held[j]) < len(subs[j]):
            cand = [b for b in range(q) if b not in used]
            best = min(cand, key=lambda b: (max(c[a, b] for a in held[j]), b))
            assert subs[j][len(held[j])] == best
            held[j].append(best)
            used.add(best)
        j = (j + 1) % m


def test_greedy_separates_duplicated_bits(lib):
    """Bits b and b + 64 are copies (correlation 1): no substring gets both."""
    rng = np.random.default_rng(0)
    base = rng.integers(0, 2, size=(4000, 64))
    corr = np.corrcoef(np.concatenate([base, base], axis=1).T.astype(float))
    for m in (2, 4, 5):
        subs = substrings_of(lib, lib.mih_greedy_substrings(corr, m, seed=1), 128, m)
        for s in subs:
            assert not any((b + 64) % 128 in s for b in s), m


def test_greedy_rejects_bad_arguments(lib):
    with pytest.raises(lib.MihError):
        lib.mih_greedy_substrings(np.eye(100), 4)
    with pytest.raises(lib.MihError):
        lib.mih_greedy_substrings(np.eye(64), 65)


# ------------------------------------------------------------------- GPU
def to_dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


@pytest.mark.gpu
@pytest.mark.parametrize("q", [64, 128, 256])
def test_bit_correlation_matches_numpy(lib, q):
    codes = synth.lsh_codes(20_011, q, 4)
    got = lib.mih_bit_correlation(to_dev(codes), q)
    bits = unpack(codes, q).astype(np.float64)
    want = np.corrcoef(bits.T)
    const = bits.std(axis=0) == 0
    want[const, :] = 0.0
    want[:, const] = 0.0
    np.testing.assert_allclose(got, want, atol=1e-9)


@pytest.mark.gpu
@pytest.mark.parametrize("q,m,n,inline", [(64, 3, 60_000, 0), (128, 4, 100_003, 0), (128, 5, 50_000, -1),
                                          (256, 9, 30_001, 0), (256, 8, 30_000, -1)])
def test_optimised_substrings_keep_results(lib, orc, q, m, n, inline):
    import torch

    db, qs = synth.lsh_codes(n, q, 0), synth.lsh_codes(150, q, 1)
    codes, queries = to_dev(db), to_dev(qs)
    order = lib.optimize_substrings(codes, q, m, seed=3)
    ix = lib.mih_build(codes, q, m, bit_order=order, inline_codes=inline)
    for k in (1, 50):
        want_ids, want_dist = orc.knn(db, qs, k)
        r = lib.mih_knn(ix, queries, k)
        assert np.array_equal(r["ids"].cpu().numpy().view(np.uint32), want_ids), k
        assert np.array_equal(r["dist"].cpu().numpy(), want_dist), k
    for rad in (3, q // 8):
        off, ids, dist = orc.rnear(db, qs, rad)
        r = lib.mih_rnear(ix, queries, rad)
        assert np.array_equal(r["offsets"].cpu().numpy(), off.astype(np.int64)), rad
        assert np.array_equal(r["ids"].cpu().numpy().view(np.uint32), ids), rad
        assert np.array_equal(r["dist"].cpu().numpy(), dist), rad
    kt = torch.from_numpy(synth.per_query_k(len(qs), seed=3, kmax=300).astype(np.int32)).cuda()
    r = lib.mih_knn(ix, queries, kt)
    off, want_ids, want_dist = orc.knn(db, qs, kt.cpu().numpy())
    assert np.array_equal(r["ids"].cpu().numpy().view(np.uint32), want_ids)
    ix.free()


@pytest.mark.gpu
def test_optimised_substrings_counters_are_alg3_on_permuted_codes(lib, orc):
    """With a bit order the tables hold the permuted codes' substrings: the
    work counters equal Algorithm 3 run on the host-permuted codes."""
    q, m, n = 128, 6, 20_000
    db, qs = synth.lsh_codes(n, q, 7), synth.lsh_codes(16, q, 8)
    order = lib.optimize_substrings(to_dev(db), q, m, seed=2)
    mo = orc.MihOracle(permute_host(db, order, q), q, m)
    pq = permute_host(qs, order, q)
    ix = lib.mih_build(to_dev(db), q, m, bit_order=order, scan_factor=-1)
    r = lib.mih_knn(ix, to_dev(qs), 25, query_stats=True)
    st = r["query_stats"].cpu().numpy()
    for i in range(len(qs)):
        ids, dist, cnt = mo.knn(pq[i], 25)
        assert np.array_equal(r["ids"].cpu().numpy().view(np.uint32)[i], ids)
        assert tuple(st[i]) == tuple(cnt), (i, st[i], cnt)
    ix.free()


@pytest.mark.gpu
def test_bit_order_is_validated(lib):
    codes = to_dev(synth.uniform_codes(1000, 64, 0))
    bad = np.arange(64, dtype=np.int32)
    bad[5] = 6
    with pytest.raises(lib.MihError):
        lib.mih_build(codes, 64, 4, bit_order=bad)
