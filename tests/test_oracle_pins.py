"""Pins for the CPU oracle, checked against things other than the oracle itself.

- brute force in numpy (bit unpacking, lexicographic sort) on tiny inputs;
- the closed form of Eq. 1 (size of a Hamming ball) for the ring enumeration;
- Propositions 1 and 2 (Sec. 2.1), exhaustively for 10-bit codes;
- the Alg. 3 stop step, lookup and candidate counts, derived independently;
- special cases: r < m (Sec. 2.1), m = 1 (Sec. 5.4), m = q (Sec. 2.2);
- values the paper prints (tests/golden/paper_values.txt).
"""
import os
from math import comb, floor, log2, log10

import numpy as np
import pytest

from paper_1307_2982_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def golden(name):
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].split()
            if line and line[0] == name:
                rows.append([float(x) if "." in x else int(x) for x in line[1:]])
    return rows


# ---------------------------------------------------------------- brute force
def unpack(codes):
    """(n, W) uint64 -> (n, 64 W) uint8 bits, bit b of word w at column 64 w + b."""
    codes = np.ascontiguousarray(codes, dtype=np.uint64)
    by = codes.view(np.uint8).reshape(codes.shape[0], -1)
    return np.unpackbits(by, axis=1, bitorder="little")


def bf_dist(codes, g):
    return (unpack(codes) != unpack(g.reshape(1, -1))).sum(axis=1).astype(np.int64)


def bf_knn(codes, g, k):
    d = bf_dist(codes, g)
    order = np.lexsort((np.arange(len(d)), d))[:k]
    ids = np.full(k, 0xFFFFFFFF, dtype=np.uint32)
    dist = np.full(k, -1, dtype=np.int32)
    ids[: len(order)] = order
    dist[: len(order)] = d[order]
    return ids, dist


def bf_substring_dist(codes, g, off, ln):
    bits = unpack(codes)
    gb = unpack(g.reshape(1, -1))
    return np.stack([(bits[:, o:o + l] != gb[:, o:o + l]).sum(axis=1) for o, l in zip(off, ln)], axis=1)


def perturb(codes, flips, seed):
    """Copies of `codes` with `flips` random bits flipped in each."""
    rng = np.random.default_rng(seed)
    bits = unpack(codes)
    for i in range(len(bits)):
        bits[i, rng.choice(bits.shape[1], size=flips, replace=False)] ^= 1
    return np.packbits(bits, axis=1, bitorder="little").view(np.uint64).reshape(len(bits), -1)


def tie_heavy(n, q, seed):
    pool = synth.uniform_codes(20, q, seed + 100)
    idx = np.random.default_rng(seed).integers(0, len(pool), n)
    return pool[idx]


def near_codes(n, q, seed, flips=3):
    """Codes clustered around a few centres: few bits flipped per code."""
    rng = np.random.default_rng(seed)
    base = synth.uniform_codes(4, q, seed + 7)[rng.integers(0, 4, n)].copy()
    bits = unpack(base)
    for i in range(n):
        pos = rng.choice(q, size=rng.integers(0, flips + 1), replace=False)
        bits[i, pos] ^= 1
    return np.packbits(bits, axis=1, bitorder="little").view(np.uint64).reshape(n, -1)


# ------------------------------------------------------------------- Hamming
@pytest.mark.parametrize("q", [64, 128, 256])
def test_hamming_matches_bit_count(orc, q):
    a = synth.uniform_codes(50, q, 1)
    b = synth.uniform_codes(50, q, 2)
    for i in range(50):
        assert orc.hamming(a[i], b[i]) == int((unpack(a[i:i + 1]) != unpack(b[i:i + 1])).sum())
    assert orc.hamming(a[0], a[0]) == 0
    assert orc.hamming(a[0], ~a[0]) == q


# -------------------------------------------------------- substring layout
def test_layout_golden(orc):
    for row in golden("layout"):
        q, m, lens = row[0], row[1], row[2:]
        off, ln = orc.substring_layout(q, m)
        assert list(ln) == lens


@pytest.mark.parametrize("q", [10, 64, 128, 256])
def test_layout_partition(orc, q):
    for m in range(1, q + 1):
        off, ln = orc.substring_layout(q, m)
        assert ln.sum() == q and off[0] == 0
        assert np.all(off[1:] == off[:-1] + ln[:-1])          # contiguous, disjoint
        assert set(ln.tolist()) <= {q // m, -(-q // m)}         # Sec. 2.1 footnote


@pytest.mark.parametrize("q", [64, 128, 256])
def test_substring_keys_bitwise(orc, q):
    codes = synth.uniform_codes(200, q, 5)
    bits = unpack(codes)
    for off, ln in [(0, 16), (21, 21), (42, 22), (56, 8), (q - 32, 32), (q - 1, 1)]:
        want = (bits[:, off:off + ln].astype(np.uint64) << np.arange(ln, dtype=np.uint64)).sum(
            axis=1, dtype=np.uint64)
        assert np.array_equal(orc.substring_keys(codes, off, ln), want)


# ----------------------------------------------------------------- k-NN
CASES = [
    ("uniform", 64, 1500), ("uniform", 128, 1000), ("uniform", 256, 700),
    ("ties", 64, 1200), ("ties", 256, 600), ("near", 128, 800),
]


def make_db(kind, q, n, seed):
    if kind == "uniform":
        return synth.uniform_codes(n, q, seed)
    if kind == "ties":
        return tie_heavy(n, q, seed)
    return near_codes(n, q, seed)


@pytest.mark.parametrize("kind,q,n", CASES)
def test_knn_matches_bruteforce(orc, kind, q, n):
    db = make_db(kind, q, n, 11)
    qs = np.concatenate([make_db(kind, q, 12, 12), db[:3]])      # includes exact hits
    for k in [1, 7, 100, n, n + 13]:
        ids, dist = orc.knn(db, qs, k)
        for i in range(len(qs)):
            wi, wd = bf_knn(db, qs[i], k)
            assert np.array_equal(ids[i], wi) and np.array_equal(dist[i], wd), (k, i)


def test_knn_all_equal_and_tiny(orc):
    q = 128
    one = synth.uniform_codes(1, q, 3)
    db = np.repeat(one, 300, axis=0)
    ids, dist = orc.knn(db, one, 10)
    assert list(ids[0]) == list(range(10)) and set(dist[0]) == {0}
    ids, dist = orc.knn(db[:1], synth.uniform_codes(2, q, 4), 4)
    assert np.array_equal(ids[:, 1:], np.full((2, 3), 0xFFFFFFFF, np.uint32))
    assert np.all(dist[:, 1:] == -1)
    ids, dist = orc.knn(db[:0], one, 3)                           # empty database
    assert np.all(ids == 0xFFFFFFFF) and np.all(dist == -1)


def test_knn_per_query_k(orc):
    db = synth.uniform_codes(900, 64, 21)
    qs = synth.uniform_codes(40, 64, 22)
    ks = synth.per_query_k(40, seed=3, kmax=200)
    off, ids, dist = orc.knn(db, qs, ks)
    for i in range(40):
        wi, wd = bf_knn(db, qs[i], int(ks[i]))
        assert np.array_equal(ids[off[i]:off[i + 1]], wi)
        assert np.array_equal(dist[off[i]:off[i + 1]], wd)


@pytest.mark.parametrize("q", [64, 256])
def test_rnear_matches_bruteforce(orc, q):
    db = near_codes(700, q, 31, flips=12)
    qs = np.concatenate([near_codes(6, q, 32, flips=12), db[:2]])
    for r in [0, 3, 10, q // 2, q, q + 4]:
        off, ids, dist = orc.rnear(db, qs, r)
        for i in range(len(qs)):
            d = bf_dist(db, qs[i])
            sel = np.nonzero(d <= r)[0]
            order = sel[np.lexsort((sel, d[sel]))]
            assert np.array_equal(ids[off[i]:off[i + 1]], order)
            assert np.array_equal(dist[off[i]:off[i + 1]], d[order])
        if r >= q:
            assert np.all(np.diff(off) == len(db))                  # r >= q: everything


# -------------------------------------------------------------- Algorithm 1
def test_table_build(orc):
    q, n = 64, 5000
    codes = synth.uniform_codes(n, q, 41)
    for off, ln in [(0, 12), (12, 20), (40, 24)]:
        keys, ids = orc.table_build(codes, off, ln)
        assert np.array_equal(np.sort(ids), np.arange(n))            # each id once
        bits = unpack(codes)
        want = (bits[:, off:off + ln].astype(np.uint64) << np.arange(ln, dtype=np.uint64)).sum(
            axis=1, dtype=np.uint64)
        assert np.array_equal(keys, want[ids])                       # key of each entry
        assert np.all((keys[1:] > keys[:-1]) | ((keys[1:] == keys[:-1]) & (ids[1:] > ids[:-1])))
        # uniform codes: distinct buckets = 2^s (1 - (1 - 2^-s)^n) in expectation (Sec. 3)
        exp = 2**ln * (1 - (1 - 2.0**-ln) ** n)
        assert abs(len(np.unique(keys)) - exp) < 6 * np.sqrt(exp) + 5


# --------------------------------------------------------- rings and Eq. 1
def test_ring_closed_form(orc):
    for s in range(0, 21):
        total = 0
        for rho in range(0, s + 2):
            x = orc.ring(s, rho)
            assert len(x) == (comb(s, rho) if rho <= s else 0)
            if len(x):
                assert np.all(np.diff(x.astype(np.int64)) > 0)
                assert np.all(np.array([bin(int(v)).count("1") for v in x]) == rho)
                assert int(x.max()) < 2**s
            total += len(x)
            assert total == sum(comb(s, z) for z in range(0, min(rho, s) + 1))   # Eq. 1


def test_ball_size_golden():
    (q, r, lg), = golden("ball_log10")
    L = sum(comb(q, z) for z in range(r + 1))                        # Eq. 1
    assert round(log10(L)) == lg


# ------------------------------------------------- Propositions 1 and 2
def test_propositions_exhaustive_10bit(orc):
    q = 10
    x = np.arange(2**q, dtype=np.uint64)
    pc = np.array([bin(v).count("1") for v in range(2**q)])
    for m in range(1, q + 1):
        off, ln = orc.substring_layout(q, m)
        sub = np.stack([np.array([bin((int(v) >> int(o)) & ((1 << int(l)) - 1)).count("1")
                                  for v in x]) for o, l in zip(off, ln)], axis=1)
        for r in range(0, q + 1):
            rp, a = r // m, r - m * (r // m)
            within = pc <= r
            p1 = (sub <= rp).any(axis=1)
            p2 = (sub[:, :a + 1] <= rp).any(axis=1) | (sub[:, a + 1:] <= rp - 1).any(axis=1)
            assert np.all(p1[within]) and np.all(p2[within]), (m, r)
            if r < m:                                                 # Sec. 2.1 special case
                assert np.all((sub[:, :r + 1] == 0).any(axis=1)[within])


# partitions of 10 bits into m contiguous substrings of unequal lengths
UNEVEN_10 = [[7, 3], [1, 9], [2, 5, 3], [1, 1, 8], [4, 1, 1, 4], [3, 3, 2, 1, 1], [1, 2, 3, 4]]


def test_propositions_exhaustive_10bit_uneven():
    """Props 1 and 2 for substrings of unequal lengths (any disjoint partition)."""
    q = 10
    x = np.arange(2**q)
    pc = np.array([bin(v).count("1") for v in range(2**q)])
    for ln in UNEVEN_10:
        m = len(ln)
        off = np.concatenate([[0], np.cumsum(ln)[:-1]])
        sub = np.stack([np.array([bin((int(v) >> int(o)) & ((1 << int(l)) - 1)).count("1") for v in x])
                        for o, l in zip(off, ln)], axis=1)
        for r in range(0, q + 1):
            rp, a = r // m, r - m * (r // m)
            within = pc <= r
            assert np.all((sub <= rp).any(axis=1)[within]), (ln, r)
            p2 = (sub[:, :a + 1] <= rp).any(axis=1) | (sub[:, a + 1:] <= rp - 1).any(axis=1)
            assert np.all(p2[within]), (ln, r)


def test_alg2_exhaustive_10bit_uneven(orc):
    """Algorithm 2 with per-table lengths on the complete 10-bit space equals the definition."""
    q = 10
    db = np.arange(2**q, dtype=np.uint64).reshape(-1, 1)
    qs = np.array([[0], [0b1011001110], [1023], [0b0000011111]], dtype=np.uint64)
    for ln in UNEVEN_10:
        mo = orc.MihOracle(db, q, len(ln), lengths=ln)
        assert list(mo.off) == list(np.concatenate([[0], np.cumsum(ln)[:-1]]))
        for r in range(0, q + 1):
            off, wid, wd = orc.rnear(db, qs, r)
            for i in range(len(qs)):
                ids, dist, cnt = mo.rnear(qs[i], r)
                assert np.array_equal(ids, wid[off[i]:off[i + 1]]), (ln, r, i)
                assert np.array_equal(dist, wd[off[i]:off[i + 1]])


@pytest.mark.parametrize("kind,q,ln,n", [
    ("near", 64, [40, 24], 2000), ("uniform", 64, [10, 22, 32], 2500), ("ties", 128, [32, 32, 16, 24, 24], 1500),
    ("near", 128, [20, 30, 26, 26, 26], 1500), ("near", 256, [32, 28, 28, 28, 28, 28, 28, 28, 28], 1000),
])
def test_alg3_uneven_lengths_equals_definition(orc, kind, q, ln, n):
    """Algorithm 3 with per-table lengths: results are the definition's and the
    counters match the independent derivation over the same partition."""
    m = len(ln)
    db = make_db(kind, q, n, 61)
    fresh = make_db(kind, q, 5, 62) if kind != "ties" else perturb(db[5:10], 6, 62)
    qs = np.concatenate([fresh, db[:2]])
    mo = orc.MihOracle(db, q, m, lengths=ln)
    off = np.concatenate([[0], np.cumsum(ln)[:-1]])
    checked = 0
    for k in [1, 10, 100]:
        wid, wd = orc.knn(db, qs, k)
        for i in range(len(qs)):
            dk = int(wd[i][min(k, n) - 1])
            want = alg3_expected_counts(db, qs[i], q, m, off, ln, dk)
            if want[0] > LOOKUP_BUDGET:
                continue
            ids, dist, cnt = mo.knn(qs[i], k)
            assert np.array_equal(ids, wid[i]) and np.array_equal(dist, wd[i]), (k, i)
            assert cnt[3] == dk and tuple(cnt[:3]) == want, (k, i, cnt, want)
            checked += 1
    assert checked >= 6


def test_oracle_rejects_bad_lengths(orc):
    db = synth.uniform_codes(10, 64, 0)
    for ln in ([32, 31], [64, 0], [33, 31, 0]):
        with pytest.raises(ValueError):
            orc.MihOracle(db, 64, len(ln), lengths=ln)


def test_prop1_golden_examples(orc):
    rng = np.random.default_rng(5)
    for r, m, rp in golden("prop1_example"):
        assert r // m == rp
        off, ln = orc.substring_layout(64, m)
        for _ in range(2000):
            pos = rng.choice(64, size=r, replace=False)
            sub = [sum(1 for p in pos if o <= p < o + l) for o, l in zip(off, ln)]
            assert min(sub) <= rp


# ------------------------------------------------ Algorithms 2 and 3 (MIH)
def test_alg2_exhaustive_10bit(orc):
    """Algorithm 2 on the complete 10-bit code space equals the definition."""
    q = 10
    db = np.arange(2**q, dtype=np.uint64).reshape(-1, 1)
    qs = np.array([[0], [0b1011001110], [1023], [0b0000011111]], dtype=np.uint64)
    for m in [1, 2, 3, 4, 5, 7, 10]:
        mo = orc.MihOracle(db, q, m)
        for r in range(0, q + 1):
            off, wid, wd = orc.rnear(db, qs, r)
            for i in range(len(qs)):
                ids, dist, cnt = mo.rnear(qs[i], r)
                assert np.array_equal(ids, wid[off[i]:off[i + 1]]), (m, r, i)
                assert np.array_equal(dist, wd[off[i]:off[i + 1]])
                if r < m:                                             # r+1 exact lookups
                    assert cnt[0] == r + 1


LOOKUP_BUDGET = 2_000_000


def alg3_expected_counts(codes, g, q, m, off, ln, dk):
    """Independent derivation of the Alg. 3 counters when it stops at step dk."""
    sd = bf_substring_dist(codes, g, off, ln)                        # (n, m)
    steps = [(t % m, t // m) for t in range(dk + 1)]
    lookups = sum(comb(int(ln[j]), rho) if rho <= ln[j] else 0 for j, rho in steps)
    raw = sum(int((sd[:, j] == rho).sum()) for j, rho in steps)
    first = (m * sd + np.arange(m)).min(axis=1)                      # first step finding i
    unique = int((first <= dk).sum())
    return lookups, raw, unique


@pytest.mark.parametrize("kind,q,m,n", [
    ("uniform", 64, 4, 3000), ("near", 64, 3, 2000), ("ties", 128, 6, 1500),
    ("near", 64, 1, 800), ("uniform", 64, 64, 400), ("near", 256, 9, 1000),
])
def test_alg3_equals_definition(orc, kind, q, m, n):
    db = make_db(kind, q, n, 51)
    fresh = make_db(kind, q, 5, 52) if kind != "ties" else perturb(db[5:10], 6, 52)
    qs = np.concatenate([fresh, db[:2]])
    mo = orc.MihOracle(db, q, m)
    off, ln = orc.substring_layout(q, m)
    checked = 0
    for k in [1, 10, 100, n + 5]:
        wid, wd = orc.knn(db, qs, k)
        for i in range(len(qs)):
            dk = int(wd[i][min(k, n) - 1])                           # k-th distance
            want = alg3_expected_counts(db, qs[i], q, m, off, ln, dk)
            if want[0] > LOOKUP_BUDGET:                              # keep the CPU suite short
                continue
            ids, dist, cnt = mo.knn(qs[i], k)
            assert np.array_equal(ids, wid[i]) and np.array_equal(dist, wd[i]), (k, i)
            assert cnt[3] == dk                                      # stops at step d_k
            assert tuple(cnt[:3]) == want
            checked += 1
            if m == 1:                                               # single table = the ball
                assert cnt[2] == int((bf_dist(db, qs[i]) <= dk).sum())
    assert checked >= 6


# ------------------------------------------------------ paper's numbers
def test_memory_formula_golden():
    for q, m, s, gb in golden("memory_gb"):
        n = 10**9
        total = m * 2 ** (s - 5) * 24 + 4 * m * min(n, 2**s) + 4 * m * n + n * m * s / 8
        assert round(total / 2**30) == gb                             # Sec. 6


def test_table4_heuristic_golden():
    for q, n, v in golden("table4_q_over_log2n"):
        assert abs(q / log2(n) - v) < 0.006                           # Table 4


def test_generators_seeded():
    a = synth.uniform_codes(1000, 128, 0)
    assert np.array_equal(a, synth.uniform_codes(1000, 128, 0))
    frac = unpack(a).mean()
    assert abs(frac - 0.5) < 0.01
    l1 = synth.lsh_codes(2000, 128, 1)
    assert np.array_equal(l1, synth.lsh_codes(2000, 128, 1))
    assert abs(unpack(l1).mean() - 0.5) < 0.1
    ks = synth.per_query_k(10000)
    assert ks.min() >= 1 and ks.max() <= 1000
    assert abs(np.median(np.log(ks)) - np.log(1001) / 2) < 0.2
    _ = floor  # noqa


# ------------------------------------------- asymmetric re-ranking (reading c17)
PAD = 0xFFFFFFFF


def _rerank_inputs(q, nq, n, k_in, seed):
    rng = np.random.default_rng(seed)
    codes = synth.uniform_codes(n, q, seed)
    ids = np.stack([rng.choice(n, size=k_in, replace=False) for _ in range(nq)]).astype(np.uint32)
    return rng, codes, ids


def _expected_rerank(codes, y, ids, k, weights):
    """Brute force: disagreement bits of each candidate against the query's
    sign bits, dotted with `weights` (exact integers here), lexsort by
    (distance, id)."""
    bits = unpack(codes)
    out_ids = np.full((len(ids), k), PAD, dtype=np.uint32)
    out_a = np.full((len(ids), k), -1.0)
    for i, row in enumerate(ids):
        valid = row[row != PAD].astype(np.int64)
        dis = bits[valid] != (y[i] > 0)[None, :]
        a = dis.astype(np.int64) @ weights
        order = np.lexsort((valid, a))[:k]
        out_ids[i, : len(order)] = valid[order]
        out_a[i, : len(order)] = a[order]
    return out_ids, out_a


@pytest.mark.parametrize("q", [64, 128, 256])
def test_rerank_asym_integer_weights(orc, q):
    """|y_b| = b + 1 with random signs: the weights lie on the grid, so the
    distance equals the integer dot product of the disagreement bits
    with (1, ..., q) -- a wrong bit index, sign test or dropped term changes
    it -- and the order is numpy's lexsort of (distance, id).  Row 0 has
    padding inside it and fewer valid candidates than k."""
    rng, codes, ids = _rerank_inputs(q, 6, 300, 40, q)
    ids[0, 7:12] = PAD
    y = (rng.choice([-1.0, 1.0], size=(6, q)) * np.arange(1, q + 1)).astype(np.float32)
    k = 38
    got_ids, got_a = orc.rerank_asym(codes, y, ids, k)
    exp_ids, exp_a = _expected_rerank(codes, y, ids, k, np.arange(1, q + 1, dtype=np.int64))
    assert np.array_equal(got_ids, exp_ids)
    assert np.array_equal(got_a, exp_a)
    assert (got_ids[0, 35:] == PAD).all() and (got_a[0, 35:] == -1.0).all()


def test_rerank_asym_unit_weights_is_hamming_knn(orc):
    """|y_b| = 1: the asymmetric distance is the Hamming distance to the
    query's sign code, so the re-ranked list is the k-NN (Sec. 1.1) of that
    code among the candidates, as the brute-force k-NN gives it."""
    q, k = 128, 25
    rng, codes, ids = _rerank_inputs(q, 4, 500, 60, 11)
    y = rng.choice([-1.0, 1.0], size=(4, q)).astype(np.float32)
    got_ids, got_a = orc.rerank_asym(codes, y, ids, k)
    for i in range(4):
        cand = np.sort(ids[i].astype(np.int64))
        g = np.packbits((y[i] > 0).astype(np.uint8), bitorder="little").view(np.uint64)
        loc, dist = bf_knn(codes[cand], g, k)
        assert np.array_equal(got_ids[i], cand[loc.astype(np.int64)])
        assert np.array_equal(got_a[i], dist.astype(np.float64))


@pytest.mark.parametrize("q", [64, 256])
def test_rerank_asym_real_projections(orc, q):
    """Real projections (the LSH generator's): the distance agrees with a
    float64 matrix product of the disagreement bits with |y| to rounding, the
    list is sorted by (distance, id) and holds exactly the row's candidates."""
    codes, _ = synth.lsh_projections(2000, q, 21)
    _, y = synth.lsh_projections(5, q, 22)
    rng = np.random.default_rng(3)
    ids = np.stack([rng.choice(2000, size=300, replace=False) for _ in range(5)]).astype(np.uint32)
    got_ids, got_a = orc.rerank_asym(codes, y, ids, 300)
    bits = unpack(codes)
    for i in range(5):
        assert np.array_equal(np.sort(got_ids[i]), np.sort(ids[i]))
        dis = bits[got_ids[i].astype(np.int64)] != (y[i] > 0)[None, :]
        ref = dis.astype(np.float64) @ np.abs(y[i].astype(np.float64))
        np.testing.assert_allclose(got_a[i], ref, rtol=1e-12, atol=0)
        key = np.lexsort((got_ids[i], got_a[i]))
        assert np.array_equal(key, np.arange(300))


def test_rerank_asym_sign_flip_invariance(orc):
    """Negating y_b and flipping bit b of every code leaves each disagreement,
    each |y_b| and so each sum unchanged, bit for bit."""
    q = 128
    codes, _ = synth.lsh_projections(1000, q, 31)
    _, y = synth.lsh_projections(3, q, 32)
    rng = np.random.default_rng(4)
    ids = np.stack([rng.choice(1000, size=200, replace=False) for _ in range(3)]).astype(np.uint32)
    flip = rng.random(q) < 0.5
    mask = np.packbits(flip.astype(np.uint8), bitorder="little").view(np.uint64)
    y2 = np.where(flip[None, :], -y, y).astype(np.float32)
    a_ids, a_a = orc.rerank_asym(codes, y, ids, 50)
    b_ids, b_a = orc.rerank_asym(codes ^ mask[None, :], y2, ids, 50)
    assert np.array_equal(a_ids, b_ids) and np.array_equal(a_a, b_a)


def _permute_bits(codes, perm):
    """Code bit perm[b] moves to bit b, for every code."""
    bits = np.ascontiguousarray(unpack(codes)[:, perm])
    return np.ascontiguousarray(np.packbits(bits, axis=1, bitorder="little")).view(np.uint64)


def test_rerank_asym_sum_is_order_free(orc):
    """The sum is exact, so it does not depend on the order of the bits:
    permuting the bits of every code and the query's values the same way
    gives the same ids and distances, bit for bit (a sum rounded term by
    term would differ in the last bits)."""
    q = 256
    codes, _ = synth.lsh_projections(1500, q, 33)
    _, y = synth.lsh_projections(4, q, 34)
    rng = np.random.default_rng(8)
    ids = np.stack([rng.choice(1500, size=400, replace=False) for _ in range(4)]).astype(np.uint32)
    perm = rng.permutation(q)
    a_ids, a_a = orc.rerank_asym(codes, y, ids, 400)
    b_ids, b_a = orc.rerank_asym(_permute_bits(codes, perm), np.ascontiguousarray(y[:, perm]), ids, 400)
    assert np.array_equal(a_ids, b_ids) and np.array_equal(a_a, b_a)


def test_rerank_asym_grid(orc):
    """The fixed-point grid: with the largest |y_b| = 1.5 (binary exponent 0)
    the weights are floor(|y_b| 2^53); a weight of 2^-60 rounds to 0 and
    adds nothing, one of 3 * 2^-52 is kept exactly."""
    codes = np.array([[0], [1 << 1], [1 << 2], [(1 << 1) | (1 << 2)]], dtype=np.uint64)
    y = np.zeros((1, 64), dtype=np.float32)
    y[0, 0] = 1.5            # query bit 0 set; every code disagrees there
    y[0, 1] = 2.0 ** -60     # below the grid
    y[0, 2] = 3 * 2.0 ** -52
    ids, a = orc.rerank_asym(codes, y, np.arange(4, dtype=np.uint32)[None, :], 4)
    # the query's bits 0..2 are set: codes 2 and 3 (bit 2 set) disagree on
    # bit 0 and at most on bit 1, whose weight is 0: 1.5 exactly; codes 0
    # and 1 also disagree on bit 2: 1.5 + 3 * 2^-52 (weight 6 on the grid)
    assert ids[0].tolist() == [2, 3, 0, 1]
    assert a[0].tolist() == [1.5, 1.5, 1.5 + 3 * 2.0 ** -52, 1.5 + 3 * 2.0 ** -52]


def test_rerank_asym_edges(orc):
    codes = synth.uniform_codes(10, 64, 1)
    y = np.ones((2, 64), dtype=np.float32)
    all_pad = np.full((2, 3), PAD, dtype=np.uint32)
    ids, a = orc.rerank_asym(codes, y, all_pad, 4)
    assert (ids == PAD).all() and (a == -1.0).all()
    with pytest.raises(ValueError):
        orc.rerank_asym(codes, y, np.array([[1, 10], [2, 3]], dtype=np.uint32), 2)
    # zero weights add nothing: with y_5 = 2.5 (query bit 5 set) and every
    # other y_b = 0, a code scores 2.5 exactly when its bit 5 is clear
    y0 = np.zeros((1, 64), dtype=np.float32)
    y0[0, 5] = 2.5
    ids, a = orc.rerank_asym(codes, y0, np.arange(10, dtype=np.uint32)[None, :], 10)
    clear5 = ((codes[:, 0] >> np.uint64(5)) & np.uint64(1)) == 0
    assert np.array_equal(a[0][np.argsort(ids[0])], np.where(clear5, 2.5, 0.0))


def test_lsh_projections_are_the_codes_signs():
    codes, proj = synth.lsh_projections(500, 128, 9)
    assert np.array_equal(codes, synth.lsh_codes(500, 128, 9))
    packed = np.packbits((proj > 0).astype(np.uint8), axis=1, bitorder="little").view(np.uint64)
    assert np.array_equal(packed, codes)
