"""GPU parity: the CUDA path through the C-ABI against the CPU oracle.

Everything here is integer work, so the bar is bit-exact: ids and distances
in (distance, id) order must equal the oracle's element by element.  The
MIH work counters (lookups, raw and unique candidates, last step) must equal
the oracle's step-by-step run of Algorithm 3.
"""
import numpy as np
import pytest

from paper_1307_2982_gb300 import synth

pytestmark = pytest.mark.gpu


def to_dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def host(t):
    return t.cpu().numpy()


def ids_of(t):
    return host(t).view(np.uint32)


def tie_heavy(n, q, seed, pool=40):
    p = synth.uniform_codes(pool, q, seed + 100)
    return p[np.random.default_rng(seed).integers(0, pool, n)]


def perturb(codes, flips, seed):
    rng = np.random.default_rng(seed)
    by = np.ascontiguousarray(codes).view(np.uint8).reshape(len(codes), -1)
    bits = np.unpackbits(by, axis=1, bitorder="little")
    for i in range(len(bits)):
        bits[i, rng.choice(bits.shape[1], size=flips, replace=False)] ^= 1
    return np.packbits(bits, axis=1, bitorder="little").view(np.uint64).reshape(len(codes), -1)


def planted(n, q, seed, nq, per_word, pool=8, fmin=None, fmax=None):
    """Clusters around `pool` random centres.  A database code is a centre with
    fmin..fmax random bits flipped; a query is a centre with `per_word` bits
    flipped in every 32-bit word.  So in table j (m = q/32, one word per table)
    the bucket of the centre's word holds the cluster members that kept word j
    (hundreds of codes, above the slice threshold) and lies at ring per_word
    from the query, and the k-th distance (about q/32 * per_word + fmin) keeps
    the query running until it reaches that ring in several tables."""
    rng = np.random.default_rng(seed)
    W32 = q // 32
    fmin = 1 if fmin is None else fmin
    fmax = W32 + 4 if fmax is None else fmax
    cent = synth.uniform_codes(pool, q, seed + 100)
    db = cent[rng.integers(0, pool, n)].copy()
    dw = db.view(np.uint32).reshape(n, W32)
    for i, f in enumerate(rng.integers(fmin, fmax + 1, n)):
        for b in rng.choice(q, size=f, replace=False):
            dw[i, b // 32] ^= np.uint32(1) << np.uint32(b % 32)
    qs = cent[rng.integers(0, pool, nq)].copy()
    qw = qs.view(np.uint32).reshape(nq, W32)
    for i in range(nq):
        for j in range(W32):
            for b in rng.choice(32, size=per_word, replace=False):
                qw[i, j] ^= np.uint32(1) << np.uint32(b)
    return db, qs


def workload(kind, q, n, nq, seed=0):
    if kind == "uniform":
        return synth.uniform_codes(n, q, seed), synth.uniform_codes(nq, q, seed + 1)
    if kind == "lsh":
        return synth.lsh_codes(n, q, seed), synth.lsh_codes(nq, q, seed + 1)
    db = tie_heavy(n, q, seed)
    return db, perturb(db[:nq], 3, seed + 2)


# (kind, q, n, nq, m list) -- sizes span many chunks/tiles with ragged tails
KNN_CASES = [
    ("uniform", 64, 100_000, 300, [4, 3, 2]),
    ("lsh", 128, 200_003, 257, [6, 4, 5]),
    ("lsh", 256, 60_001, 130, [9, 8, 12]),
    ("ties", 128, 30_000, 100, [4, 6]),
]


@pytest.mark.parametrize("kind,q,n,nq,ms", KNN_CASES)
def test_linscan_and_mih_knn_match_oracle(gpu_lib, orc, kind, q, n, nq, ms):
    mih = gpu_lib
    db, qs = workload(kind, q, n, nq)
    codes, queries = to_dev(db), to_dev(qs)
    indexes = {m: mih.mih_build(codes, q, m) for m in ms}
    for k in (1, 10, 100):
        want_ids, want_dist = orc.knn(db, qs, k)
        ls = mih.linscan_knn(codes, q, queries, k)
        assert np.array_equal(ids_of(ls["ids"]), want_ids), ("linscan ids", k)
        assert np.array_equal(host(ls["dist"]), want_dist), ("linscan dist", k)
        for m, ix in indexes.items():
            r = mih.mih_knn(ix, queries, k)
            assert np.array_equal(ids_of(r["ids"]), want_ids), ("mih ids", m, k)
            assert np.array_equal(host(r["dist"]), want_dist), ("mih dist", m, k)
    for ix in indexes.values():
        ix.free()


@pytest.mark.parametrize("kind,q,n,nq", [("uniform", 64, 100_003, 300), ("lsh", 128, 200_003, 257),
                                         ("lsh", 256, 60_001, 130), ("ties", 128, 30_000, 100),
                                         ("uniform", 128, 37, 9)])
@pytest.mark.parametrize("scan", [1, 2])
def test_linscan_kernels_match_oracle(gpu_lib, orc, kind, q, n, nq, scan):
    """Both forms of the linear scan (Sec. 5.2) give the definition's answer:
    xor + popcount (1) and fp8 tensor-core products of +-1 codes (2).  Ragged
    code and query counts, tie-heavy codes (the bounded buffers overflow and
    the second pass collects), k above n, per-query k."""
    import torch

    mih = gpu_lib
    db, qs = workload(kind, q, n, nq, seed=17)
    codes, queries = to_dev(db), to_dev(qs)
    try:
        mih.mih_set_scan_kernel(scan)
        for k in (1, 10, 100, 1000):
            want_ids, want_dist = orc.knn(db, qs, k)
            r = mih.linscan_knn(codes, q, queries, k)
            assert np.array_equal(ids_of(r["ids"]), want_ids), (scan, k)
            assert np.array_equal(host(r["dist"]), want_dist), (scan, k)
        ks = synth.per_query_k(nq, seed=5, kmax=300)
        off, wi, wd = orc.knn(db, qs, ks)
        r = mih.linscan_knn(codes, q, queries, torch.from_numpy(ks.astype(np.int32)).cuda())
        assert np.array_equal(ids_of(r["ids"]), wi) and np.array_equal(host(r["dist"]), wd)
    finally:
        mih.mih_set_scan_kernel(0)


@pytest.mark.parametrize("table_kind,inline", [(1, 1), (2, 1), (1, -1), (2, -1)])
def test_table_kinds_agree(gpu_lib, orc, table_kind, inline):
    """Direct and sparse tables (Sec. 6), with or without inline codes, agree."""
    mih = gpu_lib
    db, qs = workload("lsh", 128, 50_000, 64, seed=5)
    codes, queries = to_dev(db), to_dev(qs)
    ix = mih.mih_build(codes, 128, 6, table_kind=table_kind, inline_codes=inline)
    info = ix.info()
    assert set(info["table_kind"]) == {table_kind}
    assert info["inline_codes"] == (1 if inline > 0 else 0)
    assert sum(info["distinct_keys"]) > 0
    want_ids, want_dist = orc.knn(db, qs, 50)
    r = mih.mih_knn(ix, queries, 50)
    assert np.array_equal(ids_of(r["ids"]), want_ids)
    assert np.array_equal(host(r["dist"]), want_dist)


@pytest.mark.parametrize("kind,q,m,n", [("uniform", 64, 4, 20_000), ("lsh", 128, 6, 20_000),
                                        ("ties", 64, 3, 5_000), ("lsh", 256, 12, 8_000),
                                        ("ties", 128, 4, 5_000), ("ties", 64, 2, 5_000)])
def test_mih_work_counters_match_alg3(gpu_lib, orc, kind, q, m, n):
    """Per-query lookups, raw/unique candidates and last step equal Alg. 3 on the CPU.

    m = q/32 (every substring one 32-bit word, inline records without the
    table's own word) runs on tie-heavy codes: with 32-bit substrings and a
    few thousand codes the k-th distance of random queries reaches rings that
    the CPU run of Alg. 3 enumerates for minutes."""
    mih = gpu_lib
    db, qs = workload(kind, q, n, 24, seed=9)
    mo = orc.MihOracle(db, q, m)
    ixs = [mih.mih_build(to_dev(db), q, m, scan_factor=-1, inline_codes=il) for il in (1, -1)]  # Alg. 3 exactly
    for k, ix in ((1, ixs[0]), (25, ixs[0]), (25, ixs[1])):
        r = mih.mih_knn(ix, to_dev(qs), k, query_stats=True)
        st = host(r["query_stats"])
        for i in range(len(qs)):
            ids, dist, cnt = mo.knn(qs[i], k)
            assert np.array_equal(ids_of(r["ids"])[i], ids) and np.array_equal(host(r["dist"])[i], dist)
            assert tuple(st[i]) == tuple(cnt), (i, k, st[i], cnt)


@pytest.mark.parametrize("q,per_word,fmin,fmax", [(64, 3, 1, 5), (128, 3, 2, 8), (256, 2, 2, 8)])
def test_record_path_counters_reach_ring_2(gpu_lib, orc, q, per_word, fmin, fmax):
    """Alg. 3 counters of the inline-record path at rings rho >= 2.

    m = q/32: every substring is one 32-bit word, and the tables keep records
    without their own word.  A record reached at ring rho is kept only if every
    other word i differs from the query in at least rho + [i < j] bits (the
    first-discoverer reading of Sec. 6's duplicate removal).  The planted
    clusters put buckets of hundreds of codes (streamed by the slice kernel) at
    ring per_word >= 2 of every table, and the k-th distance is large enough
    that queries reach them.  Per-query lookups, raw and unique candidates and
    the last step must equal the oracle's Alg. 3; the results must equal the
    oracle with and without per-query counters."""
    mih = gpu_lib
    m = q // 32
    db, qs = planted(4000, q, 9, 24, per_word, fmin=fmin, fmax=fmax)
    queries = to_dev(qs)
    mo = orc.MihOracle(db, q, m)
    ixs = [mih.mih_build(to_dev(db), q, m, scan_factor=-1, inline_codes=il) for il in (1, -1)]
    info = ixs[0].info()
    assert info["inline_codes"] == 1 and max(info["max_bucket"]) > 64
    last = []
    for k in (1, 25):
        want_ids, want_dist = orc.knn(db, qs, k)
        for ix in ixs:
            r = mih.mih_knn(ix, queries, k, query_stats=True)
            st = host(r["query_stats"])
            for i in range(len(qs)):
                ids, dist, cnt = mo.knn(qs[i], k)
                assert np.array_equal(ids_of(r["ids"])[i], ids) and np.array_equal(host(r["dist"])[i], dist)
                assert tuple(st[i]) == tuple(cnt), (i, k, st[i], cnt)
            last.extend(int(x) for x in st[:, 3])
            fast = mih.mih_knn(ix, queries, k)
            assert np.array_equal(ids_of(fast["ids"]), want_ids) and np.array_equal(host(fast["dist"]), want_dist)
    # the last step t = m * rho + j reached ring rho >= 2
    assert max(last) >= 2 * m, max(last)
    for ix in ixs:
        ix.free()


@pytest.mark.parametrize("kind,q,m,n", [("lsh", 128, 6, 200_003), ("uniform", 64, 3, 50_000),
                                        ("lsh", 256, 9, 60_001)])
def test_graph_and_host_executors_agree(gpu_lib, orc, kind, q, m, n):
    """The wave loop as one CUDA graph (while node) and as a host loop give the
    oracle's results and the same work counters, wave for wave."""
    mih = gpu_lib
    db, qs = workload(kind, q, n, 257, seed=21)
    codes, queries = to_dev(db), to_dev(qs)
    ixg = mih.mih_build(codes, q, m, executor=mih.MIH_EXEC_GRAPH)
    ixh = mih.mih_build(codes, q, m, executor=mih.MIH_EXEC_HOST)
    for k in (1, 100):
        want_ids, want_dist = orc.knn(db, qs, k)
        for qstats in (False, True):
            rg = mih.mih_knn(ixg, queries, k, query_stats=qstats)
            rh = mih.mih_knn(ixh, queries, k, query_stats=qstats)
            for r in (rg, rh):
                assert np.array_equal(ids_of(r["ids"]), want_ids), (k, qstats)
                assert np.array_equal(host(r["dist"]), want_dist), (k, qstats)
            assert rg["stats"] == rh["stats"], (k, qstats, rg["stats"], rh["stats"])
            assert rg["stats"]["waves"] >= 1
            if qstats:
                assert np.array_equal(host(rg["query_stats"]), host(rh["query_stats"]))


@pytest.mark.parametrize("kind,q,m,n", [("lsh", 128, 4, 200_003), ("uniform", 64, 3, 80_000),
                                        ("lsh", 256, 9, 60_001), ("ties", 128, 4, 30_000)])
def test_two_step_waves_keep_results(gpu_lib, orc, kind, q, m, n):
    """Two Alg. 3 steps per wave (from step 1, or from step 2m) give the
    oracle's answer, as one step per wave (the default) does, in no more waves."""
    import torch

    mih = gpu_lib
    db, qs = workload(kind, q, n, 257, seed=23)
    codes, queries = to_dev(db), to_dev(qs)
    ks = synth.per_query_k(257, seed=6, kmax=1000)
    off, wi, wd = orc.knn(db, qs, ks)
    waves = {}
    for tail in (-1, 1, 2 * m, 0):
        ix = mih.mih_build(codes, q, m, tail_from=tail)
        r = mih.mih_knn(ix, queries, torch.from_numpy(ks.astype(np.int32)).cuda())
        assert np.array_equal(ids_of(r["ids"]), wi), tail
        assert np.array_equal(host(r["dist"]), wd), tail
        waves[tail] = r["stats"]["waves"]
        ix.free()
    assert waves[1] <= waves[-1] and waves[2 * m] <= waves[-1] and waves[0] == waves[-1], waves


def test_reused_wave_graph_across_calls(gpu_lib, orc):
    """Consecutive graph-executor calls reuse one instantiated graph per thread
    (updated in place, or instantiated again when the shape changes): calls
    that alternate code length, m and batch size each give the oracle's answer."""
    mih = gpu_lib
    db128, qs128 = workload("lsh", 128, 60_000, 300, seed=41)
    db64, qs64 = workload("uniform", 64, 40_000, 300, seed=42)
    ix128 = mih.mih_build(to_dev(db128), 128, 4, executor=mih.MIH_EXEC_GRAPH)
    ix64 = mih.mih_build(to_dev(db64), 64, 3, executor=mih.MIH_EXEC_GRAPH)
    for ix, db, qs, nq, k in ((ix128, db128, qs128, 300, 10), (ix128, db128, qs128, 300, 10),
                              (ix64, db64, qs64, 3, 7), (ix128, db128, qs128, 1, 100),
                              (ix64, db64, qs64, 300, 50), (ix128, db128, qs128, 257, 10)):
        want_ids, want_dist = orc.knn(db, qs[:nq], k)
        r = mih.mih_knn(ix, to_dev(qs[:nq]), k)
        assert np.array_equal(ids_of(r["ids"]), want_ids) and np.array_equal(host(r["dist"]), want_dist)
    ix128.free()
    ix64.free()


def test_per_query_k_and_padding(gpu_lib, orc):
    mih = gpu_lib
    import torch

    q, n, nq = 64, 3000, 200
    db, qs = workload("uniform", q, n, nq, seed=13)
    ks = synth.per_query_k(nq, seed=3, kmax=4000)          # some k > n: padded
    codes, queries = to_dev(db), to_dev(qs)
    off, want_ids, want_dist = orc.knn(db, qs, ks)
    kt = torch.from_numpy(ks.astype(np.int32)).cuda()
    ix = mih.mih_build(codes, q, 3)
    # device k (offsets by mih_k_offsets) and host k (offsets from the host values)
    for r in (mih.mih_knn(ix, queries, kt), mih.linscan_knn(codes, q, queries, kt),
              mih.mih_knn(ix, queries, ks), mih.mih_knn(ix, queries, torch.from_numpy(ks.astype(np.int32)))):
        assert np.array_equal(host(r["offsets"]), off.astype(np.int64))
        assert np.array_equal(ids_of(r["ids"]), want_ids)
        assert np.array_equal(host(r["dist"]), want_dist)


@pytest.mark.parametrize("q,m", [(64, 4), (64, 2), (128, 6), (128, 4), (256, 12), (256, 8)])
def test_rnear_matches_oracle(gpu_lib, orc, q, m):
    mih = gpu_lib
    db, qs = workload("lsh", q, 40_000, 50, seed=21)
    codes, queries = to_dev(db), to_dev(qs)
    ix = mih.mih_build(codes, q, m)
    for r in (0, 3, 9, q // 8, q // 4, q, q + 7):
        woff, wid, wd = orc.rnear(db, qs, r)
        if int(woff[-1]) > 3_000_000:
            continue
        got = mih.mih_rnear(ix, queries, r)
        assert np.array_equal(host(got["offsets"]), woff.astype(np.int64)), r
        assert np.array_equal(ids_of(got["ids"]), wid), r
        assert np.array_equal(host(got["dist"]), wd), r


def test_rnear_overflow_protocol(gpu_lib, orc):
    mih = gpu_lib
    import ctypes

    import torch

    q = 64
    db, qs = workload("uniform", q, 10_000, 20, seed=3)
    codes, queries = to_dev(db), to_dev(qs)
    ix = mih.mih_build(codes, q, 4)
    woff, wid, wd = orc.rnear(db, qs, 20)
    assert woff[-1] > 5
    off = torch.empty(21, dtype=torch.int64, device="cuda")
    ids = torch.empty(5, dtype=torch.int32, device="cuda")
    dist = torch.empty(5, dtype=torch.int32, device="cuda")
    total = ctypes.c_uint64(0)
    lib = mih.load()
    s = lib.mih_rnear(ix.handle, mih._ptr(queries), 20, 20, 5, mih._ptr(off), mih._ptr(ids), mih._ptr(dist),
                      ctypes.byref(total), None, None, mih._stream(None))
    assert s == mih.MIH_EOVERFLOW
    assert total.value == woff[-1]
    assert np.array_equal(host(off), woff.astype(np.int64))


def test_schedule_invariance(gpu_lib, orc):
    """A query alone and inside a batch gives the same bytes (any m)."""
    mih = gpu_lib
    db, qs = workload("lsh", 128, 100_000, 500, seed=31)
    codes, queries = to_dev(db), to_dev(qs)
    ixs = [mih.mih_build(codes, 128, m) for m in (4, 6)]
    batch = [mih.mih_knn(ix, queries, 30) for ix in ixs]
    for i in (0, 17, 499):
        single = mih.mih_knn(ixs[0], queries[i:i + 1], 30)
        for b in batch:
            assert np.array_equal(ids_of(single["ids"])[0], ids_of(b["ids"])[i])
            assert np.array_equal(host(single["dist"])[0], host(b["dist"])[i])


def test_edge_cases(gpu_lib, orc):
    mih = gpu_lib
    import torch

    q = 128
    db, qs = workload("uniform", q, 1000, 5, seed=41)
    codes, queries = to_dev(db), to_dev(qs)
    ix = mih.mih_build(codes, q, 4)
    # empty query batch
    r = mih.mih_knn(ix, queries[:0], 5)
    assert r["ids"].shape == (0, 5)
    # k at its maximum (> n): all n codes then padding
    want_ids, want_dist = orc.knn(db, qs, mih.MIH_MAX_K)
    for r in (mih.mih_knn(ix, queries, mih.MIH_MAX_K), mih.linscan_knn(codes, q, queries, mih.MIH_MAX_K)):
        assert np.array_equal(ids_of(r["ids"]), want_ids)
        assert np.array_equal(host(r["dist"]), want_dist)
    # one-code database, and an empty database
    one = mih.mih_build(codes[:1], q, 4)
    w1, d1 = orc.knn(db[:1], qs, 3)
    r = mih.mih_knn(one, queries, 3)
    assert np.array_equal(ids_of(r["ids"]), w1) and np.array_equal(host(r["dist"]), d1)
    empty = mih.mih_build(codes[:0], q, 4)
    r = mih.mih_knn(empty, queries, 3)
    assert np.all(ids_of(r["ids"]) == 0xFFFFFFFF) and np.all(host(r["dist"]) == -1)
    r = mih.linscan_knn(codes[:0], q, queries, 3)
    assert np.all(host(r["dist"]) == -1)
    # all-equal database: ties broken by id
    same = to_dev(np.repeat(db[:1], 5000, axis=0))
    ixs = mih.mih_build(same, q, 4)
    for r in (mih.mih_knn(ixs, queries[:2], 100), mih.linscan_knn(same, q, queries[:2], 100)):
        assert np.array_equal(ids_of(r["ids"])[0], np.arange(100, dtype=np.uint32))
    # invalid arguments are rejected with MIH_EINVAL
    for bad in (lambda: mih.mih_knn(ix, queries, 0), lambda: mih.mih_knn(ix, queries, mih.MIH_MAX_K + 1),
                lambda: mih.mih_build(codes, q, 3), lambda: mih.mih_build(codes, q, 129),
                lambda: mih.mih_rnear(ix, queries, -1)):
        with pytest.raises(mih.MihError) as e:
            bad()
        assert e.value.status == mih.MIH_EINVAL
    # host memory is refused, not dereferenced
    lib = mih.load()
    import ctypes

    h = ctypes.c_void_p()
    hostbuf = torch.zeros((10, 2), dtype=torch.int64)
    assert lib.mih_build(mih._ptr(hostbuf), 10, 128, 4, None, None, ctypes.byref(h)) == mih.MIH_EINVAL


@pytest.mark.parametrize("q", [64, 128, 256])
def test_big_buckets_streamed_and_gathered(gpu_lib, orc, q):
    """Buckets far above the slice threshold, with and without inline codes.

    20 patterns repeated 2500 times each (plus random codes), shuffled, so
    every substring of a pattern indexes a bucket of >= 2500 entries that
    starts at arbitrary (also odd) positions."""
    mih = gpu_lib
    rng = np.random.default_rng(77)
    pats = synth.uniform_codes(20, q, 70)
    db = np.concatenate([np.repeat(pats, 2500, axis=0), synth.uniform_codes(10_001, q, 71)])
    db = db[rng.permutation(len(db))]
    qs = np.concatenate([perturb(pats[:6], 2, 72), synth.uniform_codes(4, q, 73)])
    codes, queries = to_dev(db), to_dev(qs)
    W = q // 64
    for m in sorted({2 * W, 2 * W + 1}):
        for inline in (1, -1):
            ix = mih.mih_build(codes, q, m, inline_codes=inline)
            assert max(ix.info()["max_bucket"]) >= 2500
            for k in (10, 3000):
                want_ids, want_dist = orc.knn(db, qs, k)
                r = mih.mih_knn(ix, queries, k)
                assert np.array_equal(ids_of(r["ids"]), want_ids), (m, inline, k)
                assert np.array_equal(host(r["dist"]), want_dist), (m, inline, k)
            woff, wid, wd = orc.rnear(db, qs, 3)
            got = mih.mih_rnear(ix, queries, 3)
            assert np.array_equal(ids_of(got["ids"]), wid) and np.array_equal(host(got["dist"]), wd)
            ix.free()


@pytest.mark.parametrize("q,m,executor", [(128, 4, 2), (128, 5, 2), (64, 2, 1)])
def test_bounded_wait_timeout_path(gpu_lib, orc, q, m, executor):
    """A bounded wait on a bulk copy that runs out ends the call with
    MIH_ETIMEOUT, and the same index answers exactly afterwards.

    The wait is made to run out without any fault: with the test switch of
    mih_set_wait_limit each warp of the slice kernel makes its first wait on a
    barrier that no copy completes (limit 200 us); the warp then drains its own
    copies before leaving.  Big buckets (20 patterns x 2500 copies) make sure
    the slice kernel runs; m = q/32 streams records, m = 5 whole codes."""
    mih = gpu_lib
    rng = np.random.default_rng(91)
    pats = synth.uniform_codes(20, q, 90)
    db = np.concatenate([np.repeat(pats, 2500, axis=0), synth.uniform_codes(10_001, q, 92)])
    db = db[rng.permutation(len(db))]
    qs = np.concatenate([perturb(pats[:6], 2, 93), synth.uniform_codes(4, q, 94)])
    codes, queries = to_dev(db), to_dev(qs)
    ix = mih.mih_build(codes, q, m, inline_codes=1, executor=executor)
    try:
        mih.mih_set_wait_limit(200, True)
        for call in (lambda: mih.mih_knn(ix, queries, 10), lambda: mih.mih_rnear(ix, queries, 3)):
            with pytest.raises(mih.MihError) as e:
                call()
            assert e.value.status == mih.MIH_ETIMEOUT, str(e.value)
    finally:
        mih.mih_set_wait_limit(0, False)
    want_ids, want_dist = orc.knn(db, qs, 10)
    r = mih.mih_knn(ix, queries, 10)
    assert np.array_equal(ids_of(r["ids"]), want_ids) and np.array_equal(host(r["dist"]), want_dist)
    woff, wid, wd = orc.rnear(db, qs, 3)
    got = mih.mih_rnear(ix, queries, 3)
    assert np.array_equal(ids_of(got["ids"]), wid) and np.array_equal(host(got["dist"]), wd)
    ix.free()


UNEVEN_CASES = [
    ("lsh", 128, [29, 24, 25, 25, 25], 100_003),
    ("uniform", 64, [22, 23, 19], 50_000),
    ("lsh", 256, [31, 31, 31, 27, 27, 27, 27, 27, 28], 30_001),
    ("ties", 128, [30, 26, 24, 24, 24], 5_000),
    ("lsh", 128, [16, 32, 32, 24, 24], 60_000),
]


@pytest.mark.parametrize("kind,q,lengths,n", UNEVEN_CASES)
def test_per_table_lengths_match_oracle(gpu_lib, orc, kind, q, lengths, n):
    """Per-table substring lengths (open in the Conclusion): results equal the
    definition, and the Alg. 3 counters equal the oracle's over the same
    partition (Props. 1-2 hold for any disjoint partition)."""
    mih = gpu_lib
    m = len(lengths)
    db, qs = workload(kind, q, n, 97, seed=71)
    codes, queries = to_dev(db), to_dev(qs)
    ix = mih.mih_build(codes, q, m, substring_length=lengths)
    info = ix.info()
    assert info["substring_length"] == lengths
    assert info["substring_offset"] == [int(x) for x in np.concatenate([[0], np.cumsum(lengths)[:-1]])]
    for k in (1, 10, 100):
        want_ids, want_dist = orc.knn(db, qs, k)
        r = mih.mih_knn(ix, queries, k)
        assert np.array_equal(ids_of(r["ids"]), want_ids), k
        assert np.array_equal(host(r["dist"]), want_dist), k
    woff, wid, wd = orc.rnear(db, qs, q // 16)
    got = mih.mih_rnear(ix, queries, q // 16)
    assert np.array_equal(ids_of(got["ids"]), wid) and np.array_equal(host(got["dist"]), wd)
    ix.free()
    # Alg. 3 counters on a smaller database
    small = db[:min(n, 8000)]
    mo = orc.MihOracle(small, q, m, lengths=lengths)
    ixs = mih.mih_build(to_dev(small), q, m, substring_length=lengths, scan_factor=-1)
    r = mih.mih_knn(ixs, to_dev(qs[:24]), 10, query_stats=True)
    st = host(r["query_stats"])
    for i in range(24):
        ids, dist, cnt = mo.knn(qs[i], 10)
        assert np.array_equal(ids_of(r["ids"])[i], ids) and np.array_equal(host(r["dist"])[i], dist)
        assert tuple(st[i]) == tuple(cnt), (i, st[i], cnt)
    ixs.free()


def test_per_table_lengths_are_validated(gpu_lib):
    mih = gpu_lib
    codes = to_dev(synth.uniform_codes(1000, 128, 3))
    for m, ln in ((5, [30, 30, 30, 30, 9]), (4, [33, 31, 32, 32]), (5, [32, 32, 32, 32, 0]), (3, [64, 32, 32])):
        with pytest.raises(mih.MihError) as e:
            mih.mih_build(codes, 128, m, substring_length=ln)
        assert e.value.status == mih.MIH_EINVAL


def test_autotune_layout(gpu_lib, orc):
    """The layout autotuner times the Sec. 2.1 layout against the cost-model
    layout for the measured stop steps and returns a valid partition; the
    index built on it is exact."""
    mih = gpu_lib
    db, _ = workload("lsh", 128, 300_000, 1)
    hold = synth.lsh_codes(400, 128, 9)
    lengths, times = mih.mih_autotune_layout(to_dev(db), 128, to_dev(hold), 50, 5)
    assert len(lengths) == 5 and sum(lengths) == 128 and all(1 <= s <= 32 for s in lengths)
    assert times["uniform"] > 0 and times["cost_model"] > 0
    ix = mih.mih_build(to_dev(db), 128, 5, substring_length=lengths)
    want_ids, want_dist = orc.knn(db, hold[:60], 50)
    r = mih.mih_knn(ix, to_dev(hold[:60]), 50)
    assert np.array_equal(ids_of(r["ids"]), want_ids) and np.array_equal(host(r["dist"]), want_dist)


@pytest.mark.parametrize("q,m,sizes,k", [(128, 4, [40_000, 25_001, 35_000], 100), (64, 3, [30_000, 70, 20_000], 100),
                                         (256, 9, [500, 300, 400], 2000)])
def test_db_shards_merge_to_the_whole_answer(gpu_lib, orc, q, m, sizes, k):
    """A database split into id ranges, one index per range, answers merged by
    mih_merge_topk: equal to the oracle over the whole database (Sec. 1.1).
    Covers a range with fewer than k codes and k above the whole database."""
    import torch

    mih = gpu_lib
    n = sum(sizes)
    db, qs = workload("lsh", q, n, 77, seed=81)
    codes, queries = to_dev(db), to_dev(qs)
    bases = list(np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64))
    ids, dist = [], []
    for lo, sz in zip(bases, sizes):
        ix = mih.mih_build(codes[lo:lo + sz].contiguous(), q, m)
        r = mih.mih_knn(ix, queries, k)
        ids.append(r["ids"])
        dist.append(r["dist"])
        ix.free()
    got = mih.mih_merge_topk(torch.stack(ids).contiguous(), torch.stack(dist).contiguous(), bases, k)
    want_ids, want_dist = orc.knn(db, qs, k)
    assert np.array_equal(ids_of(got["ids"]), want_ids)
    assert np.array_equal(host(got["dist"]), want_dist)
    # merging fewer results than each part holds
    got5 = mih.mih_merge_topk(torch.stack(ids).contiguous(), torch.stack(dist).contiguous(), bases, 5)
    w5, d5 = orc.knn(db, qs, 5)
    assert np.array_equal(ids_of(got5["ids"]), w5) and np.array_equal(host(got5["dist"]), d5)


def test_measured_ceilings_are_plausible(gpu_lib):
    """The ceilings the rooflines are quoted against: positive, and within a
    factor of the unit counts and clock (popc: at most 64 per SM and clock)."""
    mih = gpu_lib
    c = mih.mih_measure_ceilings(gather_bytes=1 << 30)
    assert c["sms"] > 0 and c["sm_clock_mhz"] > 0
    upper = 64.0 * c["sms"] * c["sm_clock_mhz"] * 1e6
    assert 0 < c["popc_per_s"] <= upper * 1.05
    assert c["b1_mma_pairs128_per_s"] > 0 and c["fp8_mma_tflops"] > 0 and c["gather32_gbs"] > 0
    assert c["fp8_mma_pairs128_per_s"] == pytest.approx(c["fp8_mma_tflops"] * 1e12 / 256.0)


@pytest.mark.parametrize("q,m", [(128, 4), (128, 5), (64, 2), (256, 8)])
def test_slice_shapes_and_search_tuning(gpu_lib, orc, q, m):
    """Every shape of the big-bucket slice kernel gives the oracle's answer
    (m = q/32 streams records, other m whole codes), and mih_tune_search keeps
    a valid choice that stays exact.  Big buckets: 20 patterns x 2500 copies."""
    mih = gpu_lib
    rng = np.random.default_rng(101)
    pats = synth.uniform_codes(20, q, 102)
    db = np.concatenate([np.repeat(pats, 2500, axis=0), synth.uniform_codes(20_001, q, 103)])
    db = db[rng.permutation(len(db))]
    qs = np.concatenate([perturb(pats[:8], 3, 104), synth.uniform_codes(8, q, 105)])
    codes, queries = to_dev(db), to_dev(qs)
    for k in (10, 3000):
        want_ids, want_dist = orc.knn(db, qs, k)
        for shape in (0, 1, 2):
            ix = mih.mih_build(codes, q, m, inline_codes=1, slice_shape=shape)
            r = mih.mih_knn(ix, queries, k)
            assert np.array_equal(ids_of(r["ids"]), want_ids), (shape, k)
            assert np.array_equal(host(r["dist"]), want_dist), (shape, k)
            ix.free()
    ix = mih.mih_build(codes, q, m, inline_codes=1)
    best, table = mih.mih_tune_search(ix, queries, 100)
    assert best["slice_shape"] in mih.SLICE_SHAPES and len(table) == 9 and all(v > 0 for v in table.values())
    want_ids, want_dist = orc.knn(db, qs, 100)
    r = mih.mih_knn(ix, queries, 100)
    assert np.array_equal(ids_of(r["ids"]), want_ids) and np.array_equal(host(r["dist"]), want_dist)
    with pytest.raises(mih.MihError):
        mih.mih_build(codes, q, m, slice_shape=3)
    ix.free()


def test_autotune_picks_a_candidate(gpu_lib, orc):
    """Sec. 6: m chosen by timing the search on hold-out queries."""
    mih = gpu_lib
    db, _ = workload("lsh", 128, 200_000, 1)
    hold = synth.lsh_codes(300, 128, 9)
    best, times = mih.mih_autotune(to_dev(db), 128, to_dev(hold), 20, candidates=[3, 4, 5, 6])
    assert best in (4, 5, 6) and set(times) == {4, 5, 6}          # m = 3 needs 43-bit substrings: skipped
    assert all(t > 0 for t in times.values()) and times[best] == min(times.values())
    best2, times2 = mih.mih_autotune(to_dev(db), 128, to_dev(hold), 20)    # around q / log2(n) = 7.2
    assert best2 in times2 and set(times2) == {6, 7, 8}
    ix = mih.mih_build(to_dev(db), 128, best)
    want_ids, want_dist = orc.knn(db, hold[:50], 20)
    r = mih.mih_knn(ix, to_dev(hold[:50]), 20)
    assert np.array_equal(ids_of(r["ids"]), want_ids) and np.array_equal(host(r["dist"]), want_dist)
