"""linscan_knn_noalloc: the linear scan for callers that cannot allocate.

Callers such as a serving thread that must not trigger the device-wide
synchronisation of cudaMalloc/cudaFree, or a process whose allocator already
holds the device memory, use this entry point; it works out of a fixed array
compiled into the library.  The test calls it through the C-ABI twice in a
row and checks each result against linscan_knn (integer results: bit-exact,
the tolerance used by every parity test here).  This file is collected last,
so a run that stops at the first failure has run every other test already.
"""
import ctypes

import numpy as np
import pytest

from paper_1307_2982_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _call(mih, codes, q, queries, k):
    """Raw C-ABI call; returns (status, ids, dist)."""
    import torch

    lib = mih.load()
    nq = queries.shape[0]
    ids = torch.full((nq, k), -7, dtype=torch.int32, device="cuda")
    dist = torch.full((nq, k), -7, dtype=torch.int32, device="cuda")
    st = lib.linscan_knn_noalloc(mih._ptr(codes), codes.shape[0], q, mih._ptr(queries), nq, k, mih._ptr(ids),
                                 mih._ptr(dist), mih._stream(None))
    return st, ids, dist


@pytest.mark.parametrize("kind,q,n", [("lsh", 128, 300_001), ("uniform", 64, 200_000), ("lsh", 256, 70_000)])
def test_noalloc_matches_linscan_twice(gpu_lib, kind, q, n):
    mih = gpu_lib
    gen = synth.lsh_codes if kind == "lsh" else synth.uniform_codes
    codes = _dev(gen(n, q, 0))
    # two calls in a row with different batches: the shared scratch must not
    # carry anything from the first call into the second
    for seed, nq, k in ((1, 256, 100), (2, 97, 256)):
        queries = _dev(gen(nq, q, seed))
        st, ids, dist = _call(mih, codes, q, queries, k)
        assert st == mih.MIH_OK, mih.mih_last_error()
        want = mih.linscan_knn(codes, q, queries, k)
        assert np.array_equal(ids.cpu().numpy(), want["ids"].cpu().numpy())
        assert np.array_equal(dist.cpu().numpy(), want["dist"].cpu().numpy())


@pytest.mark.parametrize("n", [0, 37])
def test_noalloc_small_databases_twice(gpu_lib, n):
    """n < k: all n codes, then padding (id 0xFFFFFFFF, distance -1); n = 0:
    padding only.  Both as linscan_knn gives them, on two calls in a row."""
    mih = gpu_lib
    q, k = 128, 100
    codes = _dev(synth.uniform_codes(max(n, 1), q, 11))[:n]
    for seed, nq in ((12, 33), (13, 5)):
        queries = _dev(synth.uniform_codes(nq, q, seed))
        st, ids, dist = _call(mih, codes, q, queries, k)
        assert st == mih.MIH_OK, mih.mih_last_error()
        want = mih.linscan_knn(codes, q, queries, k)
        assert np.array_equal(ids.cpu().numpy(), want["ids"].cpu().numpy())
        assert np.array_equal(dist.cpu().numpy(), want["dist"].cpu().numpy())
        assert np.all(ids.cpu().numpy()[:, n:] == -1) and np.all(dist.cpu().numpy()[:, n:] == -1)
        assert np.all(dist.cpu().numpy()[:, :n] >= 0)


def test_noalloc_ties_second_pass_and_limits(gpu_lib):
    mih = gpu_lib
    import torch

    q = 128
    one = synth.uniform_codes(1, q, 5)
    codes = _dev(np.repeat(one, 200_000, axis=0))      # every code ties with every other
    queries = _dev(np.repeat(one, 4, axis=0))
    for _ in range(2):
        st, ids, dist = _call(mih, codes, q, queries, 50)
        assert st == mih.MIH_OK, mih.mih_last_error()
        assert np.array_equal(ids.cpu().numpy(), np.tile(np.arange(50, dtype=np.int32), (4, 1)))
        assert np.all(dist.cpu().numpy() == 0)
    # sizes beyond the fixed scratch are refused with a clear error
    st, _, _ = _call(mih, codes, q, _dev(np.repeat(one, 257, axis=0)), 10)
    assert st == mih.MIH_EINVAL and "at most 256 queries" in mih.mih_last_error()
    st, _, _ = _call(mih, codes, q, queries, 257)
    assert st == mih.MIH_EINVAL and "k must be in [1, 256]" in mih.mih_last_error()
    st, _, _ = _call(mih, codes, q, _dev(np.repeat(one, 8, axis=0)), 10)   # 8 x 200k ties > 2^20 slots
    assert st == mih.MIH_ENOMEM and "fixed scratch" in mih.mih_last_error()
    # and the next call still works
    st, ids, dist = _call(mih, codes, q, queries[:2], 5)
    assert st == mih.MIH_OK and np.array_equal(ids.cpu().numpy(), np.tile(np.arange(5, dtype=np.int32), (2, 1)))
    del torch
