"""CPU oracle for exact search in Hamming space -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct CPU code (C in ``hamming_oracle.c``, loaded
with ctypes) that states what the GPU library must compute.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it;
the library under ``paper_1307_2982_gb300/`` never does, and the two share no
code.

Paper: Norouzi, Punjani & Fleet, "Fast Exact Search in Hamming Space with
Multi-Index Hashing" (arXiv:1307.2982).

Functions and the passages they follow:

- ``hamming``              Sec. 1.1 (Hamming distance), Sec. 6 "Hamming Distance"
- ``substring_layout``     Sec. 2.1 footnote (floor/ceil substring lengths)
- ``substring_keys``       Sec. 2.1 (contiguous disjoint substrings)
- ``knn``                  Sec. 1.1 (k-NN problem), by definition
- ``rnear``                Sec. 1.1 (r-neighbour problem), by definition
- ``table_build``          Algorithm 1
- ``ring``                 Algorithm 3 (buckets at exactly r' bits)
- ``MihOracle.knn``        Algorithm 3 (with step counters)
- ``MihOracle.rnear``      Algorithm 2 (with step counters)
- ``rerank_asym``          Sec. 5.1 / Conclusion: re-ranking by an asymmetric
                           Hamming distance (the reading is in the C source)

Every function is pinned by ``tests/test_oracle_pins.py`` to something other
than itself (numpy brute force, Eq. 1, Propositions 1-2, special cases).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from math import comb

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hamming_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

PAD_ID = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no -march flags: it runs on x86 and Arm)."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        u64, i32 = ctypes.c_uint64, ctypes.c_int
        lib.orc_hamming.argtypes = [P, P, i32]
        lib.orc_hamming.restype = i32
        lib.orc_substring_layout.argtypes = [i32, i32, P, P]
        lib.orc_substring_keys.argtypes = [P, u64, i32, i32, i32, P]
        lib.orc_knn.argtypes = [P, u64, i32, P, u64, P, P, P, P, i32]
        lib.orc_knn.restype = i32
        lib.orc_rnear_count.argtypes = [P, u64, i32, P, u64, i32, P, i32]
        lib.orc_rnear_count.restype = i32
        lib.orc_rnear_fill.argtypes = [P, u64, i32, P, u64, i32, P, P, P, i32]
        lib.orc_rnear_fill.restype = i32
        lib.orc_table_build.argtypes = [P, u64, i32, i32, i32, P, P]
        lib.orc_table_build.restype = i32
        lib.orc_ring.argtypes = [i32, i32, P, u64]
        lib.orc_ring.restype = u64
        lib.orc_rerank_asym.argtypes = [P, u64, i32, P, u64, P, ctypes.c_uint32, ctypes.c_uint32, P, P]
        lib.orc_rerank_asym.restype = i32
        lib.orc_mih_knn_flat.argtypes = [i32, i32, P, u64, i32, P, P, P, P, P,
                                         ctypes.c_uint32, P, P, P]
        lib.orc_mih_knn_flat.restype = i32
        lib.orc_mih_rnear_flat.argtypes = [i32, i32, P, u64, i32, P, P, P, P, P,
                                           i32, u64, P, P, P]
        lib.orc_mih_rnear_flat.restype = ctypes.c_int64
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _codes(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    if a.ndim == 1:
        a = a.reshape(-1, 1)
    return a


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def hamming(a, b) -> int:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    return _load().orc_hamming(_ptr(a), _ptr(b), a.size)


def substring_layout(q: int, m: int):
    off = np.zeros(m, dtype=np.int32)
    ln = np.zeros(m, dtype=np.int32)
    _load().orc_substring_layout(q, m, _ptr(off), _ptr(ln))
    return off, ln


def substring_keys(codes, off: int, length: int) -> np.ndarray:
    codes = _codes(codes)
    keys = np.zeros(codes.shape[0], dtype=np.uint64)
    _load().orc_substring_keys(_ptr(codes), codes.shape[0], codes.shape[1], off, length, _ptr(keys))
    return keys


def knn(codes, queries, k, nthreads: int | None = None):
    """(ids[nq][k], dist[nq][k]) for a uniform k, or CSR lists for per-query k.

    With an int k: returns two (nq, k) arrays.  With an array k: returns
    (offsets[nq+1], ids, dist) flattened.
    """
    codes, queries = _codes(codes), _codes(queries)
    nq = queries.shape[0]
    uniform = np.isscalar(k)
    kv = np.full(nq, k, dtype=np.uint32) if uniform else np.ascontiguousarray(k, dtype=np.uint32)
    off = np.zeros(nq + 1, dtype=np.uint64)
    off[1:] = np.cumsum(kv.astype(np.uint64))
    tot = int(off[-1])
    ids = np.zeros(max(tot, 1), dtype=np.uint32)
    dist = np.zeros(max(tot, 1), dtype=np.int32)
    st = _load().orc_knn(_ptr(codes), codes.shape[0], codes.shape[1], _ptr(queries), nq,
                         _ptr(kv), _ptr(off), _ptr(ids), _ptr(dist),
                         nthreads or default_threads())
    if st:
        raise MemoryError("oracle knn failed")
    if uniform:
        return ids[:tot].reshape(nq, int(k)), dist[:tot].reshape(nq, int(k))
    return off, ids[:tot], dist[:tot]


def rerank_asym(codes, proj, ids, k: int):
    """(ids[nq][k], a[nq][k]): every row of candidate ids (uint32 [nq][k_in],
    0xFFFFFFFF = padding) ordered by (asymmetric Hamming distance, id) to the
    query's real values proj[nq][q] (float32), first k kept, padded with
    0xFFFFFFFF / -1.0."""
    codes = _codes(codes)
    proj = np.ascontiguousarray(proj, dtype=np.float32)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    nq, q = proj.shape
    if ids.ndim != 2 or ids.shape[0] != nq or q != 64 * codes.shape[1]:
        raise ValueError("rerank_asym: shapes do not match")
    out_ids = np.zeros((nq, k), dtype=np.uint32)
    out_a = np.zeros((nq, k), dtype=np.float64)
    st = _load().orc_rerank_asym(_ptr(codes), codes.shape[0], q, _ptr(proj), nq, _ptr(ids),
                                 ids.shape[1], k, _ptr(out_ids), _ptr(out_a))
    if st == -2:
        raise ValueError("rerank_asym: candidate id out of range")
    if st:
        raise MemoryError("oracle rerank_asym failed")
    return out_ids, out_a


def rnear(codes, queries, r: int, nthreads: int | None = None):
    """(offsets[nq+1], ids, dist): all codes within r bits, (distance, id) order."""
    codes, queries = _codes(codes), _codes(queries)
    nq = queries.shape[0]
    lib = _load()
    nt = nthreads or default_threads()
    counts = np.zeros(nq, dtype=np.uint64)
    lib.orc_rnear_count(_ptr(codes), codes.shape[0], codes.shape[1], _ptr(queries), nq, r,
                        _ptr(counts), nt)
    off = np.zeros(nq + 1, dtype=np.uint64)
    off[1:] = np.cumsum(counts)
    tot = int(off[-1])
    ids = np.zeros(max(tot, 1), dtype=np.uint32)
    dist = np.zeros(max(tot, 1), dtype=np.int32)
    lib.orc_rnear_fill(_ptr(codes), codes.shape[0], codes.shape[1], _ptr(queries), nq, r,
                       _ptr(off), _ptr(ids), _ptr(dist), nt)
    return off, ids[:tot], dist[:tot]


def table_build(codes, off: int, length: int):
    """Algorithm 1 for one substring: (keys sorted, ids) ordered by (key, id)."""
    codes = _codes(codes)
    n = codes.shape[0]
    keys = np.zeros(max(n, 1), dtype=np.uint64)
    ids = np.zeros(max(n, 1), dtype=np.uint32)
    if _load().orc_table_build(_ptr(codes), n, codes.shape[1], off, length, _ptr(keys), _ptr(ids)):
        raise MemoryError("oracle table build failed")
    return keys[:n], ids[:n]


def ring(s: int, rho: int) -> np.ndarray:
    """All x < 2^s with popcount(x) == rho, increasing (brute force, s <= 26)."""
    if s > 26:
        raise ValueError("brute-force ring limited to s <= 26")
    cap = comb(s, rho) if 0 <= rho <= s else 0
    out = np.zeros(max(cap, 1), dtype=np.uint64)
    c = _load().orc_ring(s, rho, _ptr(out), cap)
    return out[: int(c)]


class MihOracle:
    """Algorithms 1-3 on the CPU: m tables over the codes, searched step by step.

    ``counters`` of each search: lookups (buckets examined), raw candidates
    (bucket entries read), unique candidates, last step executed.

    ``lengths`` (optional, m entries summing to q) gives table j the
    contiguous substring of lengths[j] bits that follows table j-1's, the
    per-table lengths the Conclusion (Sec. 8) leaves open; Propositions 1 and 2
    (Sec. 2.1) hold for any partition of the bits into m disjoint substrings.
    Default: the floor/ceil layout of the Sec. 2.1 footnote.
    """

    def __init__(self, codes, q: int, m: int, lengths=None):
        self.codes = _codes(codes)
        self.n, self.W = self.codes.shape
        self.q, self.m = q, m
        if lengths is None:
            self.off, self.len = substring_layout(q, m)
        else:
            self.len = np.ascontiguousarray(lengths, dtype=np.int32)
            if self.len.shape != (m,) or int(self.len.sum()) != q or int(self.len.min()) < 1:
                raise ValueError("lengths must be m positive entries summing to q")
            self.off = np.concatenate([[0], np.cumsum(self.len)[:-1]]).astype(np.int32)
        if int(self.len.max()) > 64:
            raise ValueError("oracle substring keys hold at most 64 bits")
        self.keys, self.ids = [], []
        for j in range(m):
            kj, ij = table_build(self.codes, int(self.off[j]), int(self.len[j]))
            self.keys.append(np.ascontiguousarray(kj) if self.n else np.zeros(1, np.uint64))
            self.ids.append(np.ascontiguousarray(ij) if self.n else np.zeros(1, np.uint32))
        self._kp = (ctypes.c_void_p * m)(*[k.ctypes.data for k in self.keys])
        self._ip = (ctypes.c_void_p * m)(*[i.ctypes.data for i in self.ids])

    def knn(self, g, k: int):
        g = np.ascontiguousarray(g, dtype=np.uint64).reshape(-1)
        ids = np.zeros(max(k, 1), dtype=np.uint32)
        dist = np.zeros(max(k, 1), dtype=np.int32)
        cnt = np.zeros(4, dtype=np.int64)
        st = _load().orc_mih_knn_flat(self.q, self.m, _ptr(self.codes), self.n, self.W,
                                      _ptr(self.off), _ptr(self.len), self._kp, self._ip,
                                      _ptr(g), k, _ptr(ids), _ptr(dist), _ptr(cnt))
        if st:
            raise MemoryError("oracle MIH knn failed")
        return ids[:k], dist[:k], cnt

    def rnear(self, g, r: int):
        g = np.ascontiguousarray(g, dtype=np.uint64).reshape(-1)
        cnt = np.zeros(4, dtype=np.int64)
        lib = _load()
        args = (self.q, self.m, _ptr(self.codes), self.n, self.W, _ptr(self.off),
                _ptr(self.len), self._kp, self._ip, _ptr(g), r)
        tot = lib.orc_mih_rnear_flat(*args, 0, None, None, _ptr(cnt))
        if tot < 0:
            raise MemoryError("oracle MIH rnear failed")
        ids = np.zeros(max(tot, 1), dtype=np.uint32)
        dist = np.zeros(max(tot, 1), dtype=np.int32)
        lib.orc_mih_rnear_flat(*args, tot, _ptr(ids), _ptr(dist), _ptr(cnt))
        return ids[:tot], dist[:tot], cnt
