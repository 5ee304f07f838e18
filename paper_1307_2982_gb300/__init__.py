"""Exact k-NN and r-neighbour search in Hamming space by multi-index hashing
on one GB300 GPU (sm_103a).

Thin ctypes binding over the C-ABI of ``include/mih.h`` (library
``libmih.so``, built in-tree by :func:`build`).  The functions keep the C
names; they only marshal arguments (torch CUDA tensors -> device pointers,
the current torch stream -> ``cudaStream_t``) and turn a non-OK status into
:class:`MihError`.  Every step of the search runs in the library's CUDA
kernels; there is no CPU path.

Method: Norouzi, Punjani & Fleet, "Fast Exact Search in Hamming Space with
Multi-Index Hashing" (arXiv:1307.2982).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmih.so")
_lib = None

MIH_OK, MIH_EINVAL, MIH_ENOMEM, MIH_ECUDA, MIH_EOVERFLOW, MIH_ETIMEOUT, MIH_EINTERNAL = range(7)
MIH_TABLE_AUTO, MIH_TABLE_DIRECT, MIH_TABLE_SPARSE = 0, 1, 2
MIH_EXEC_AUTO, MIH_EXEC_HOST, MIH_EXEC_GRAPH = 0, 1, 2
MIH_SCAN_AUTO, MIH_SCAN_POPC, MIH_SCAN_TENSOR = 0, 1, 2
MIH_SLICE_SHAPE_3K_8W, MIH_SLICE_SHAPE_8K_4W, MIH_SLICE_SHAPE_4K_8W = 0, 1, 2
SLICE_SHAPES = ("3KB stages x 8 warps x 2", "8KB stages x 4 warps x 2", "4KB stages x 8 warps x 2")
MIH_MAX_K = 8192
PAD_ID = 0xFFFFFFFF

EXPORTS = (
    "mih_build", "mih_free", "mih_index_get_info", "mih_knn", "mih_rnear", "linscan_knn",
    "mih_substring_layout", "mih_cost_model", "mih_suggest_m", "mih_status_str",
    "mih_last_error", "mih_version", "mih_set_timing", "mih_last_profile", "linscan_knn_noalloc",
    "mih_autotune", "mih_greedy_substrings", "mih_bit_correlation", "mih_set_wait_limit",
    "mih_cost_layout", "mih_autotune_layout", "mih_merge_topk", "mih_measure_ceilings",
    "mih_set_scan_kernel", "mih_k_offsets", "mih_tune_search", "mih_rerank_asym", "mih_rerank_asym_csr",
)


class MihError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


class mih_params(ctypes.Structure):
    _fields_ = [("table_kind", ctypes.c_int32), ("scan_factor", ctypes.c_int32),
                ("inline_codes", ctypes.c_int32), ("probe", ctypes.c_int32), ("executor", ctypes.c_int32),
                ("tail_from", ctypes.c_int32), ("bit_order", ctypes.POINTER(ctypes.c_int32)),
                ("substring_length", ctypes.POINTER(ctypes.c_int32)), ("slice_shape", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


class mih_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in (
        "lookups", "candidates_raw", "candidates_unique", "steps", "phase2_queries", "waves",
        "candidates_sliced")]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


# mih_profile.kernel_ms / kernel_launches index (MIH_PROF_* in include/mih.h)
PROF_KINDS = ("chunk", "slice", "probe", "plan", "stop", "select", "scan", "rerank")


class mih_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("main_launches", ctypes.c_uint64),
                ("main_ms", ctypes.c_double), ("call_ms", ctypes.c_double),
                ("kernel_ms", ctypes.c_double * len(PROF_KINDS)),
                ("kernel_launches", ctypes.c_uint64 * len(PROF_KINDS))]

    def as_dict(self):
        d = {f: (float(getattr(self, f)) if "ms" in f else int(getattr(self, f)))
             for f in ("launches", "main_launches", "main_ms", "call_ms")}
        d["kernel_ms"] = {k: float(v) for k, v in zip(PROF_KINDS, self.kernel_ms)}
        d["kernel_launches"] = {k: int(v) for k, v in zip(PROF_KINDS, self.kernel_launches)}
        return d


class mih_ceilings(ctypes.Structure):
    _fields_ = [("popc_per_s", ctypes.c_double), ("b1_mma_pairs128_per_s", ctypes.c_double),
                ("fp8_mma_tflops", ctypes.c_double), ("fp8_mma_pairs128_per_s", ctypes.c_double),
                ("gather32_gbs", ctypes.c_double), ("sms", ctypes.c_int32), ("sm_clock_mhz", ctypes.c_double)]

    def as_dict(self):
        return {f: (int(getattr(self, f)) if f == "sms" else float(getattr(self, f))) for f, _ in self._fields_}


class mih_index_info(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int32), ("m", ctypes.c_int32), ("W", ctypes.c_int32),
                ("substring_offset", ctypes.c_int32 * 256), ("substring_length", ctypes.c_int32 * 256),
                ("table_kind", ctypes.c_int32 * 256), ("n", ctypes.c_uint64),
                ("distinct_keys", ctypes.c_uint64 * 256), ("max_bucket", ctypes.c_uint64 * 256),
                ("index_bytes", ctypes.c_uint64), ("inline_codes", ctypes.c_int32)]


def build(force: bool = False, verbose: bool = False) -> str:
    from . import build_ext

    return build_ext.build(force=force, verbose=verbose)


def load():
    """Load libmih.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_1307_2982_gb300.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    P, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    st = ctypes.c_int
    lib.mih_build.argtypes = [P, u64, i32, i32, P, P, ctypes.POINTER(P)]
    lib.mih_build.restype = st
    lib.mih_free.argtypes = [P]
    lib.mih_free.restype = None
    lib.mih_index_get_info.argtypes = [P, P]
    lib.mih_index_get_info.restype = st
    lib.mih_knn.argtypes = [P, P, u32, P, u32, P, P, P, P, P, P]
    lib.mih_knn.restype = st
    lib.mih_rnear.argtypes = [P, P, u32, i32, u64, P, P, P, ctypes.POINTER(u64), P, P, P]
    lib.mih_rnear.restype = st
    lib.linscan_knn.argtypes = [P, u64, i32, P, u32, P, u32, P, P, P, P]
    lib.linscan_knn.restype = st
    lib.mih_substring_layout.argtypes = [i32, i32, P, P]
    lib.mih_substring_layout.restype = st
    lib.mih_cost_model.argtypes = [i32, u64, i32, i32]
    lib.mih_cost_model.restype = ctypes.c_double
    lib.mih_cost_layout.argtypes = [i32, u64, i32, P, i32, P]
    lib.mih_cost_layout.restype = ctypes.c_double
    lib.mih_autotune_layout.argtypes = [P, u64, i32, P, u32, u32, i32, P, P, P, P]
    lib.mih_autotune_layout.restype = st
    lib.mih_tune_search.argtypes = [P, P, u32, u32, P, P, P]
    lib.mih_tune_search.restype = st
    lib.mih_k_offsets.argtypes = [P, u32, P, P]
    lib.mih_k_offsets.restype = st
    lib.mih_set_scan_kernel.argtypes = [i32]
    lib.mih_set_scan_kernel.restype = st
    lib.mih_measure_ceilings.argtypes = [P, u64, P]
    lib.mih_measure_ceilings.restype = st
    lib.mih_merge_topk.argtypes = [P, P, u32, u32, u32, P, u32, P, P, P]
    lib.mih_merge_topk.restype = st
    lib.mih_rerank_asym.argtypes = [P, u64, i32, P, u32, P, u32, u32, P, P, P]
    lib.mih_rerank_asym.restype = st
    lib.mih_rerank_asym_csr.argtypes = [P, u64, i32, P, u32, P, P, u32, P, P, P, P]
    lib.mih_rerank_asym_csr.restype = st
    lib.mih_suggest_m.argtypes = [i32, u64]
    lib.mih_suggest_m.restype = i32
    lib.mih_status_str.argtypes = [st]
    lib.mih_status_str.restype = ctypes.c_char_p
    lib.mih_last_error.argtypes = []
    lib.mih_last_error.restype = ctypes.c_char_p
    lib.mih_version.argtypes = []
    lib.mih_version.restype = ctypes.c_char_p
    lib.mih_autotune.argtypes = [P, u64, i32, P, u32, u32, P, i32, P, P, ctypes.POINTER(i32), P]
    lib.mih_autotune.restype = st
    lib.linscan_knn_noalloc.argtypes = [P, u64, i32, P, u32, u32, P, P, P]
    lib.linscan_knn_noalloc.restype = st
    lib.mih_set_wait_limit.argtypes = [u32, i32]
    lib.mih_set_wait_limit.restype = st
    lib.mih_set_timing.argtypes = [i32]
    lib.mih_set_timing.restype = None
    lib.mih_last_profile.argtypes = [P]
    lib.mih_last_profile.restype = st
    lib.mih_greedy_substrings.argtypes = [P, i32, i32, u64, P]
    lib.mih_greedy_substrings.restype = st
    lib.mih_bit_correlation.argtypes = [P, u64, i32, P, P]
    lib.mih_bit_correlation.restype = st
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != MIH_OK:
        lib = load()
        detail = lib.mih_last_error().decode() or lib.mih_status_str(status).decode()
        raise MihError(status, where, detail)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _codes_arg(codes, q: int):
    """(n, q/64) int64/uint64 CUDA tensor -> (pointer, n)."""
    if not codes.is_cuda:
        raise ValueError("codes must be a CUDA tensor")
    if codes.dim() != 2 or codes.shape[1] * 64 != q or not codes.is_contiguous():
        raise ValueError(f"codes must be a contiguous (n, {q // 64}) tensor")
    if codes.element_size() != 8:
        raise ValueError("codes must have 8-byte elements (int64 or uint64 bit patterns)")
    return _ptr(codes), codes.shape[0]


# ----------------------------------------------------------------- host-only
def mih_status_str(status: int) -> str:
    return load().mih_status_str(status).decode()


def mih_last_error() -> str:
    return load().mih_last_error().decode()


def mih_version() -> str:
    return load().mih_version().decode()


def mih_set_timing(level):
    """0/False off, 1/True main kernels and the call, 2 also every kernel kind
    (mih_knn then runs its waves from a host loop)."""
    load().mih_set_timing(int(level))


def mih_set_wait_limit(limit_us: int = 0, expire_first_wait: bool = False):
    """Limit of the bounded device waits of this thread's calls (0 = 1 s); with
    expire_first_wait the slice kernel's first waits run out (timeout test)."""
    _check(load().mih_set_wait_limit(limit_us, 1 if expire_first_wait else 0), "mih_set_wait_limit")


def mih_set_scan_kernel(kind: int):
    """linscan_knn's kernel for this thread: MIH_SCAN_AUTO, MIH_SCAN_POPC or MIH_SCAN_TENSOR."""
    _check(load().mih_set_scan_kernel(int(kind)), "mih_set_scan_kernel")


def mih_measure_ceilings(gather_bytes: int = 8 << 30, stream=None) -> dict:
    """Measured POPC, b1/fp8 mma.sync and random 32-byte gather rates of this GPU."""
    c = mih_ceilings()
    _check(load().mih_measure_ceilings(ctypes.byref(c), gather_bytes, _stream(stream)), "mih_measure_ceilings")
    return c.as_dict()


def mih_last_profile() -> dict:
    p = mih_profile()
    _check(load().mih_last_profile(ctypes.byref(p)), "mih_last_profile")
    return p.as_dict()


def mih_substring_layout(q: int, m: int):
    off = (ctypes.c_int32 * max(m, 1))()
    ln = (ctypes.c_int32 * max(m, 1))()
    _check(load().mih_substring_layout(q, m, off, ln), "mih_substring_layout")
    return list(off)[:m], list(ln)[:m]


def mih_cost_model(q: int, n: int, s: int, r: int) -> float:
    return float(load().mih_cost_model(q, n, s, r))


def mih_suggest_m(q: int, n: int) -> int:
    return int(load().mih_suggest_m(q, n))


def mih_cost_layout(q: int, n: int, m: int, step_weight):
    """Per-table lengths minimising Eq. 7 table by table over Alg. 3 stopped at
    step t with weight step_weight[t].  Returns (lengths list, cost)."""
    w = np.ascontiguousarray(step_weight, dtype=np.float64)
    out = np.zeros(max(m, 1), dtype=np.int32)
    c = float(load().mih_cost_layout(q, n, m, w.ctypes.data, int(w.size), out.ctypes.data))
    if c < 0:
        raise MihError(MIH_EINVAL, "mih_cost_layout", "invalid arguments")
    return [int(x) for x in out[:m]], c


def mih_greedy_substrings(corr, m: int, seed: int = 0):
    """Greedy bit-to-substring assignment of Sec. 5.5 from a (q, q) correlation
    matrix; returns the int32 bit order for ``mih_build(bit_order=...)``."""
    c = np.ascontiguousarray(corr, dtype=np.float64)
    q = c.shape[0]
    if c.shape != (q, q):
        raise ValueError("corr must be square")
    out = np.empty(q, dtype=np.int32)
    _check(load().mih_greedy_substrings(c.ctypes.data, q, m, seed, out.ctypes.data), "mih_greedy_substrings")
    return out


def mih_bit_correlation(codes, q: int, stream=None):
    """(q, q) float64 correlation between the bits of the device codes (Sec. 5.5)."""
    ptr, n = _codes_arg(codes, q)
    out = np.empty((q, q), dtype=np.float64)
    _check(load().mih_bit_correlation(ptr, n, q, out.ctypes.data, _stream(stream)), "mih_bit_correlation")
    return out


def optimize_substrings(sample_codes, q: int, m: int, seed: int = 0, stream=None):
    """Bit order of optimised substrings (Sec. 5.5) from sample codes on the device."""
    return mih_greedy_substrings(mih_bit_correlation(sample_codes, q, stream=stream), m, seed)


# ------------------------------------------------------------------- index
class MihIndex:
    """Owns a ``mih_index*``; keeps the borrowed code tensor alive."""

    def __init__(self, handle, codes, q: int, m: int):
        self.handle = handle
        self.codes = codes
        self.q, self.m = q, m
        self.n = codes.shape[0]

    def info(self) -> dict:
        inf = mih_index_info()
        _check(load().mih_index_get_info(self.handle, ctypes.byref(inf)), "mih_index_get_info")
        m = inf.m
        return {
            "q": inf.q, "m": m, "n": int(inf.n), "index_bytes": int(inf.index_bytes),
            "substring_offset": list(inf.substring_offset)[:m],
            "substring_length": list(inf.substring_length)[:m],
            "table_kind": list(inf.table_kind)[:m],
            "distinct_keys": [int(x) for x in list(inf.distinct_keys)[:m]],
            "max_bucket": [int(x) for x in list(inf.max_bucket)[:m]],
            "inline_codes": int(inf.inline_codes),
        }

    def free(self):
        if self.handle:
            load().mih_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mih_build(codes, q: int, m: int, table_kind: int = MIH_TABLE_AUTO, scan_factor: int = 0,
              inline_codes: int = 0, probe: int = 0, executor: int = MIH_EXEC_AUTO, bit_order=None,
              substring_length=None, tail_from: int = 0, slice_shape: int = 0, stream=None) -> MihIndex:
    ptr, n = _codes_arg(codes, q)
    p = mih_params()
    p.table_kind = table_kind
    p.scan_factor = scan_factor
    p.inline_codes = inline_codes
    p.probe = probe
    p.executor = executor
    p.tail_from = tail_from
    p.slice_shape = slice_shape
    if bit_order is not None:
        order = np.ascontiguousarray(bit_order, dtype=np.int32)
        if order.shape != (q,):
            raise ValueError("bit_order must hold q entries")
        p.bit_order = order.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    if substring_length is not None:
        lens = np.ascontiguousarray(substring_length, dtype=np.int32)
        p.substring_length = lens.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    h = ctypes.c_void_p()
    _check(load().mih_build(ptr, n, q, m, ctypes.byref(p), _stream(stream), ctypes.byref(h)), "mih_build")
    return MihIndex(h, codes, q, m)


def mih_autotune(codes, q: int, queries, k: int, candidates=None, stream=None, **build):
    """Pick m by timing mih_knn on hold-out queries (Sec. 6).  Returns (best_m, {m: ms per query})."""
    cptr, n = _codes_arg(codes, q)
    qptr, nq = _codes_arg(queries, q)
    p = mih_params()
    for key, v in build.items():
        setattr(p, key, v)
    cand = None if candidates is None else (ctypes.c_int * len(candidates))(*candidates)
    ncand = 3 if candidates is None else len(candidates)
    times = (ctypes.c_double * ncand)()
    best = ctypes.c_int(0)
    _check(load().mih_autotune(cptr, n, q, qptr, nq, k, cand, ncand if candidates else 0, ctypes.byref(p),
                               _stream(stream), ctypes.byref(best), times), "mih_autotune")
    ms = list(candidates) if candidates else [mih_suggest_m(q, n) + d for d in (-1, 0, 1)]
    return best.value, {m: t for m, t in zip(ms, times) if t >= 0}


def mih_autotune_layout(codes, q: int, queries, k: int, m: int, stream=None, **build):
    """Per-table lengths for m tables, timed on hold-out queries.  Returns
    (lengths, {"uniform": ms per query, "cost_model": ms per query})."""
    cptr, n = _codes_arg(codes, q)
    qptr, nq = _codes_arg(queries, q)
    p = mih_params()
    for key, v in build.items():
        setattr(p, key, v)
    out = np.zeros(m, dtype=np.int32)
    times = (ctypes.c_double * 2)()
    _check(load().mih_autotune_layout(cptr, n, q, qptr, nq, k, m, ctypes.byref(p), _stream(stream),
                                      out.ctypes.data, times), "mih_autotune_layout")
    return [int(x) for x in out], {"uniform": times[0], "cost_model": times[1]}


class mih_search_tuning(ctypes.Structure):
    _fields_ = [("slice_shape", ctypes.c_int32), ("tail_from", ctypes.c_int32)]


def mih_tune_search(index: MihIndex, queries, k: int, stream=None):
    """Slice-kernel shape and two-step start of the index's k-NN waves, timed on
    hold-out queries and kept in the index.  Returns (best dict, {(shape, tail): ms per query})."""
    qptr, nq = _codes_arg(queries, index.q)
    best = mih_search_tuning()
    times = (ctypes.c_double * 9)()
    _check(load().mih_tune_search(index.handle, qptr, nq, k, _stream(stream), ctypes.byref(best), times),
           "mih_tune_search")
    tails = ("2m", "m", "never")
    table = {f"{SLICE_SHAPES[sh]} / tail {tails[t]}": times[sh * 3 + t] for sh in range(3) for t in range(3)
             if times[sh * 3 + t] >= 0}
    return {"slice_shape": SLICE_SHAPES[best.slice_shape], "tail_from": int(best.tail_from)}, table


def mih_free(index: MihIndex):
    index.free()


def _k_args(nq, k, device, stream=None):
    """Uniform int k, or per-query k -> C arguments (k, k_uniform, offsets, output shape).

    Host k (numpy array or CPU tensor): the CSR offsets and their total come
    from the host values and both arrays are copied to the device, with no
    device synchronisation.  Device k: the library computes the offsets
    (mih_k_offsets) and the total is read back once, to size the outputs."""
    import torch

    if isinstance(k, int):
        return None, k, None, (nq, k)
    if isinstance(k, torch.Tensor) and k.is_cuda:
        kt = k.to(torch.int32).contiguous()
        off = torch.empty(nq + 1, dtype=torch.int64, device=device)
        _check(load().mih_k_offsets(_ptr(kt), nq, _ptr(off), _stream(stream)), "mih_k_offsets")
        return kt, 0, off, (int(off[-1].item()),)
    if isinstance(k, torch.Tensor):
        kc = k if (k.dtype == torch.int32 and k.is_contiguous()) else k.to(torch.int32).contiguous()
        kh = kc.numpy()
    else:
        kh = np.ascontiguousarray(k, dtype=np.int32)
        kc = torch.from_numpy(kh)
    if kh.shape != (nq,):
        raise ValueError("per-query k must hold one entry per query")
    offh = np.zeros(nq + 1, dtype=np.int64)
    np.cumsum(kh, dtype=np.int64, out=offh[1:])
    kt = kc.to(device, non_blocking=True)
    off = torch.from_numpy(offh).to(device)
    return kt, 0, off, (int(offh[-1]),)


def mih_knn(index: MihIndex, queries, k, stream=None, query_stats: bool = False, out=None):
    """Exact k-NN (Alg. 3).  Returns (ids int32-view of uint32, dist, [offsets], stats dict[, qstats])."""
    import torch

    qptr, nq = _codes_arg(queries, index.q)
    kt, ku, off, shape = _k_args(nq, k, queries.device, stream)
    if out is None:
        ids = torch.empty(shape, dtype=torch.int32, device=queries.device)
        dist = torch.empty(shape, dtype=torch.int32, device=queries.device)
    else:
        ids, dist = out
    qs = torch.empty((nq, 4), dtype=torch.int64, device=queries.device) if query_stats else None
    st = mih_stats()
    _check(load().mih_knn(index.handle, qptr, nq, _ptr(kt), ku, _ptr(off), _ptr(ids), _ptr(dist), _ptr(qs),
                          ctypes.byref(st), _stream(stream)), "mih_knn")
    res = {"ids": ids, "dist": dist, "stats": st.as_dict()}
    if off is not None:
        res["offsets"] = off
    if qs is not None:
        res["query_stats"] = qs
    return res


def mih_rnear(index: MihIndex, queries, r: int, capacity: int | None = None, stream=None,
              query_stats: bool = False):
    """All codes within r bits (Alg. 2), CSR (offsets, ids, dist) in (distance, id) order.

    With capacity None the call sizes the output itself (count call, then fill)."""
    import torch

    qptr, nq = _codes_arg(queries, index.q)
    dev = queries.device
    off = torch.empty(nq + 1, dtype=torch.int64, device=dev)
    qs = torch.empty((nq, 4), dtype=torch.int64, device=dev) if query_stats else None
    lib = load()
    total = ctypes.c_uint64(0)
    st = mih_stats()
    if capacity is None:
        s = lib.mih_rnear(index.handle, qptr, nq, r, 0, _ptr(off), None, None, ctypes.byref(total), None, None,
                          _stream(stream))
        if s not in (MIH_OK, MIH_EOVERFLOW):
            _check(s, "mih_rnear")
        capacity = int(total.value)
    ids = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    dist = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    _check(lib.mih_rnear(index.handle, qptr, nq, r, capacity, _ptr(off), _ptr(ids), _ptr(dist),
                         ctypes.byref(total), _ptr(qs), ctypes.byref(st), _stream(stream)), "mih_rnear")
    t = int(total.value)
    res = {"offsets": off, "ids": ids[:t], "dist": dist[:t], "total": t, "stats": st.as_dict()}
    if qs is not None:
        res["query_stats"] = qs
    return res


def linscan_knn(codes, q: int, queries, k, stream=None, out=None):
    """Exact k-NN by linear scan (Sec. 5.2 baseline)."""
    import torch

    cptr, n = _codes_arg(codes, q)
    qptr, nq = _codes_arg(queries, q)
    kt, ku, off, shape = _k_args(nq, k, queries.device, stream)
    if out is None:
        ids = torch.empty(shape, dtype=torch.int32, device=queries.device)
        dist = torch.empty(shape, dtype=torch.int32, device=queries.device)
    else:
        ids, dist = out
    _check(load().linscan_knn(cptr, n, q, qptr, nq, _ptr(kt), ku, _ptr(off), _ptr(ids), _ptr(dist),
                              _stream(stream)), "linscan_knn")
    res = {"ids": ids, "dist": dist}
    if off is not None:
        res["offsets"] = off
    return res


def mih_merge_topk(ids, dist, id_base, k: int, stream=None, out=None):
    """Exact k-NN of a database split into id ranges: ids/dist are (parts, nq,
    k_in) CUDA int32 tensors of the parts' answers (ids relative to each part),
    id_base the parts' first global ids.  Returns {"ids", "dist"} (nq, k)."""
    import torch

    if not (ids.is_cuda and dist.is_cuda):
        raise ValueError("ids and dist must be CUDA tensors")
    if ids.dim() != 3 or ids.shape != dist.shape or not (ids.is_contiguous() and dist.is_contiguous()):
        raise ValueError("ids and dist must be contiguous (parts, nq, k_in) tensors")
    parts, nq, k_in = ids.shape
    base = np.ascontiguousarray(id_base, dtype=np.uint32)
    if base.shape != (parts,):
        raise ValueError("id_base must hold one entry per part")
    if out is None:
        oi = torch.empty((nq, k), dtype=torch.int32, device=ids.device)
        od = torch.empty((nq, k), dtype=torch.int32, device=ids.device)
    else:
        oi, od = out
    _check(load().mih_merge_topk(_ptr(ids), _ptr(dist), parts, nq, k_in, base.ctypes.data, k, _ptr(oi), _ptr(od),
                                 _stream(stream)), "mih_merge_topk")
    return {"ids": oi, "dist": od}


def mih_rerank_asym(codes, q: int, proj, ids, k: int, stream=None, out=None):
    """Re-rank each row of candidate ids (nq, k_in) CUDA int32 (bit patterns of
    uint32; -1 = padding) by the asymmetric Hamming distance to the query's
    real projections proj (nq, q) float32 CUDA.  Returns {"ids": (nq, k)
    int32, "a": (nq, k) float64}."""
    import torch

    cptr, n = _codes_arg(codes, q)
    if not (proj.is_cuda and ids.is_cuda):
        raise ValueError("proj and ids must be CUDA tensors")
    if proj.dtype != torch.float32 or proj.dim() != 2 or proj.shape[1] != q or not proj.is_contiguous():
        raise ValueError(f"proj must be a contiguous (nq, {q}) float32 tensor")
    if ids.dim() != 2 or ids.shape[0] != proj.shape[0] or ids.element_size() != 4 or not ids.is_contiguous():
        raise ValueError("ids must be a contiguous (nq, k_in) tensor of 4-byte ids")
    nq, k_in = ids.shape
    if out is None:
        oi = torch.empty((nq, k), dtype=torch.int32, device=ids.device)
        oa = torch.empty((nq, k), dtype=torch.float64, device=ids.device)
    else:
        oi, oa = out
    _check(load().mih_rerank_asym(cptr, n, q, _ptr(proj), nq, _ptr(ids), k_in, k, _ptr(oi), _ptr(oa),
                                  _stream(stream)), "mih_rerank_asym")
    return {"ids": oi, "a": oa}


def mih_rerank_asym_csr(codes, q: int, proj, ids, in_offsets, out_offsets, k_in_max: int | None = None,
                        stream=None, out=None):
    """mih_rerank_asym for CSR rows: row i's candidates are
    ids[in_offsets[i]:in_offsets[i+1]] (CUDA int32 / uint32 bit patterns, -1 =
    padding), its results out[out_offsets[i]:out_offsets[i+1]].  Offsets:
    (nq + 1,) CUDA int64.  k_in_max: the longest candidate row (read from
    in_offsets when None).  Returns {"ids": int32, "a": float64}, flat."""
    import torch

    cptr, n = _codes_arg(codes, q)
    if not (proj.is_cuda and ids.is_cuda and in_offsets.is_cuda and out_offsets.is_cuda):
        raise ValueError("proj, ids and the offsets must be CUDA tensors")
    if proj.dtype != torch.float32 or proj.dim() != 2 or proj.shape[1] != q or not proj.is_contiguous():
        raise ValueError(f"proj must be a contiguous (nq, {q}) float32 tensor")
    nq = proj.shape[0]
    for t in (in_offsets, out_offsets):
        if t.dim() != 1 or t.shape[0] != nq + 1 or t.element_size() != 8 or not t.is_contiguous():
            raise ValueError("offsets must be contiguous (nq + 1,) tensors of 8-byte integers")
    if ids.element_size() != 4 or not ids.is_contiguous():
        raise ValueError("ids must be a contiguous tensor of 4-byte ids")
    if k_in_max is None:
        k_in_max = int((in_offsets[1:] - in_offsets[:-1]).max().item()) if nq > 0 else 1
    total = int(out_offsets[-1].item()) if nq > 0 else 0
    if out is None:
        oi = torch.empty(max(total, 1), dtype=torch.int32, device=ids.device)
        oa = torch.empty(max(total, 1), dtype=torch.float64, device=ids.device)
    else:
        oi, oa = out
    _check(load().mih_rerank_asym_csr(cptr, n, q, _ptr(proj), nq, _ptr(ids), _ptr(in_offsets), max(k_in_max, 1),
                                      _ptr(out_offsets), _ptr(oi), _ptr(oa), _stream(stream)), "mih_rerank_asym_csr")
    return {"ids": oi[:total], "a": oa[:total]}


def mih_knn_asym(index, codes, queries, proj, k: int, k_candidates: int, stream=None):
    """The Hamming k_candidates-NN of each query by mih_knn, re-ranked by
    mih_rerank_asym to k results: the two calls in sequence."""
    r = mih_knn(index, queries, k_candidates, stream=stream)
    return mih_rerank_asym(codes, index.q, proj, r["ids"], k, stream=stream)


def linscan_knn_noalloc(codes, q: int, queries, k: int, stream=None, out=None):
    """linscan_knn with a uniform k that allocates no device memory (nq, k <= 256).

    For callers that cannot allocate during a search; the library's fixed
    scratch array is shared by all calls on a device, so calls must not
    overlap on the GPU."""
    import torch

    cptr, n = _codes_arg(codes, q)
    qptr, nq = _codes_arg(queries, q)
    if out is None:
        ids = torch.empty((nq, k), dtype=torch.int32, device=queries.device)
        dist = torch.empty((nq, k), dtype=torch.int32, device=queries.device)
    else:
        ids, dist = out
    _check(load().linscan_knn_noalloc(cptr, n, q, qptr, nq, k, _ptr(ids), _ptr(dist), _stream(stream)),
           "linscan_knn_noalloc")
    return {"ids": ids, "dist": dist}
