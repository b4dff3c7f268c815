"""Thin ctypes binding of libcobs_gpu.so (include/cobs_gpu.h), same names.

Argument marshalling only: every step of the query path runs in the CUDA
library.  There is no fallback: importing this module without a loadable
library raises.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

from . import _build

COBS_OK = 0
COBS_PENDING = 1
COBS_ERR_ARG = -1
COBS_ERR_OOM = -2
COBS_ERR_CUDA = -3
COBS_ERR_TIMEOUT = -4
COBS_ERR_BUDGET = -5
COBS_ERR_FORMAT = -6
COBS_ERR_OVERFLOW = -7
COBS_ERR_NOT_FOUND = -8
COBS_ERR_CANCELLED = -9

ABI_VERSION = 4  # COBS_GPU_ABI_VERSION of include/cobs_gpu.h that the structs below mirror

COBS_PLAIN = 1
COBS_BATCHED = 2
COBS_GRAPH = 4

u8p = ctypes.POINTER(ctypes.c_uint8)
u16p = ctypes.POINTER(ctypes.c_uint16)
u32p = ctypes.POINTER(ctypes.c_uint32)
u64p = ctypes.POINTER(ctypes.c_uint64)
vp = ctypes.c_void_p


class cobs_params(ctypes.Structure):
    _fields_ = [("term_kind", ctypes.c_uint32), ("q", ctypes.c_uint32), ("num_hashes", ctypes.c_uint32),
                ("score_bits", ctypes.c_uint32), ("fpr", ctypes.c_double), ("block_docs", ctypes.c_uint64),
                ("width", ctypes.c_uint64)]


class cobs_block_info(ctypes.Structure):
    _fields_ = [("n_docs", ctypes.c_uint64), ("doc_begin", ctypes.c_uint64), ("w", ctypes.c_uint64),
                ("rowbytes", ctypes.c_uint64), ("row_offset", ctypes.c_uint64), ("max_terms", ctypes.c_uint64)]


class cobs_hits(ctypes.Structure):
    _fields_ = [("n_terms", ctypes.c_uint32), ("min_score", ctypes.c_uint32), ("n_hits", ctypes.c_uint32),
                ("_pad", ctypes.c_uint32), ("doc_ids", u32p), ("scores", u32p)]


class cobs_result(ctypes.Structure):
    _fields_ = [("n_queries", ctypes.c_uint64), ("hits", ctypes.POINTER(cobs_hits))]


class cobs_engine_cfg(ctypes.Structure):
    _fields_ = [("max_queries", ctypes.c_uint64), ("max_query_bytes", ctypes.c_uint64), ("max_hits", ctypes.c_uint64),
                ("slice_bytes", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32), ("l2_hints", ctypes.c_uint32),
                ("split", ctypes.c_uint32), ("stage_bytes", ctypes.c_uint64), ("gather_feed", ctypes.c_uint32),
                ("split_part", ctypes.c_uint32), ("class_streams", ctypes.c_uint32),
                ("tuned_from_cache", ctypes.c_uint32)]


class cobs_query_stats(ctypes.Structure):
    _fields_ = [("ms_terms", ctypes.c_double), ("ms_gather", ctypes.c_double), ("ms_hits", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("row_bytes", ctypes.c_uint64), ("terms", ctypes.c_uint64),
                ("n_tiles", ctypes.c_uint64), ("gather_launches", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("slice_bytes", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32), ("l2_hints", ctypes.c_uint32),
                ("split_queries", ctypes.c_uint32), ("ms_host", ctypes.c_double),
                ("h2d_index_bytes", ctypes.c_uint64), ("split_part", ctypes.c_uint32),
                ("stream_numa_node", ctypes.c_int32)]


class cobs_serve_cfg(ctypes.Structure):
    _fields_ = [("score_budget_bytes", ctypes.c_uint64), ("max_inflight_waves", ctypes.c_uint32),
                ("max_wave_queries", ctypes.c_uint32), ("wait_timeout_ms", ctypes.c_uint32),
                ("form", ctypes.c_uint32)]


class cobs_serve_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("waves", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("qps", ctypes.c_double), ("seconds", ctypes.c_double), ("mean_wave_queries", ctypes.c_double),
                ("mean_wave_ms", ctypes.c_double), ("max_wave_ms", ctypes.c_double),
                ("cancelled", ctypes.c_uint64), ("failed", ctypes.c_uint64)]


_PROTOS = {
    "cobs_build_device": (ctypes.c_int, [ctypes.POINTER(cobs_params), vp, vp, ctypes.c_uint64, ctypes.c_int, vp,
                                         ctypes.POINTER(vp)]),
    "cobs_build_device_resident": (ctypes.c_int, [ctypes.POINTER(cobs_params), vp, vp, vp, ctypes.c_uint64, vp,
                                                  ctypes.POINTER(vp)]),
    "cobs_build": (ctypes.c_int, [ctypes.POINTER(cobs_params), vp, vp, ctypes.c_uint64, ctypes.POINTER(vp)]),
    "cobs_device_index_download": (ctypes.c_int, [vp, ctypes.POINTER(vp)]),
    "cobs_load_device": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.POINTER(vp)]),
    "cobs_load_device_streamed": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.POINTER(vp)]),
    "cobs_multi_index_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_uint64, ctypes.POINTER(vp)]),
    "cobs_index_merge": (ctypes.c_int, [vp, vp, ctypes.POINTER(vp)]),
    "cobs_index_insert": (ctypes.c_int, [vp, vp, vp, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(vp)]),
    "cobs_shard_plan": (ctypes.c_int, [vp, ctypes.c_uint32, vp, vp]),
    "cobs_index_shard": (ctypes.c_int, [vp, vp, ctypes.c_uint32, ctypes.POINTER(vp), vp, u64p]),
    "cobs_hits_merge": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint64, vp, vp, vp, vp, vp, vp, vp]),
    "cobs_index_save": (ctypes.c_int, [vp, ctypes.c_char_p]),
    "cobs_index_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(vp)]),
    "cobs_index_info": (ctypes.c_int, [vp, ctypes.POINTER(cobs_params), u64p, u64p,
                                       ctypes.POINTER(ctypes.POINTER(cobs_block_info)), ctypes.POINTER(u64p),
                                       ctypes.POINTER(u64p), ctypes.POINTER(u8p), u64p]),
    "cobs_device_index_info": (ctypes.c_int, [vp, ctypes.POINTER(cobs_params), u64p, u64p,
                                              ctypes.POINTER(ctypes.POINTER(cobs_block_info)), ctypes.POINTER(vp),
                                              u64p]),
    "cobs_index_free": (None, [vp]),
    "cobs_device_index_free": (None, [vp]),
    "cobs_query_batch": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_uint64, ctypes.c_uint32, vp,
                                        ctypes.POINTER(ctypes.POINTER(cobs_result))]),
    "cobs_result_free": (None, [ctypes.POINTER(cobs_result)]),
    "cobs_engine_create": (ctypes.c_int, [vp, ctypes.POINTER(cobs_engine_cfg), vp, ctypes.POINTER(vp)]),
    "cobs_engine_free": (None, [vp]),
    "cobs_engine_query_device": (ctypes.c_int, [vp, vp, vp, vp, vp, ctypes.c_uint64, ctypes.c_uint32]),
    "cobs_engine_query_host": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_uint64, ctypes.c_uint32,
                                              ctypes.POINTER(ctypes.POINTER(cobs_result))]),
    "cobs_engine_submit_host": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_uint64, ctypes.c_uint32]),
    "cobs_engine_results_device": (ctypes.c_int, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                                  ctypes.POINTER(vp), ctypes.POINTER(vp)]),
    "cobs_engine_download": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.POINTER(cobs_result))]),
    "cobs_engine_stats": (ctypes.c_int, [vp, ctypes.POINTER(cobs_query_stats)]),
    "cobs_engine_autotune": (ctypes.c_int, [vp, vp, vp, vp, vp, ctypes.c_uint64, ctypes.POINTER(cobs_engine_cfg)]),
    "cobs_serve_start": (ctypes.c_int, [vp, ctypes.POINTER(cobs_serve_cfg), ctypes.POINTER(vp)]),
    "cobs_serve_submit": (ctypes.c_int, [vp, vp, ctypes.c_uint64, ctypes.c_uint16, u64p]),
    "cobs_serve_poll": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.POINTER(cobs_hits)]),
    "cobs_serve_cancel": (ctypes.c_int, [vp, ctypes.c_uint64]),
    "cobs_hits_release": (None, [vp, ctypes.c_uint64]),
    "cobs_serve_stop": (ctypes.c_int, [vp, ctypes.POINTER(cobs_serve_stats)]),
    "cobs_query_one_noalloc": (ctypes.c_int, [vp, vp, ctypes.c_uint64, ctypes.c_uint16, vp, vp, vp,
                                              ctypes.c_uint64, vp]),
    "cobs_probe_l2_read": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, vp, vp]),
    "cobs_debug_barrett_mod": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_uint64, vp, vp]),
    "cobs_last_error": (ctypes.c_char_p, []),
    "cobs_bloom_width": (ctypes.c_uint64, [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double]),
    "cobs_version": (ctypes.c_char_p, []),
    "cobs_abi_version": (ctypes.c_uint32, []),
    "cobs_debug_fail_alloc": (None, [ctypes.c_int64]),
    "cobs_debug_build_scratch": (None, [ctypes.c_uint64]),
}

# the serve loop's entry points, also exported by a host-only scheduler build
SERVE_PROTOS = {k: _PROTOS[k] for k in ("cobs_serve_submit", "cobs_serve_poll", "cobs_serve_cancel",
                                        "cobs_hits_release", "cobs_serve_stop", "cobs_last_error")}

_lib = None


def lib(build: bool = True, path: str | None = None):
    """Load libcobs_gpu.so (building it first when `build`); `path` loads another
    build of the library instead (it must be the first call)."""
    global _lib
    if _lib is None:
        if path is None:
            path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libcobs_gpu.so not found at {path}; run the build first")
        L = ctypes.CDLL(path)
        for name, (res, args) in _PROTOS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        if L.cobs_abi_version() != ABI_VERSION:  # the structs above mirror one version of the header
            raise RuntimeError(f"{path} has ABI version {L.cobs_abi_version()}, this binding expects "
                               f"{ABI_VERSION}: rebuild the library")
        _lib = L
    return _lib


class CobsError(RuntimeError):
    def __init__(self, status, where, msg=None):
        if msg is None:
            msg = lib().cobs_last_error().decode(errors="replace")
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


def check(status, where):
    if status != COBS_OK:
        raise CobsError(status, where)
    return status


def _ptr(a):
    """Host numpy array or torch tensor -> address."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def make_params(term_kind=0, q=31, num_hashes=1, fpr=0.3, block_docs=0, score_bits=32, width=0, **_ignored):
    return cobs_params(term_kind, q, num_hashes, score_bits, fpr, block_docs, width)


def result_to_python(res_ptr):
    """Copy a cobs_result into [(n_terms, min_score, ids np.uint32, scores np.uint32)] and free it."""
    res = res_ptr.contents
    out = []
    for i in range(res.n_queries):
        h = res.hits[i]
        n = h.n_hits
        ids = np.ctypeslib.as_array(h.doc_ids, shape=(n,)).copy() if n else np.zeros(0, np.uint32)
        sc = np.ctypeslib.as_array(h.scores, shape=(n,)).copy() if n else np.zeros(0, np.uint32)
        out.append((h.n_terms, h.min_score, ids, sc))
    lib().cobs_result_free(res_ptr)
    return out


_HITS_DT = np.dtype([("n_terms", "<u4"), ("min_score", "<u4"), ("n_hits", "<u4"), ("_pad", "<u4"),
                     ("doc_ids", "<u8"), ("scores", "<u8")])


def result_to_arrays(res_ptr):
    """Copy a cobs_result into flat arrays (n_terms, min_score, hit_offsets[n+1],
    ids, scores) and free it.  The hits of all queries are contiguous in query
    order inside a result, so two copies suffice."""
    res = res_ptr.contents
    n = res.n_queries
    if n == 0:
        lib().cobs_result_free(res_ptr)
        z = np.zeros(0, np.uint32)
        return z, z, np.zeros(1, np.uint64), z, z
    raw = (ctypes.c_char * (32 * n)).from_address(ctypes.addressof(res.hits.contents))
    h = np.frombuffer(raw, dtype=_HITS_DT).copy()
    off = np.zeros(n + 1, np.uint64)
    np.cumsum(h["n_hits"], out=off[1:])
    total = int(off[-1])
    if total:
        first = int(np.argmax(h["n_hits"] > 0))
        base_ids = int(h["doc_ids"][first]) - 4 * int(off[first])
        base_sc = int(h["scores"][first]) - 4 * int(off[first])
        ids = np.frombuffer((ctypes.c_char * (4 * total)).from_address(base_ids), np.uint32).copy()
        sc = np.frombuffer((ctypes.c_char * (4 * total)).from_address(base_sc), np.uint32).copy()
    else:
        ids = sc = np.zeros(0, np.uint32)
    lib().cobs_result_free(res_ptr)
    return h["n_terms"].copy(), h["min_score"].copy(), off, ids, sc


class _Owned:
    """Explicit release: close() (also on leaving a `with` block) frees the
    object now instead of when it is collected.  A device index refuses while an
    engine, a server or a multi-index view that uses it is still open."""

    def _depends_on(self, other):
        users = other.__dict__.setdefault("_users", weakref.WeakSet())
        users.add(self)

    def close(self):
        live = [u for u in self.__dict__.get("_users", ()) if getattr(u, "h", None)]
        if live:
            raise RuntimeError(f"close the {len(live)} object(s) using this {type(self).__name__} first")
        self.__del__()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


class HostIndex(_Owned):
    """cobs_index (host copy)."""

    def __init__(self, handle):
        self.h = vp(handle)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.cobs_index_free(self.h)
            self.h = None

    def info(self):
        P = cobs_params()
        nd, nb, rb = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        blocks = ctypes.POINTER(cobs_block_info)()
        perm, nterms = u64p(), u64p()
        rows = u8p()
        check(lib().cobs_index_info(self.h, ctypes.byref(P), ctypes.byref(nd), ctypes.byref(nb), ctypes.byref(blocks),
                                    ctypes.byref(perm), ctypes.byref(nterms), ctypes.byref(rows), ctypes.byref(rb)),
              "cobs_index_info")
        n = nd.value
        bl = [{k: int(getattr(blocks[i], k)) for k, _ in cobs_block_info._fields_} for i in range(nb.value)]
        arr = lambda p, m: np.ctypeslib.as_array(p, shape=(m,)).copy() if m else np.zeros(0, np.uint64)  # noqa: E731
        rows_np = np.ctypeslib.as_array(rows, shape=(rb.value,)).copy() if rb.value else np.zeros(0, np.uint8)
        return dict(params=P, n_docs=n, blocks=bl, perm=arr(perm, n), nterms=arr(nterms, n), rows=rows_np)

    def save(self, path):
        check(lib().cobs_index_save(self.h, path.encode()), "cobs_index_save")

    @staticmethod
    def load(path):
        h = vp()
        check(lib().cobs_index_load(path.encode(), ctypes.byref(h)), "cobs_index_load")
        return HostIndex(h.value)

    def insert(self, docs, doc_off, device=0):
        """cobs_index_insert: a new index with documents added (ids after self's)."""
        docs = np.ascontiguousarray(docs, dtype=np.uint8)
        doc_off = np.ascontiguousarray(doc_off, dtype=np.uint64)
        h = vp()
        check(lib().cobs_index_insert(self.h, _ptr(docs) if len(docs) else None, _ptr(doc_off), len(doc_off) - 1,
                                      device, ctypes.byref(h)), "cobs_index_insert")
        return HostIndex(h.value)

    def shard_plan(self, n_shards):
        """cobs_shard_plan: (block -> shard array, bytes per shard)."""
        nb = len(self.info()["blocks"])
        bs = np.zeros(max(nb, 1), np.uint32)
        sb = np.zeros(n_shards, np.uint64)
        check(lib().cobs_shard_plan(self.h, n_shards, _ptr(bs), _ptr(sb)), "cobs_shard_plan")
        return bs[:nb], sb

    def shard(self, block_shard, shard):
        """cobs_index_shard: (shard index, ids in this index of its documents)."""
        bs = np.ascontiguousarray(block_shard, dtype=np.uint32)
        gids = np.zeros(max(self.info()["n_docs"], 1), np.uint64)
        n = ctypes.c_uint64()
        h = vp()
        check(lib().cobs_index_shard(self.h, _ptr(bs), shard, ctypes.byref(h), _ptr(gids), ctypes.byref(n)),
              "cobs_index_shard")
        return HostIndex(h.value), gids[:n.value].copy()

    def merge(self, other):
        """cobs_index_merge: self's documents, then other's (ids shifted by self's count)."""
        h = vp()
        check(lib().cobs_index_merge(self.h, other.h, ctypes.byref(h)), "cobs_index_merge")
        return HostIndex(h.value)


class DeviceIndex(_Owned):
    """cobs_device_index (resident in HBM)."""

    def __init__(self, handle):
        self.h = vp(handle)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.cobs_device_index_free(self.h)
            self.h = None

    @staticmethod
    def build(params, docs, doc_off, device=0, stream=None):
        docs = np.ascontiguousarray(docs, dtype=np.uint8)
        doc_off = np.ascontiguousarray(doc_off, dtype=np.uint64)
        h = vp()
        check(lib().cobs_build_device(ctypes.byref(params), _ptr(docs), _ptr(doc_off), len(doc_off) - 1, device,
                                      stream, ctypes.byref(h)), "cobs_build_device")
        return DeviceIndex(h.value)

    @staticmethod
    def build_resident(params, docs_dev, doc_off_dev, doc_off_host, stream=None):
        h = vp()
        doc_off_host = np.ascontiguousarray(doc_off_host, dtype=np.uint64)
        check(lib().cobs_build_device_resident(ctypes.byref(params), _ptr(docs_dev), _ptr(doc_off_dev),
                                               _ptr(doc_off_host), len(doc_off_host) - 1, stream, ctypes.byref(h)),
              "cobs_build_device_resident")
        return DeviceIndex(h.value)

    @staticmethod
    def load(host_index: HostIndex, device=0, stream=None):
        h = vp()
        check(lib().cobs_load_device(host_index.h, device, stream, ctypes.byref(h)), "cobs_load_device")
        return DeviceIndex(h.value)

    @staticmethod
    def multi(parts):
        """cobs_multi_index_create: one index over several resident ones (borrowed rows)."""
        arr = (vp * len(parts))(*[p.h for p in parts])
        h = vp()
        check(lib().cobs_multi_index_create(arr, len(parts), ctypes.byref(h)), "cobs_multi_index_create")
        view = DeviceIndex(h.value)
        view._parts = list(parts)  # the view borrows their rows
        for p in parts:
            view._depends_on(p)
        return view

    @staticmethod
    def load_streamed(host_index: HostIndex, device=0, stream=None):
        """cobs_load_device_streamed: rows in pinned host memory, streamed per batch."""
        h = vp()
        check(lib().cobs_load_device_streamed(host_index.h, device, stream, ctypes.byref(h)),
              "cobs_load_device_streamed")
        return DeviceIndex(h.value)

    def download(self) -> HostIndex:
        h = vp()
        check(lib().cobs_device_index_download(self.h, ctypes.byref(h)), "cobs_device_index_download")
        return HostIndex(h.value)

    def info(self):
        P = cobs_params()
        nd, nb, rb = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        blocks = ctypes.POINTER(cobs_block_info)()
        rows = vp()
        check(lib().cobs_device_index_info(self.h, ctypes.byref(P), ctypes.byref(nd), ctypes.byref(nb),
                                           ctypes.byref(blocks), ctypes.byref(rows), ctypes.byref(rb)),
              "cobs_device_index_info")
        bl = [{k: int(getattr(blocks[i], k)) for k, _ in cobs_block_info._fields_} for i in range(nb.value)]
        return dict(params=P, n_docs=nd.value, blocks=bl, rows_dev=rows.value, rows_bytes=rb.value)

    def query(self, queries, q_off, thr, flags=COBS_BATCHED, stream=None):
        """cobs_query_batch with host buffers; returns a list per query."""
        queries = np.ascontiguousarray(queries, dtype=np.uint8)
        q_off = np.ascontiguousarray(q_off, dtype=np.uint64)
        thr = np.ascontiguousarray(thr, dtype=np.uint16)
        res = ctypes.POINTER(cobs_result)()
        check(lib().cobs_query_batch(self.h, _ptr(queries), _ptr(q_off), _ptr(thr), len(q_off) - 1, flags, stream,
                                     ctypes.byref(res)), "cobs_query_batch")
        return result_to_python(res)


class Engine(_Owned):
    """cobs_engine: reusable query workspace on one device index."""

    def __init__(self, dix: DeviceIndex, stream=None, slice_bytes=0, ctas_per_sm=0, max_hits=0, l2_hints=0, split=0,
                 stage_bytes=0, gather_feed=0, split_part=0, class_streams=0):
        self.dix = dix
        self._depends_on(dix)
        cfg = cobs_engine_cfg(0, 0, max_hits, slice_bytes, ctas_per_sm, l2_hints, split, stage_bytes, gather_feed,
                              split_part, class_streams, 0)
        h = vp()
        check(lib().cobs_engine_create(dix.h, ctypes.byref(cfg), stream, ctypes.byref(h)), "cobs_engine_create")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.cobs_engine_free(self.h)
            self.h = None

    def query_device(self, q_dev, off_dev, off_host, thr_dev, flags=COBS_BATCHED):
        off_host = np.ascontiguousarray(off_host, dtype=np.uint64)
        self._off_host = off_host  # keep alive for a possible re-run
        check(lib().cobs_engine_query_device(self.h, _ptr(q_dev), _ptr(off_dev), _ptr(off_host), _ptr(thr_dev),
                                             len(off_host) - 1, flags), "cobs_engine_query_device")

    def query_host(self, queries, q_off, thr, flags=COBS_BATCHED):
        queries = np.ascontiguousarray(queries, dtype=np.uint8)
        q_off = np.ascontiguousarray(q_off, dtype=np.uint64)
        thr = np.ascontiguousarray(thr, dtype=np.uint16)
        res = ctypes.POINTER(cobs_result)()
        check(lib().cobs_engine_query_host(self.h, _ptr(queries), _ptr(q_off), _ptr(thr), len(q_off) - 1, flags,
                                           ctypes.byref(res)), "cobs_engine_query_host")
        return result_to_python(res)

    def submit_host(self, queries, q_off, thr, flags=COBS_BATCHED):
        """cobs_engine_submit_host: queue copies and query, return at once; collect
        with download / download_arrays.  Pinned query bytes must stay unchanged
        until then."""
        self._inputs = (np.ascontiguousarray(queries, dtype=np.uint8), np.ascontiguousarray(q_off, dtype=np.uint64),
                        np.ascontiguousarray(thr, dtype=np.uint16))  # kept alive until the next submit
        qb, qo, th = self._inputs
        check(lib().cobs_engine_submit_host(self.h, _ptr(qb), _ptr(qo), _ptr(th), len(qo) - 1, flags),
              "cobs_engine_submit_host")

    def query_host_arrays(self, queries, q_off, thr, flags=COBS_BATCHED):
        """cobs_engine_query_host, results as flat arrays (see result_to_arrays)."""
        res = ctypes.POINTER(cobs_result)()
        check(lib().cobs_engine_query_host(self.h, _ptr(queries), _ptr(q_off), _ptr(thr), len(q_off) - 1, flags,
                                           ctypes.byref(res)), "cobs_engine_query_host")
        return result_to_arrays(res)

    def download(self):
        res = ctypes.POINTER(cobs_result)()
        check(lib().cobs_engine_download(self.h, ctypes.byref(res)), "cobs_engine_download")
        return result_to_python(res)

    def download_arrays(self):
        res = ctypes.POINTER(cobs_result)()
        check(lib().cobs_engine_download(self.h, ctypes.byref(res)), "cobs_engine_download")
        return result_to_arrays(res)

    def results_device(self):
        ptrs = [vp() for _ in range(5)]
        check(lib().cobs_engine_results_device(self.h, *[ctypes.byref(p) for p in ptrs]), "cobs_engine_results_device")
        return [p.value for p in ptrs]

    def stats(self):
        st = cobs_query_stats()
        check(lib().cobs_engine_stats(self.h, ctypes.byref(st)), "cobs_engine_stats")
        return {k: getattr(st, k) for k, _ in cobs_query_stats._fields_}

    def autotune(self, q_dev, off_dev, off_host, thr_dev):
        off_host = np.ascontiguousarray(off_host, dtype=np.uint64)
        cfg = cobs_engine_cfg()
        check(lib().cobs_engine_autotune(self.h, _ptr(q_dev), _ptr(off_dev), _ptr(off_host), _ptr(thr_dev),
                                         len(off_host) - 1, ctypes.byref(cfg)), "cobs_engine_autotune")
        return dict(slice_bytes=cfg.slice_bytes, ctas_per_sm=cfg.ctas_per_sm, l2_hints=cfg.l2_hints, split=cfg.split,
                    split_part=cfg.split_part, class_streams=cfg.class_streams,
                    from_cache=bool(cfg.tuned_from_cache))


class Server(_Owned):
    """cobs_server: continuous-batching serve loop."""

    def __init__(self, dix: DeviceIndex, score_budget_bytes=0, max_inflight_waves=0, max_wave_queries=0,
                 wait_timeout_ms=0, form=0):
        self.dix = dix
        self._depends_on(dix)
        self._L = lib()
        cfg = cobs_serve_cfg(score_budget_bytes, max_inflight_waves, max_wave_queries, wait_timeout_ms, form)
        h = vp()
        check(self._L.cobs_serve_start(dix.h, ctypes.byref(cfg), ctypes.byref(h)), "cobs_serve_start")
        self.h = h

    @classmethod
    def attach(cls, library, handle):
        """Wrap a server handle made by another build of the serve entry points
        (same names and prototypes, e.g. a host-only scheduler build)."""
        self = cls.__new__(cls)
        self.dix, self._L, self.h = None, library, handle
        return self

    def _check(self, st, where):
        if st != COBS_OK:
            raise CobsError(st, where, self._L.cobs_last_error().decode(errors="replace"))

    def submit(self, q: bytes, thr: int) -> int:
        t = ctypes.c_uint64()
        buf = np.frombuffer(q, dtype=np.uint8) if len(q) else np.zeros(1, np.uint8)
        self._check(self._L.cobs_serve_submit(self.h, _ptr(buf), len(q), thr, ctypes.byref(t)), "cobs_serve_submit")
        return t.value

    def poll(self, ticket):
        """None while pending, else (n_terms, min_score, ids, scores) and the ticket
        is released; raises CobsError (with .status) on a failed or cancelled one."""
        h = cobs_hits()
        st = self._L.cobs_serve_poll(self.h, ticket, ctypes.byref(h))
        if st == COBS_PENDING:
            return None
        self._check(st, "cobs_serve_poll")
        n = h.n_hits
        ids = np.ctypeslib.as_array(h.doc_ids, shape=(n,)).copy() if n else np.zeros(0, np.uint32)
        sc = np.ctypeslib.as_array(h.scores, shape=(n,)).copy() if n else np.zeros(0, np.uint32)
        self._L.cobs_hits_release(self.h, ticket)
        return (h.n_terms, h.min_score, ids, sc)

    def cancel(self, ticket):
        self._check(self._L.cobs_serve_cancel(self.h, ticket), "cobs_serve_cancel")

    def release(self, ticket):
        self._L.cobs_hits_release(self.h, ticket)

    def stop(self):
        st = cobs_serve_stats()
        if getattr(self, "h", None):
            self._check(self._L.cobs_serve_stop(self.h, ctypes.byref(st)), "cobs_serve_stop")
            self.h = None
        return {k: getattr(st, k) for k, _ in cobs_serve_stats._fields_}

    def __del__(self):
        if getattr(self, "h", None) and getattr(self, "_L", None) is not None:
            self._L.cobs_serve_stop(self.h, None)
            self.h = None


def bloom_width(h, v, p):
    return int(lib().cobs_bloom_width(h, v, p))


def probe_l2_read(buf_ptr, nbytes, reps, sink_ptr, ctas_per_sm=0, stream=None):
    """cobs_probe_l2_read on a device buffer (pointers as integers); queued on `stream`."""
    check(lib().cobs_probe_l2_read(ctypes.c_void_p(buf_ptr), nbytes, reps, ctas_per_sm, ctypes.c_void_p(sink_ptr),
                                   ctypes.c_void_p(stream)), "cobs_probe_l2_read")


def debug_barrett_mod(x_ptr, n, w, out_ptr, stream=None):
    """cobs_debug_barrett_mod: out[i] = x[i] mod w on the device (pointers as integers)."""
    check(lib().cobs_debug_barrett_mod(ctypes.c_void_p(x_ptr), n, w, ctypes.c_void_p(out_ptr),
                                       ctypes.c_void_p(stream)), "cobs_debug_barrett_mod")


def hits_merge(shard_results, global_ids):
    """cobs_hits_merge of a batch: shard_results[s] = (hit_offsets, ids, scores)
    with shard-local ids (e.g. from download_arrays), global_ids[s] the shard's
    id map; returns (hit_offsets, ids, scores) in the order of the unsharded index."""
    n = len(shard_results)
    offs = [np.ascontiguousarray(r[0], dtype=np.uint64) for r in shard_results]
    ids = [np.ascontiguousarray(r[1], dtype=np.uint32) for r in shard_results]
    sc = [np.ascontiguousarray(r[2], dtype=np.uint32) for r in shard_results]
    gid = [np.ascontiguousarray(g, dtype=np.uint64) for g in global_ids]
    nq = len(offs[0]) - 1 if n else 0
    total = sum(int(o[-1] - o[0]) for o in offs)
    P = ctypes.c_void_p * max(n, 1)
    out_off = np.zeros(nq + 1, np.uint64)
    out_ids = np.zeros(max(total, 1), np.uint32)
    out_sc = np.zeros(max(total, 1), np.uint32)
    check(lib().cobs_hits_merge(n, nq, P(*[x.ctypes.data for x in offs]), P(*[x.ctypes.data for x in ids]),
                                P(*[x.ctypes.data for x in sc]), P(*[x.ctypes.data for x in gid]), _ptr(out_off),
                                _ptr(out_ids), _ptr(out_sc)), "cobs_hits_merge")
    return out_off, out_ids[:total].copy(), out_sc[:total].copy()
