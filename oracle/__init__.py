"""CPU oracle for the COBS query path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, single-threaded C++ (``cobs_oracle.cpp``) that restates the
method of Bingmann et al., "COBS: a Compact Bit-Sliced Signature Index"
(arXiv:1905.09624), Sec. 2.1-2.3, step by step.  Only the tests, the smoke
check and the benchmark's CPU-baseline leg load it.  The CUDA library never
imports, links or calls anything here; the two share no code.

Parity status of each function (what pins it, besides itself):
  xxh64          libxxhash known answers (ctypes, test time) and the spec's
                 published hash of the empty input.
  terms          brute force over all 4^k strings for small k; reverse complement
                 checked against string reversal and base complement.
  bloom_width    the Sec. 2.1 bound evaluated at the returned width (<= p) and at
                 width-1 (> p); the w/v ratios for (h=1,p=0.3) and (h=3,p=0.1).
  plan/build     exact mode (identity hash, w >= 4^k): the index becomes an exact
                 inverted index and scores equal brute-force containment.
  query          exact mode as above; no false negatives with XXH64; classic equals
                 compact with one block; false-positive score statistics against the
                 binomial law of Theorem 1; generated corpora (exact mode equals
                 brute-force containment, XXH64 scores never below it).
  binom_tail_ge  the paper's worked example (l=70, p=0.3, K=0.5 -> 0.000143) and
                 exact rational sums on small cases; Chernoff bound >= tail.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lib = None

HASH_XXH64 = 0
HASH_IDENTITY = 1


class Params(ctypes.Structure):
    _fields_ = [("term_kind", ctypes.c_uint32), ("q", ctypes.c_uint32), ("num_hashes", ctypes.c_uint32),
                ("hash_kind", ctypes.c_uint32), ("fpr", ctypes.c_double), ("block_docs", ctypes.c_uint64),
                ("width_override", ctypes.c_uint64)]


class Block(ctypes.Structure):
    _fields_ = [("n_docs", ctypes.c_uint64), ("doc_begin", ctypes.c_uint64), ("w", ctypes.c_uint64),
                ("rowbytes", ctypes.c_uint64), ("row_offset", ctypes.c_uint64), ("max_terms", ctypes.c_uint64)]


def _L():
    global _lib
    if _lib is None:
        build_lib()
        L = ctypes.CDLL(_LIB)
        vp, u64, u32, dbl = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double
        L.orc_xxh64.restype = u64
        L.orc_xxh64.argtypes = [vp, u64, u64]
        L.orc_terms.restype = u64
        L.orc_terms.argtypes = [vp, u64, u32, u32, vp, u64]
        L.orc_distinct_terms.restype = u64
        L.orc_distinct_terms.argtypes = [vp, u64, u32, u32, vp, u64]
        L.orc_hash_term.restype = u64
        L.orc_hash_term.argtypes = [u64, u32]
        L.orc_bloom_width.restype = u64
        L.orc_bloom_width.argtypes = [u32, u64, dbl]
        L.orc_doc_counts.restype = None
        L.orc_doc_counts.argtypes = [vp, vp, u64, u64, u32, u32, vp]
        L.orc_plan.restype = ctypes.c_int
        L.orc_plan.argtypes = [ctypes.POINTER(Params), vp, u64, ctypes.POINTER(vp)]
        L.orc_fill_columns.restype = ctypes.c_int
        L.orc_fill_columns.argtypes = [vp, vp, vp, u64, u64, u64]
        L.orc_build.restype = ctypes.c_int
        L.orc_build.argtypes = [ctypes.POINTER(Params), vp, vp, u64, ctypes.POINTER(vp)]
        L.orc_index_free.argtypes = [vp]
        L.orc_index_n_blocks.restype = u64
        L.orc_index_n_blocks.argtypes = [vp]
        L.orc_index_n_docs.restype = u64
        L.orc_index_n_docs.argtypes = [vp]
        L.orc_index_block.argtypes = [vp, u64, ctypes.POINTER(Block)]
        L.orc_index_perm.restype = vp
        L.orc_index_perm.argtypes = [vp]
        L.orc_index_nterms.restype = vp
        L.orc_index_nterms.argtypes = [vp]
        L.orc_index_rows.restype = vp
        L.orc_index_rows.argtypes = [vp]
        L.orc_index_rows_bytes.restype = u64
        L.orc_index_rows_bytes.argtypes = [vp]
        L.orc_scores.restype = u64
        L.orc_scores.argtypes = [vp, vp, u64, vp]
        L.orc_query.restype = u64
        L.orc_query.argtypes = [vp, vp, u64, u32, ctypes.POINTER(u64), ctypes.POINTER(u64), vp, vp, u64]
        L.orc_exact_scores.restype = u64
        L.orc_exact_scores.argtypes = [vp, vp, u64, u32, u32, vp, u64, vp]
        for f in ("orc_binom_tail_ge", "orc_binom_pmf"):
            getattr(L, f).restype = dbl
            getattr(L, f).argtypes = [u64, dbl, u64]
        L.orc_chernoff.restype = dbl
        L.orc_chernoff.argtypes = [u64, dbl, dbl]
        L.orc_bloom_fpr.restype = dbl
        L.orc_bloom_fpr.argtypes = [u32, u64, u64]
        L.orc_bloom_fpr_bound.restype = dbl
        L.orc_bloom_fpr_bound.argtypes = [u32, u64, u64]
        _lib = L
    return _lib


def _buf(b):
    if isinstance(b, (bytes, bytearray)):
        a = np.frombuffer(bytes(b), dtype=np.uint8)
    else:
        a = np.ascontiguousarray(b)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def xxh64(data: bytes, seed: int) -> int:
    a, p = _buf(data)
    return int(_L().orc_xxh64(p, len(a), seed))


def terms(s: bytes, kind: int, q: int) -> np.ndarray:
    a, p = _buf(s)
    cap = max(len(a), 1)
    out = np.empty(cap, dtype=np.uint64)
    n = _L().orc_terms(p, len(a), kind, q, out.ctypes.data_as(ctypes.c_void_p), cap)
    return out[:n].copy()


def distinct_terms(s: bytes, kind: int, q: int) -> np.ndarray:
    a, p = _buf(s)
    cap = max(len(a), 1)
    out = np.empty(cap, dtype=np.uint64)
    n = _L().orc_distinct_terms(p, len(a), kind, q, out.ctypes.data_as(ctypes.c_void_p), cap)
    return out[:n].copy()


def hash_term(t: int, i: int) -> int:
    return int(_L().orc_hash_term(t, i))


def bloom_width(h: int, v: int, p: float) -> int:
    return int(_L().orc_bloom_width(h, v, p))


def binom_tail_ge(l, p, t):
    return float(_L().orc_binom_tail_ge(l, p, t))


def binom_pmf(l, p, i):
    return float(_L().orc_binom_pmf(l, p, i))


def chernoff(l, K, p):
    return float(_L().orc_chernoff(l, K, p))


def bloom_fpr(h, v, w):
    return float(_L().orc_bloom_fpr(h, v, w))


def bloom_fpr_bound(h, v, w):
    return float(_L().orc_bloom_fpr_bound(h, v, w))


def make_params(term_kind=0, q=31, num_hashes=1, fpr=0.3, block_docs=0, hash_kind=HASH_XXH64, width_override=0,
                **_ignored):
    return Params(term_kind, q, num_hashes, hash_kind, fpr, block_docs, width_override)


class Index:
    """An oracle index (block table, permutation, row bytes)."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_index_free(self._h)
            self._h = None

    @property
    def n_docs(self):
        return int(_L().orc_index_n_docs(self._h))

    def blocks(self):
        out = []
        for b in range(int(_L().orc_index_n_blocks(self._h))):
            blk = Block()
            _L().orc_index_block(self._h, b, ctypes.byref(blk))
            out.append({k: int(getattr(blk, k)) for k, _ in Block._fields_})
        return out

    def perm(self):
        n = self.n_docs
        p = _L().orc_index_perm(self._h)
        return np.ctypeslib.as_array(ctypes.cast(p, ctypes.POINTER(ctypes.c_uint64)), shape=(n,)).copy() \
            if n else np.zeros(0, np.uint64)

    def nterms(self):
        n = self.n_docs
        p = _L().orc_index_nterms(self._h)
        return np.ctypeslib.as_array(ctypes.cast(p, ctypes.POINTER(ctypes.c_uint64)), shape=(n,)).copy() \
            if n else np.zeros(0, np.uint64)

    def rows_view(self):
        nb = int(_L().orc_index_rows_bytes(self._h))
        if nb == 0:
            return np.zeros(0, np.uint8)
        p = _L().orc_index_rows(self._h)
        return np.ctypeslib.as_array(ctypes.cast(p, ctypes.POINTER(ctypes.c_uint8)), shape=(nb,))

    def rows(self):
        return self.rows_view().copy()

    def fill_columns(self, docs, doc_off, blk, j0, j1):
        _, pd = _buf(docs)
        _, po = _buf(doc_off)
        rc = _L().orc_fill_columns(self._h, pd, po, blk, j0, j1)
        assert rc == 0

    def scores(self, query: bytes):
        out = np.empty(self.n_docs, dtype=np.uint32)
        a, p = _buf(query)
        l = _L().orc_scores(self._h, p, len(a), out.ctypes.data_as(ctypes.c_void_p))
        return int(l), out

    def query(self, query: bytes, thr_permille: int):
        """Returns (l, min_score, ids, scores) with hits sorted by (score desc, id asc)."""
        a, p = _buf(query)
        n = self.n_docs
        ids = np.empty(max(n, 1), dtype=np.uint32)
        sc = np.empty(max(n, 1), dtype=np.uint32)
        ell = ctypes.c_uint64()
        mn = ctypes.c_uint64()
        k = _L().orc_query(self._h, p, len(a), thr_permille, ctypes.byref(ell), ctypes.byref(mn),
                           ids.ctypes.data_as(ctypes.c_void_p), sc.ctypes.data_as(ctypes.c_void_p), n)
        return int(ell.value), int(mn.value), ids[:k].copy(), sc[:k].copy()


def build_lib() -> str:
    """Compile the oracle (g++ -O2, portable flags only)."""
    src = os.path.join(_HERE, "cobs_oracle.cpp")
    os.makedirs(_LIBDIR, exist_ok=True)
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, src])
        os.replace(tmp, _LIB)
    return _LIB


def build_index(params: Params, docs, doc_off) -> Index:
    """Single-threaded oracle build (counts, plan, bits)."""
    _, pd = _buf(docs)
    _, po = _buf(doc_off)
    h = ctypes.c_void_p()
    rc = _L().orc_build(ctypes.byref(params), pd, po, len(doc_off) - 1, ctypes.byref(h))
    if rc != 0:
        raise ValueError("oracle build rejected the parameters")
    return Index(h.value)


def doc_counts(docs, doc_off, d0, d1, kind, q):
    _, pd = _buf(docs)
    _, po = _buf(doc_off)
    out = np.empty(max(d1 - d0, 1), dtype=np.uint64)
    _L().orc_doc_counts(pd, po, d0, d1, kind, q, out.ctypes.data_as(ctypes.c_void_p))
    return out[:d1 - d0]


def plan(params: Params, v) -> Index:
    v = np.ascontiguousarray(v, dtype=np.uint64)
    h = ctypes.c_void_p()
    rc = _L().orc_plan(ctypes.byref(params), v.ctypes.data_as(ctypes.c_void_p), len(v), ctypes.byref(h))
    if rc != 0:
        raise ValueError("oracle plan rejected the parameters")
    return Index(h.value)


def doc_counts_threaded(params: Params, docs, doc_off, nthreads=None):
    """Distinct-term counts of every document: doc_counts on disjoint document
    ranges from several Python threads (ctypes drops the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    n = len(doc_off) - 1
    nthreads = nthreads or os.cpu_count() or 1
    v = np.empty(n, dtype=np.uint64)
    step = max(1, (n + 4 * nthreads - 1) // (4 * nthreads))
    ranges = [(a, min(n, a + step)) for a in range(0, n, step)]
    with ThreadPoolExecutor(nthreads) as ex:
        for (a, b), res in zip(ranges, ex.map(lambda r: doc_counts(docs, doc_off, r[0], r[1],
                                                                   params.term_kind, params.q), ranges)):
            v[a:b] = res
    return v


def fill_threaded(ix: Index, docs, doc_off, blocks=None, nthreads=None):
    """Bloom bits of the given blocks (all by default): fill_columns on disjoint
    column ranges (multiples of 8, so disjoint bytes) from several threads."""
    from concurrent.futures import ThreadPoolExecutor
    nthreads = nthreads or os.cpu_count() or 1
    all_blocks = ix.blocks()
    jobs = []
    for bi in (range(len(all_blocks)) if blocks is None else blocks):
        nb = all_blocks[bi]["n_docs"]
        cstep = max(8, ((nb + 4 * nthreads - 1) // (4 * nthreads) + 7) // 8 * 8)
        jobs += [(bi, j, min(nb, j + cstep)) for j in range(0, nb, cstep)]
    with ThreadPoolExecutor(nthreads) as ex:
        list(ex.map(lambda jb: ix.fill_columns(docs, doc_off, *jb), jobs))


def build_index_threaded(params: Params, docs, doc_off, nthreads=None) -> Index:
    """The same oracle functions as build_index, called on disjoint document and
    column ranges from several Python threads (ctypes drops the GIL), so a large
    oracle index is ready in seconds.  Each call is the single-threaded oracle."""
    ix = plan(params, doc_counts_threaded(params, docs, doc_off, nthreads))
    fill_threaded(ix, docs, doc_off, None, nthreads)
    return ix


def exact_scores(docs, doc_off, kind, q, query: bytes):
    _, pd = _buf(docs)
    _, po = _buf(doc_off)
    a, p = _buf(query)
    n = len(doc_off) - 1
    out = np.empty(max(n, 1), dtype=np.uint32)
    l = _L().orc_exact_scores(pd, po, n, kind, q, p, len(a), out.ctypes.data_as(ctypes.c_void_p))
    return int(l), out[:n]
