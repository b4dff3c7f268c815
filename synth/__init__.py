"""Seeded synthetic workloads shaped like the paper's corpora (Sec. 3).

This module only draws inputs: documents, queries, thresholds and arrival
times.  It holds none of the index or query arithmetic, and both the CUDA
library and the CPU oracle consume the arrays it returns.

The paper's McCortex microbial documents and unitig-derived query sets
(Sec. 3, "Data" and "Queries") are not available; the five workloads below
stand in for them with the same shapes (document count, length distribution,
k, query lengths, thresholds).
"""
from __future__ import annotations

import ctypes
import json
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libsynth.so")
_lib = None

TERM_DNA_CANONICAL = 0
TERM_DNA_FORWARD = 1
TERM_BYTES = 2


def build() -> str:
    """Compile the generator library (plain C, portable: no -march flags)."""
    src = os.path.join(_HERE, "synth.c")
    os.makedirs(_LIBDIR, exist_ok=True)
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


u64 = ctypes.c_uint64


def lognormal_lengths(seed, n, median, sigma, lo, hi):
    out = np.empty(n, dtype=np.uint64)
    _L().synth_lengths_lognormal(u64(seed), u64(n), ctypes.c_double(median), ctypes.c_double(sigma),
                                 u64(lo), u64(hi), _p(out))
    return out


def _offsets(lengths):
    off = np.zeros(len(lengths) + 1, dtype=np.uint64)
    np.cumsum(lengths, out=off[1:])
    return off


def dna_docs(seed, lengths, nthreads=None):
    off = _offsets(np.asarray(lengths, dtype=np.uint64))
    out = np.empty(int(off[-1]), dtype=np.uint8)
    _L().synth_fill_dna(u64(seed), u64(len(lengths)), _p(off), _p(out),
                        ctypes.c_int(nthreads or os.cpu_count() or 1))
    return out, off


def vocab(seed, n_words, minlen=3, maxlen=12):
    off = np.zeros(n_words + 1, dtype=np.uint64)
    _L().synth_vocab(u64(seed), u64(n_words), ctypes.c_uint32(minlen), ctypes.c_uint32(maxlen), None, _p(off))
    words = np.empty(int(off[-1]), dtype=np.uint8)
    _L().synth_vocab(u64(seed), u64(n_words), ctypes.c_uint32(minlen), ctypes.c_uint32(maxlen), _p(words), _p(off))
    return words, off


def text_docs(seed, lengths, words, word_off, zipf_s=1.1, nthreads=None):
    n_words = len(word_off) - 1
    cdf = np.empty(n_words, dtype=np.float64)
    _L().synth_zipf_cdf(u64(n_words), ctypes.c_double(zipf_s), _p(cdf))
    off = _offsets(np.asarray(lengths, dtype=np.uint64))
    out = np.empty(int(off[-1]), dtype=np.uint8)
    _L().synth_fill_text(u64(seed), u64(len(lengths)), _p(off), _p(words), _p(word_off), u64(n_words),
                         _p(cdf), _p(out), ctypes.c_int(nthreads or os.cpu_count() or 1))
    return out, off


def dna_queries(seed, n, docs, doc_off, n_tp, fixed_len=0, median=0.0, sigma=0.0, lo=0, hi=0,
                rate_lo=0.0, rate_hi=0.0):
    n_docs = len(doc_off) - 1
    lens = (doc_off[1:] - doc_off[:-1]).astype(np.uint64)
    by_len = np.lexsort((np.arange(n_docs), lens)).astype(np.uint64)
    q_len = np.empty(n, dtype=np.uint64)
    src = np.empty(n, dtype=np.int64)
    start = np.empty(n, dtype=np.uint64)
    rate = np.empty(n, dtype=np.float64)
    L = _L()
    L.synth_dna_query_plan(u64(seed), u64(n), u64(n_tp), u64(fixed_len), ctypes.c_double(median),
                           ctypes.c_double(sigma), u64(lo), u64(hi), ctypes.c_double(rate_lo),
                           ctypes.c_double(rate_hi), _p(doc_off), u64(n_docs), _p(by_len),
                           _p(q_len), _p(src), _p(start), _p(rate))
    q_off = _offsets(q_len)
    out = np.empty(int(q_off[-1]), dtype=np.uint8)
    L.synth_dna_query_fill(u64(seed), u64(n), _p(docs), _p(doc_off), _p(src), _p(start), _p(rate),
                           _p(q_off), _p(out))
    return out, q_off, src


def text_queries(seed, n, docs, doc_off, len_lo, len_hi, edit_rate):
    n_docs = len(doc_off) - 1
    cap = 2 * len_hi * n + 16
    out = np.empty(cap, dtype=np.uint8)
    q_off = np.zeros(n + 1, dtype=np.uint64)
    src = np.empty(n, dtype=np.int64)
    L = _L()
    L.synth_text_queries.restype = ctypes.c_uint64
    used = L.synth_text_queries(u64(seed), u64(n), u64(len_lo), u64(len_hi), ctypes.c_double(edit_rate),
                                _p(docs), _p(doc_off), u64(n_docs), _p(src), _p(out), _p(q_off))
    return out[:used].copy(), q_off, src


def choice_u16(seed, n, choices):
    ch = np.asarray(choices, dtype=np.uint16)
    out = np.empty(n, dtype=np.uint16)
    _L().synth_choice_u16(u64(seed), u64(n), _p(ch), ctypes.c_uint32(len(ch)), _p(out))
    return out


def arrivals(seed, n, rate):
    out = np.empty(n, dtype=np.float64)
    _L().synth_arrivals(u64(seed), u64(n), ctypes.c_double(rate), _p(out))
    return out


@dataclass
class Workload:
    """One synthetic workload: index parameters, documents and a query set."""
    name: str
    term_kind: int
    q: int
    num_hashes: int
    fpr: float
    block_docs: int          # 0 = classic (one block, input order)
    score_bits: int
    docs: np.ndarray         # uint8, all documents concatenated
    doc_off: np.ndarray      # uint64[n_docs + 1]
    queries: np.ndarray      # uint8, all queries concatenated
    q_off: np.ndarray        # uint64[n_queries + 1]
    thresholds: np.ndarray   # uint16 permille per query
    src: np.ndarray          # int64 source document per query, -1 = random
    meta: dict = field(default_factory=dict)

    @property
    def n_docs(self):
        return len(self.doc_off) - 1

    @property
    def n_queries(self):
        return len(self.q_off) - 1

    def params(self):
        return dict(term_kind=self.term_kind, q=self.q, num_hashes=self.num_hashes, fpr=self.fpr,
                    block_docs=self.block_docs, score_bits=self.score_bits)

    def query_list(self):
        return [bytes(self.queries[int(self.q_off[i]):int(self.q_off[i + 1])]) for i in range(self.n_queries)]

    def doc_list(self):
        return [bytes(self.docs[int(self.doc_off[i]):int(self.doc_off[i + 1])]) for i in range(self.n_docs)]


def config1(seed_docs=1001, seed_q=2001, n_docs=64, doc_len=5000, n_q=200, q_len=100):
    """Classic index: 64 uniform ACGT documents of 5,000 bases, k=31 canonical,
    h=1, p=0.3, 200 queries of 100 bases (half exact substrings, half random), K=0.8,
    16-bit scores."""
    docs, off = dna_docs(seed_docs, np.full(n_docs, doc_len, dtype=np.uint64))
    qb, qo, src = dna_queries(seed_q, n_q, docs, off, n_tp=n_q // 2, fixed_len=q_len)
    return Workload("cfg1-classic-64docs", TERM_DNA_CANONICAL, 31, 1, 0.3, 0, 16, docs, off, qb, qo,
                    np.full(n_q, 800, dtype=np.uint16), src)


def config2(seed_docs=1002, seed_q=2002, n_docs=10_000, median=100_000, lo=10_000, hi=1_000_000,
            block_docs=8192, n_q=10_000, q_len=1000, thresholds=(500, 800, 1000)):
    """Compact index: 10,000 uniform ACGT documents, log-normal lengths (median
    100 kb, sigma 0.3, clipped to 10 kb..1 Mb), k=31 canonical, h=1, p=0.3,
    blocks of 8,192; 10,000 queries of 1,000 bases with 1% substitutions; query i
    gets threshold thresholds[i % 3]; 32-bit scores."""
    lens = lognormal_lengths(seed_docs, n_docs, median, 0.3, lo, hi)
    docs, off = dna_docs(seed_docs, lens)
    qb, qo, src = dna_queries(seed_q, n_q, docs, off, n_tp=n_q, fixed_len=q_len, rate_lo=0.01, rate_hi=0.01)
    thr = np.array([thresholds[i % len(thresholds)] for i in range(n_q)], dtype=np.uint16)
    return Workload("cfg2-compact-10kdocs", TERM_DNA_CANONICAL, 31, 1, 0.3, block_docs, 32, docs, off, qb, qo,
                    thr, src)


def config3(seed_docs=1003, seed_q=2003, n_docs=100_000, median=200_000, lo=20_000, hi=5_000_000,
            block_docs=8192, n_q=50_000, q_median=3162.0, q_sigma=1.151, q_lo=100, q_hi=100_000):
    """Batched uneven queries: 100,000 ACGT documents (log-normal median 200 kb,
    sigma 0.3, clipped to 20 kb..5 Mb), blocks of 8,192; 50,000 queries, lengths
    log-normal 100 b..100 kb, half substrings with per-query substitution rate
    U[0, 5%], half random; K=0.8; 32-bit scores."""
    lens = lognormal_lengths(seed_docs, n_docs, median, 0.3, lo, hi)
    docs, off = dna_docs(seed_docs, lens)
    qb, qo, src = dna_queries(seed_q, n_q, docs, off, n_tp=n_q // 2, median=q_median, sigma=q_sigma,
                              lo=q_lo, hi=q_hi, rate_lo=0.0, rate_hi=0.05)
    return Workload("cfg3-batched-100kdocs", TERM_DNA_CANONICAL, 31, 1, 0.3, block_docs, 32, docs, off, qb, qo,
                    np.full(n_q, 800, dtype=np.uint16), src)


def config4(seed_docs=1004, seed_q=2004, n_docs=50_000, n_words=200_000, median=20_000, lo=1_000,
            hi=1_000_000, block_docs=4096, n_q=100_000, q_lo=64, q_hi=512):
    """q-gram text index: Zipf(1.1) words from a 200,000-word random lowercase
    vocabulary, log-normal document lengths (median 20 KB), q=8 byte q-grams,
    h=3, p=0.1, blocks of 4,096; 100,000 queries of 64..512 bytes with 2% edits;
    K=0.7; 32-bit scores."""
    words, woff = vocab(seed_docs, n_words)
    lens = lognormal_lengths(seed_docs, n_docs, median, 0.3, lo, hi)
    docs, off = text_docs(seed_docs, lens, words, woff)
    qb, qo, src = text_queries(seed_q, n_q, docs, off, q_lo, q_hi, 0.02)
    return Workload("cfg4-text-qgram", TERM_BYTES, 8, 3, 0.1, block_docs, 32, docs, off, qb, qo,
                    np.full(n_q, 700, dtype=np.uint16), src)


WORKLOADS_JSON = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads.json")
_RECIPES = ("config1", "config2", "config3", "config4")


def workload(name: str, path: str | None = None, **overrides) -> Workload:
    """A workload by name from a JSON file that maps names to a recipe
    (config1..config4 above) and its parameters; `overrides` replace parameters.
    The default file, workloads.json beside this module, holds the recipes'
    default parameters (cfg1..cfg4, cfg2-small) and the serving queries (cfg5)."""
    with open(path or WORKLOADS_JSON) as f:
        table = json.load(f)
    if name not in table:
        raise ValueError(f"unknown workload {name!r} (known: {', '.join(sorted(table))})")
    entry = table[name]
    if entry["recipe"] not in _RECIPES:
        raise ValueError(f"workload {name!r} is not a document and query set (recipe {entry['recipe']})")
    params = dict(entry["params"])
    params.update(overrides)
    if "thresholds" in params:
        params["thresholds"] = tuple(params["thresholds"])
    return globals()[entry["recipe"]](**params)


def serving_params(name: str = "cfg5", path: str | None = None) -> dict:
    """Parameters of the serving-queries recipe (config5_queries) from the JSON file."""
    with open(path or WORKLOADS_JSON) as f:
        entry = json.load(f)[name]
    if entry["recipe"] != "config5_queries":
        raise ValueError(f"workload {name!r} is not a serving query set")
    return dict(entry["params"])


def config5_queries(wl2: Workload, seed_q=2005, n_q=20_000, q_median=3162.0, q_sigma=1.151, q_lo=100,
                    q_hi=100_000, rate=1000.0):
    """Serving requests on the compact 10,000-document index: query lengths
    log-normal 100 b..100 kb (half mutated substrings, half random), thresholds
    uniform in {0.5, 0.7, 0.9, 1.0}, Poisson arrival times at `rate` per second."""
    qb, qo, src = dna_queries(seed_q, n_q, wl2.docs, wl2.doc_off, n_tp=n_q // 2, median=q_median,
                              sigma=q_sigma, lo=q_lo, hi=q_hi, rate_lo=0.0, rate_hi=0.05)
    thr = choice_u16(seed_q, n_q, [500, 700, 900, 1000])
    t = arrivals(3005, n_q, rate)
    return qb, qo, thr, src, t
