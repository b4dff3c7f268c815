"""The device build's two bit-set paths and its waves, against the oracle index.

A block whose Bloom filter (w_b bits) fits in shared memory gets its bits from
per-document filters and a bit-matrix transpose; a wider block from one global
atomicOr per window and hash.  The boundary is w_b = 1,736,704 bits (212 KB):
both sides of it, and an index with blocks on both paths, must equal the
oracle's byte for byte.  A small scratch budget (cobs_debug_build_scratch)
makes a small build run its distinct counts and its filter tiles in many waves;
the index must not change.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_1905_09624_gb300 import cobs

from parity import assert_index_equal, assert_results_equal, oracle_index, small_compact

pytestmark = pytest.mark.gpu

W_FILTER_MAX = 1_736_704  # largest w_b whose filter the build keeps in shared memory


def _tiny(seed, n_docs, block_docs):
    lens = synth.lognormal_lengths(seed, n_docs, 300, 0.5, 40, 2000)
    docs, off = synth.dna_docs(seed, lens)
    qb, qo, src = synth.dna_queries(seed + 1, 12, docs, off, n_tp=6, fixed_len=120, rate_lo=0.0, rate_hi=0.02)
    thr = synth.choice_u16(seed + 2, 12, [300, 800, 1000])
    return synth.Workload("tiny", 0, 31, 1, 0.3, block_docs, 32, docs, off, qb, qo, thr, src)


@pytest.mark.parametrize("width", [W_FILTER_MAX, W_FILTER_MAX + 1])
def test_filter_limit_both_sides(width):
    wl = _tiny(301, 40, 16)
    P = dict(wl.params())
    ref = oracle.build_index(oracle.make_params(width_override=width, **P), wl.docs, wl.doc_off)
    dix = cobs.DeviceIndex.build(cobs.make_params(width=width, **P), wl.docs, wl.doc_off)
    assert all(b["w"] == width for b in dix.info()["blocks"])
    assert_index_equal(dix, ref)
    got = dix.query(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
    assert_results_equal(got, ref, wl.query_list(), wl.thresholds)


def test_blocks_on_both_paths():
    # compact blocks whose Bloom sizes straddle the limit: one 4 Mb document in
    # the last block makes its w_b far wider than shared memory
    lens = np.array([300] * 24 + [4_000_000], dtype=np.uint64)
    docs, off = synth.dna_docs(303, lens)
    qb, qo, src = synth.dna_queries(304, 10, docs, off, n_tp=10, fixed_len=200, rate_lo=0.0, rate_hi=0.0)
    thr = np.full(10, 1000, np.uint16)
    wl = synth.Workload("straddle", 0, 31, 1, 0.3, 8, 32, docs, off, qb, qo, thr, src)
    ref = oracle_index(wl)
    dix = cobs.DeviceIndex.build(cobs.make_params(**wl.params()), wl.docs, wl.doc_off)
    ws = [b["w"] for b in dix.info()["blocks"]]
    assert min(ws) <= W_FILTER_MAX < max(ws)
    assert_index_equal(dix, ref)
    got = dix.query(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
    assert_results_equal(got, ref, wl.query_list(), wl.thresholds)


@pytest.mark.parametrize("block_docs", [0, 256])
def test_build_in_many_waves(block_docs):
    wl = small_compact(seed=307, n_docs=700, block_docs=block_docs, n_q=30, q_len=200)
    ref = oracle_index(wl)
    L = cobs.lib()
    L.cobs_debug_build_scratch(64 * 1024)  # a few documents' sets, one 256-column tile per wave
    try:
        dix = cobs.DeviceIndex.build(cobs.make_params(**wl.params()), wl.docs, wl.doc_off)
    finally:
        L.cobs_debug_build_scratch(0)
    assert_index_equal(dix, ref)
    if block_docs == 0:
        assert dix.info()["blocks"][0]["n_docs"] == 700  # one block: three 256-column waves
    got = dix.query(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
    assert_results_equal(got, ref, wl.query_list(), wl.thresholds)


def test_low_entropy_documents_overflow_their_partitions():
    # byte 2-grams over a 3-letter alphabet: at most 9 distinct terms, so nearly
    # all windows of a document fall into a few partitions and overflow them;
    # those documents are counted again with global sets
    rng = np.random.default_rng(311)
    lens = rng.integers(1000, 20000, 30).astype(np.uint64)
    docs = rng.choice(np.frombuffer(b"xyz", np.uint8), int(lens.sum())).astype(np.uint8)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    qb, qo = docs[:500].copy(), np.array([0, 200, 500], np.uint64)
    thr = np.array([500, 1000], np.uint16)
    wl = synth.Workload("low-entropy", 2, 2, 2, 0.3, 8, 32, docs, off, qb, qo, thr, np.zeros(2, np.int64))
    ref = oracle_index(wl)
    dix = cobs.DeviceIndex.build(cobs.make_params(**wl.params()), wl.docs, wl.doc_off)
    assert_index_equal(dix, ref)
    got = dix.query(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
    assert_results_equal(got, ref, wl.query_list(), wl.thresholds)


def test_document_beyond_the_partition_limit():
    # 7 M windows need more than 2,048 partitions (of 3,072 windows each): this
    # document's distinct count uses a global set, the others' partitions
    lens = np.array([500] * 6 + [7_000_030], dtype=np.uint64)
    docs, off = synth.dna_docs(313, lens)
    qb, qo, src = synth.dna_queries(314, 6, docs, off, n_tp=6, fixed_len=300, rate_lo=0.0, rate_hi=0.0)
    thr = np.full(6, 1000, np.uint16)
    wl = synth.Workload("one-long", 0, 31, 1, 0.3, 4, 32, docs, off, qb, qo, thr, src)
    ref = oracle_index(wl)
    dix = cobs.DeviceIndex.build(cobs.make_params(**wl.params()), wl.docs, wl.doc_off)
    assert_index_equal(dix, ref)
    got = dix.query(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
    assert_results_equal(got, ref, wl.query_list(), wl.thresholds)
