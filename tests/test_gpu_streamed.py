"""Streamed device index (rows in pinned host memory, copied block by block into
a ring of device staging slots per batch) against the CPU oracle, bit for bit."""
import numpy as np
import pytest

import synth
from paper_1905_09624_gb300 import cobs

from parity import assert_index_equal, assert_results_equal, device_index, oracle_index, small_compact

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def streamed():
    # 5 blocks of 128 documents (the last one partial)
    wl = small_compact(seed=23, n_docs=600, median=3000, block_docs=128, n_q=120)
    ref = oracle_index(wl)
    host = device_index(wl).download()
    sdix = cobs.DeviceIndex.load_streamed(host)
    info = sdix.info()
    slot = max(b["w"] * b["rowbytes"] for b in info["blocks"])
    return wl, ref, sdix, info, slot


def test_streamed_index_is_the_index(streamed):
    wl, ref, sdix, info, slot = streamed
    assert len(info["blocks"]) == 5
    assert not info["rows_dev"]  # rows live in host memory
    assert_index_equal(sdix, ref)


@pytest.mark.parametrize("slots", [1, 2, 3, 5])
@pytest.mark.parametrize("flags", [cobs.COBS_BATCHED, cobs.COBS_GRAPH])
def test_streamed_results_every_ring_size(streamed, slots, flags):
    wl, ref, sdix, info, slot = streamed
    eng = cobs.Engine(sdix, stage_bytes=slots * ((slot + 255) // 256 * 256))
    for rep in range(2):  # the second batch reuses the ring (and the graph)
        got = eng.query_host(wl.queries, wl.q_off, wl.thresholds, flags)
        assert_results_equal(got, ref, wl.query_list(), wl.thresholds)
        assert eng.stats()["h2d_index_bytes"] == info["rows_bytes"]


def test_streamed_batches_of_changing_size(streamed):
    wl, ref, sdix, info, slot = streamed
    eng = cobs.Engine(sdix)
    ql = wl.query_list()
    for lo, hi in [(0, 7), (7, 120), (50, 51), (0, 120)]:
        qs = ql[lo:hi]
        off = np.zeros(len(qs) + 1, np.uint64)
        off[1:] = np.cumsum([len(x) for x in qs])
        qb = np.frombuffer(b"".join(qs), np.uint8)
        thr = wl.thresholds[lo:hi]
        got = eng.query_host(qb, off, thr, cobs.COBS_BATCHED)
        assert_results_equal(got, ref, qs, thr)


def test_streamed_split_long_queries():
    lens = synth.lognormal_lengths(71, 300, 20000, 0.5, 5000, 100000)
    docs, off = synth.dna_docs(71, lens)
    qb, qo, src = synth.dna_queries(72, 12, docs, off, n_tp=8, median=10000, sigma=0.5, lo=5000, hi=30000,
                                    rate_lo=0.0, rate_hi=0.005)
    thr = synth.choice_u16(73, 12, [1, 500, 900])
    wl = synth.Workload("streamed-split", 0, 31, 1, 0.3, 128, 32, docs, off, qb, qo, thr, src)
    ref = oracle_index(wl)
    sdix = cobs.DeviceIndex.load_streamed(device_index(wl).download())
    eng = cobs.Engine(sdix, split=2)
    got = eng.query_host(qb, qo, thr, cobs.COBS_BATCHED)
    assert eng.stats()["split_queries"] > 0
    assert_results_equal(got, ref, wl.query_list(), thr)


def test_streamed_errors(streamed):
    wl, ref, sdix, info, slot = streamed
    with pytest.raises(cobs.CobsError) as e:
        cobs.Engine(sdix, stage_bytes=slot // 2)
    assert e.value.status == cobs.COBS_ERR_ARG
    with pytest.raises(cobs.CobsError) as e:
        sdix.query(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_PLAIN)
    assert e.value.status == cobs.COBS_ERR_ARG


@pytest.mark.parametrize("slice_bytes", [32, 128, 256])
@pytest.mark.parametrize("slots", [1, 2])
def test_streamed_wide_rows_in_column_units(slice_bytes, slots):
    # blocks of 5,000 and 1,300 documents: rows of 640 and 176 bytes, so the first
    # block is copied and gathered in two column units (512 + 128 bytes)
    lens = synth.lognormal_lengths(83, 6300, 400, 0.4, 60, 3000)
    docs, off = synth.dna_docs(83, lens)
    qb, qo, src = synth.dna_queries(84, 60, docs, off, n_tp=40, fixed_len=150, rate_lo=0.0, rate_hi=0.02)
    thr = synth.choice_u16(85, 60, [200, 700, 1000])
    wl = synth.Workload("wide-rows", 0, 31, 1, 0.3, 5000, 32, docs, off, qb, qo, thr, src)
    ref = oracle_index(wl)
    host = device_index(wl).download()
    sdix = cobs.DeviceIndex.load_streamed(host)
    info = sdix.info()
    assert [b["rowbytes"] for b in info["blocks"]] == [640, 176]
    slot = max(b["w"] * b["rowbytes"] for b in info["blocks"])
    eng = cobs.Engine(sdix, slice_bytes=slice_bytes, stage_bytes=slots * ((slot + 255) // 256 * 256))
    for flags in (cobs.COBS_BATCHED, cobs.COBS_GRAPH, cobs.COBS_GRAPH):
        got = eng.query_host(wl.queries, wl.q_off, wl.thresholds, flags)
        assert_results_equal(got, ref, wl.query_list(), wl.thresholds)
        assert eng.stats()["h2d_index_bytes"] == info["rows_bytes"]
