"""Host-injected allocation failures (cobs_debug_fail_alloc) on the GPU path.

Every device and pinned-host allocation of the library goes through one place;
the injection makes the n-th one fail as if memory were exhausted, without
attempting it, so nothing reaches the device.  Each sweep runs a call with
n = 0, 1, 2, ... until it succeeds: every failing attempt must return
COBS_ERR_OOM and leave what it touched freeable, and the objects that survive a
failure (an engine, a server) must still give results identical to the
oracle's.  A download after a failed batch is refused instead of reading
buffers the batch never filled.
"""
import time

import numpy as np
import pytest

from paper_1905_09624_gb300 import cobs

from parity import assert_index_equal, assert_results_equal, device_index, oracle_index, small_compact

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def injection_off():
    cobs.lib().cobs_debug_fail_alloc(-1)
    yield
    cobs.lib().cobs_debug_fail_alloc(-1)


def sweep(fn, limit=300):
    """fn() with allocation n failing, n = 0, 1, ...; returns (n, fn's value) of
    the first attempt that needed no more than n allocations."""
    L = cobs.lib()
    for n in range(limit):
        L.cobs_debug_fail_alloc(n)
        try:
            out = fn()
        except cobs.CobsError as e:
            L.cobs_debug_fail_alloc(-1)
            assert e.status == cobs.COBS_ERR_OOM, (n, str(e))
            continue
        L.cobs_debug_fail_alloc(-1)
        return n, out
    raise AssertionError(f"still failing after {limit} allocations")


@pytest.fixture(scope="module")
def wl_ref():
    wl = small_compact(seed=91, n_docs=300, block_docs=64, n_q=40, q_len=250)
    return wl, oracle_index(wl)


def test_build_and_load_under_allocation_failures(wl_ref):
    wl, ref = wl_ref
    P = cobs.make_params(**wl.params())
    n, dix = sweep(lambda: cobs.DeviceIndex.build(P, wl.docs, wl.doc_off))
    assert n >= 5  # the build allocates documents, tables, rows and scratch
    assert_index_equal(dix, ref)
    host = dix.download()
    n, dix2 = sweep(lambda: cobs.DeviceIndex.load(host))
    assert n >= 2
    assert_index_equal(dix2, ref)
    n, dix3 = sweep(lambda: cobs.DeviceIndex.load_streamed(host))
    got = cobs.Engine(dix3).query_host(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
    assert_results_equal(got, ref, wl.query_list(), wl.thresholds)


@pytest.mark.parametrize("form", [cobs.COBS_BATCHED, cobs.COBS_GRAPH, cobs.COBS_PLAIN])
def test_engine_survives_failed_batches(wl_ref, form):
    wl, ref = wl_ref
    dix = device_index(wl)
    ql = wl.query_list()
    # a new engine per attempt: creation and the first batch's buffers
    n, got = sweep(lambda: cobs.Engine(dix).query_host(wl.queries, wl.q_off, wl.thresholds, form))
    assert n >= 3
    assert_results_equal(got, ref, ql, wl.thresholds)
    # one engine kept across failed batches of growing size
    eng = cobs.Engine(dix)
    for k in (5, 20, 40):
        qo = wl.q_off[: k + 1]
        n, got = sweep(lambda: eng.query_host(wl.queries[: int(qo[-1])], qo, wl.thresholds[:k], form))
        assert_results_equal(got, ref, ql[:k], wl.thresholds[:k])


def test_download_after_failed_batch_is_refused(wl_ref):
    wl, ref = wl_ref
    dix = device_index(wl)
    eng = cobs.Engine(dix)
    with pytest.raises(cobs.CobsError) as e:
        eng.download()  # no batch yet
    assert e.value.status == cobs.COBS_ERR_ARG
    cobs.lib().cobs_debug_fail_alloc(0)
    with pytest.raises(cobs.CobsError) as e:
        eng.query_host(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
    assert e.value.status == cobs.COBS_ERR_OOM
    cobs.lib().cobs_debug_fail_alloc(-1)
    for call in (eng.download, eng.stats, eng.results_device):
        with pytest.raises(cobs.CobsError) as e:
            call()
        assert e.value.status == cobs.COBS_ERR_ARG
    got = eng.query_host(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
    assert_results_equal(got, ref, wl.query_list(), wl.thresholds)


def test_hit_capacity_regrowth_under_failures(wl_ref):
    # a hit capacity of 64 overflows on this batch: the engine grows its hit
    # buffers and re-runs the batch while the results are collected
    wl, ref = wl_ref
    dix = device_index(wl)
    thr = np.full(len(wl.thresholds), 1, np.uint16)  # every document with a shared term is a hit
    eng0 = cobs.Engine(dix, max_hits=64)
    want = eng0.query_host(wl.queries, wl.q_off, thr, cobs.COBS_BATCHED)
    assert sum(len(r[2]) for r in want) > 64
    assert_results_equal(want, ref, wl.query_list(), thr)
    n, got = sweep(lambda: cobs.Engine(dix, max_hits=64).query_host(wl.queries, wl.q_off, thr, cobs.COBS_BATCHED))
    assert_results_equal(got, ref, wl.query_list(), thr)


def test_autotune_under_failures(wl_ref):
    import torch
    wl, ref = wl_ref
    dix = device_index(wl)
    d_q = torch.from_numpy(wl.queries).cuda()
    d_off = torch.from_numpy(wl.q_off.view(np.int64)).cuda()
    d_thr = torch.from_numpy(wl.thresholds.view(np.int16)).cuda()
    eng = cobs.Engine(dix)
    eng.query_host(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
    for n in (0, 1, 3, 6):  # failures at the flush buffer, the slice tables and the sweep's batches
        cobs.lib().cobs_debug_fail_alloc(n)
        try:
            eng.autotune(d_q, d_off, wl.q_off, d_thr)
        except cobs.CobsError as e:
            assert e.status == cobs.COBS_ERR_OOM
        finally:
            cobs.lib().cobs_debug_fail_alloc(-1)
        got = eng.query_host(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_GRAPH)
        assert_results_equal(got, ref, wl.query_list(), wl.thresholds)


def test_serve_wave_launch_failure(wl_ref):
    wl, ref = wl_ref
    dix = device_index(wl)
    ql = wl.query_list()
    srv = cobs.Server(dix, max_inflight_waves=1, max_wave_queries=4)
    cobs.lib().cobs_debug_fail_alloc(0)  # the first wave's staging buffers cannot be allocated
    t_bad = srv.submit(ql[0], int(wl.thresholds[0]))
    t0 = time.time()
    while True:
        try:
            r = srv.poll(t_bad)
        except cobs.CobsError as e:
            assert e.status == cobs.COBS_ERR_OOM
            break
        assert r is None, "the wave should have failed"
        assert time.time() - t0 < 30
        time.sleep(0.001)
    cobs.lib().cobs_debug_fail_alloc(-1)
    tickets = [srv.submit(q, int(wl.thresholds[i])) for i, q in enumerate(ql)]
    got = []
    for t in tickets:
        while (r := srv.poll(t)) is None:
            assert time.time() - t0 < 60
            time.sleep(0.0005)
        got.append(r)
    stats = srv.stop()
    assert stats["failed"] == 1 and stats["completed"] >= len(ql)
    assert_results_equal(got, ref, ql, wl.thresholds)
