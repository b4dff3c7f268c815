"""Continuous-batching serve loop (cobs_serve_*): every result equals the
oracle's and the batched form's, alone and mixed under load; budget admission
and error codes."""
import threading
import time

import numpy as np
import pytest

import synth
from paper_1905_09624_gb300 import cobs

from parity import assert_results_equal, device_index, oracle_index, small_compact

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served():
    wl = small_compact(seed=71, n_docs=500, block_docs=200, n_q=120, q_len=400)
    # uneven lengths as in the serving workload
    qb, qo, src = synth.dna_queries(72, 120, wl.docs, wl.doc_off, n_tp=60, median=800, sigma=1.0, lo=20, hi=8000,
                                    rate_lo=0.0, rate_hi=0.05)
    thr = synth.choice_u16(73, 120, [500, 700, 900, 1000])
    wl.queries, wl.q_off, wl.thresholds, wl.src = qb, qo, thr, src
    return wl, oracle_index(wl), device_index(wl)


def _wait(srv, tickets, timeout=60.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, "serve results did not arrive"
        time.sleep(0.0005)
    return [out[t] for t in tickets]


def test_serve_matches_oracle_and_batched(served):
    wl, ref, dix = served
    ql = wl.query_list()
    srv = cobs.Server(dix, max_inflight_waves=3, max_wave_queries=16)
    tickets = [srv.submit(q, int(wl.thresholds[i])) for i, q in enumerate(ql)]
    got = _wait(srv, tickets)
    stats = srv.stop()
    assert stats["completed"] == len(ql) and stats["waves"] >= len(ql) // 16
    assert 0 < stats["p50_ms"] <= stats["p99_ms"] <= stats["max_ms"]
    assert_results_equal(got, ref, ql, wl.thresholds)
    batched = dix.query(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
    for a, b in zip(got, batched):
        assert a[0] == b[0] and a[1] == b[1] and np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


def test_serve_plain_form_matches_oracle(served):
    # waves of one query in the plain form (the one-query-per-launch baseline of
    # the serving comparison): the same results as the oracle
    wl, ref, dix = served
    ql = wl.query_list()
    srv = cobs.Server(dix, max_inflight_waves=1, max_wave_queries=1, form=cobs.COBS_PLAIN)
    tickets = [srv.submit(q, int(wl.thresholds[i])) for i, q in enumerate(ql)]
    got = _wait(srv, tickets)
    stats = srv.stop()
    assert stats["completed"] == len(ql) and stats["waves"] == len(ql)
    assert_results_equal(got, ref, ql, wl.thresholds)


def test_serve_rejects_unknown_form(served):
    _, _, dix = served
    with pytest.raises(cobs.CobsError):
        cobs.Server(dix, form=7)


def test_same_result_alone_and_mixed_under_load(served):
    wl, ref, dix = served
    ql = wl.query_list()
    probe = [3, 50, 99]
    srv = cobs.Server(dix, max_inflight_waves=2, max_wave_queries=8)
    alone = {}
    for i in probe:  # each probe alone on an idle server
        alone[i] = _wait(srv, [srv.submit(ql[i], int(wl.thresholds[i]))])[0]
    # the same probes submitted from a second thread while a stream of requests is in flight
    mixed_tickets = {}
    stop = threading.Event()

    def background():
        k = 0
        while not stop.is_set():
            j = (k * 7) % len(ql)
            srv.submit(ql[j], int(wl.thresholds[j]))
            k += 1
            time.sleep(0.0002)

    th = threading.Thread(target=background)
    th.start()
    time.sleep(0.05)
    for i in probe:
        mixed_tickets[i] = srv.submit(ql[i], int(wl.thresholds[i]))
        time.sleep(0.003)
    mixed = {i: _wait(srv, [mixed_tickets[i]])[0] for i in probe}
    stop.set()
    th.join()
    stats = srv.stop()
    assert stats["waves"] > len(probe)
    for i in probe:
        a, b = alone[i], mixed[i]
        assert a[0] == b[0] and a[1] == b[1] and np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
    assert_results_equal([alone[i] for i in probe], ref, [ql[i] for i in probe],
                         [wl.thresholds[i] for i in probe])


def test_budget_admission_and_errors(served):
    wl, ref, dix = served
    ql = wl.query_list()
    n_docs = wl.n_docs
    # a budget that admits about two requests at a time: everything still completes
    one = n_docs * 4 + 64
    srv = cobs.Server(dix, score_budget_bytes=3 * one + 200_000, max_inflight_waves=2, max_wave_queries=64)
    small = [i for i, q in enumerate(ql) if len(q) < 600][:20]
    tickets = [srv.submit(ql[i], int(wl.thresholds[i])) for i in small]
    got = _wait(srv, tickets)
    assert_results_equal(got, ref, [ql[i] for i in small], [wl.thresholds[i] for i in small])
    # a request that can never fit is refused at submit
    with pytest.raises(cobs.CobsError) as e:
        srv.submit(b"ACGT" * 50000, 500)
    assert e.value.status == cobs.COBS_ERR_BUDGET
    with pytest.raises(cobs.CobsError) as e:
        srv.submit(ql[0], 0)
    assert e.value.status == cobs.COBS_ERR_ARG
    h = cobs.cobs_hits()
    assert cobs.lib().cobs_serve_poll(srv.h, 987654321, h) == cobs.COBS_ERR_NOT_FOUND
    stats = srv.stop()
    assert stats["rejected"] >= 1 and stats["completed"] == len(small)


def test_wave_timeout_fails_its_tickets_and_the_server_recovers():
    # A 1 ms wait limit that a wave cannot meet: one query of 2 M windows on an
    # index of 313 blocks (its row pass alone takes far longer).  The ticket fails
    # with COBS_ERR_TIMEOUT while the device work finishes on its own (the slot
    # is reused only after that); later requests complete and match the batched
    # form.
    wl = small_compact(seed=83, n_docs=40000, median=500, sigma=0.3, lo=100, hi=2000, block_docs=128, n_q=8,
                       q_len=300)
    dix = device_index(wl)
    assert len(dix.info()["blocks"]) == 313
    rng = np.random.default_rng(5)
    big = bytes(rng.choice(np.frombuffer(b"ACGT", np.uint8), 2_000_030))
    srv = cobs.Server(dix, max_inflight_waves=2, wait_timeout_ms=1)
    t = srv.submit(big, 900)
    t0 = time.time()
    with pytest.raises(cobs.CobsError) as e:
        while srv.poll(t) is None:
            assert time.time() - t0 < 60, "ticket did not resolve"
            time.sleep(0.001)
    assert e.value.status == cobs.COBS_ERR_TIMEOUT
    # the server still answers: a short query completes (retried while the
    # device finishes the timed-out work) with the batched form's result
    ql = wl.query_list()
    want = dix.query(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
    for attempt in range(100):
        try:
            got = _wait(srv, [srv.submit(ql[0], int(wl.thresholds[0]))])[0]
            break
        except cobs.CobsError as e:
            assert e.status == cobs.COBS_ERR_TIMEOUT
            time.sleep(0.05)
    else:
        raise AssertionError("no request completed after the timeout")
    assert (got[0], got[1]) == (want[0][0], want[0][1])
    assert np.array_equal(got[2], want[0][2]) and np.array_equal(got[3], want[0][3])
    stats = srv.stop()
    assert stats["completed"] >= 1


def test_cancel_on_the_device_and_in_the_queue(served):
    # one slot and one query per wave: the longest query runs while the others
    # queue; cancelling it (on the device) and a queued one drops exactly those
    wl, ref, dix = served
    ql = wl.query_list()
    order = sorted(range(len(ql)), key=lambda i: -len(ql[i]))[:12]
    srv = cobs.Server(dix, max_inflight_waves=1, max_wave_queries=1)
    tickets = [srv.submit(ql[i], int(wl.thresholds[i])) for i in order]
    srv.cancel(tickets[0])
    srv.cancel(tickets[5])
    keep = [k for k in range(len(order)) if k not in (0, 5)]
    got = _wait(srv, [tickets[k] for k in keep])
    assert_results_equal(got, ref, [ql[order[k]] for k in keep], [wl.thresholds[order[k]] for k in keep])
    for k in (0, 5):
        with pytest.raises(cobs.CobsError) as e:
            srv.poll(tickets[k])
        assert e.value.status == cobs.COBS_ERR_CANCELLED
        srv.release(tickets[k])
        with pytest.raises(cobs.CobsError) as e:
            srv.poll(tickets[k])
        assert e.value.status == cobs.COBS_ERR_NOT_FOUND
    stats = srv.stop()
    assert stats["cancelled"] == 2 and stats["completed"] >= len(keep)
