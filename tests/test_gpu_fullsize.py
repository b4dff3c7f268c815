"""The benchmark workloads at full size in the launch configuration bench.py
times: the bench workload (10,000 compact documents, 10,000 queries of 1,000
bases), the text q-gram workload (50,000 documents, h = 3) and the batched
uneven-query workload (100,000 documents, 50,000 queries of 100 b - 100 kb).
Device indexes are compared with the oracle's byte for byte (for the 8 GB
index: the plan in full and three blocks' rows), and seeded samples of the
results query by query."""
import numpy as np
import pytest

import oracle
import synth
from paper_1905_09624_gb300 import cobs

from parity import assert_index_equal, assert_results_equal, oracle_index

pytestmark = pytest.mark.gpu


def test_cfg2_full_size_index_and_sampled_queries():
    import torch
    wl = synth.config2()
    dix = cobs.DeviceIndex.build(cobs.make_params(**wl.params()), wl.docs, wl.doc_off)
    ref = oracle_index(wl, threaded=True)
    assert [b["n_docs"] for b in ref.blocks()] == [8192, 1808]
    assert_index_equal(dix, ref)
    # batched form, default engine, device-resident inputs (as in bench.py)
    stream = torch.cuda.Stream()
    eng = cobs.Engine(dix, stream=stream.cuda_stream)
    d_q = torch.from_numpy(wl.queries).cuda()
    d_off = torch.from_numpy(wl.q_off.view(np.int64)).cuda()
    d_thr = torch.from_numpy(wl.thresholds.view(np.int16)).cuda()
    torch.cuda.synchronize()
    eng.query_device(d_q, d_off, wl.q_off, d_thr, cobs.COBS_BATCHED)
    got = eng.download()
    sample = np.random.default_rng(2024).choice(wl.n_queries, 120, replace=False).tolist()
    assert_results_equal(got, ref, wl.query_list(), wl.thresholds, which=sample)
    # the captured graph (the form bench.py times) gives every query's hits exactly
    batched = eng.download_arrays()
    for _ in range(2):  # capture, then replay
        eng.query_device(d_q, d_off, wl.q_off, d_thr, cobs.COBS_GRAPH)
        graph = eng.download_arrays()
        assert all(np.array_equal(a, b) for a, b in zip(graph, batched))
    # so does the plain form, one query per launch, on the whole batch
    eng.query_device(d_q, d_off, wl.q_off, d_thr, cobs.COBS_PLAIN)
    plain = eng.download_arrays()
    assert all(np.array_equal(a, b) for a, b in zip(plain, batched))
    # and so does the pipelined host path of the end-to-end measurement
    pin = torch.empty(len(wl.queries), dtype=torch.uint8, pin_memory=True).numpy()
    pin[:] = wl.queries
    eng.submit_host(pin, wl.q_off, wl.thresholds, cobs.COBS_GRAPH)
    host = eng.download_arrays()
    assert all(np.array_equal(a, b) for a, b in zip(host, batched))
    # every query is a mutated substring of its source document (1% substitutions,
    # each changing at most 31 of about 970 terms): at K = 0.5 nearly all find it
    half = [i for i in range(wl.n_queries) if wl.thresholds[i] == 500]
    found = sum(wl.src[i] in got[i][2].tolist() for i in half)
    assert found >= 0.99 * len(half), (found, len(half))


def _graph_form_results(dix, wl):
    """Every query of the workload through the engine in the bench's launch
    configuration (default engine), as the captured graph, replayed once."""
    import torch
    stream = torch.cuda.Stream()
    eng = cobs.Engine(dix, stream=stream.cuda_stream)
    d_q = torch.from_numpy(wl.queries).cuda()
    d_off = torch.from_numpy(wl.q_off.view(np.int64)).cuda()
    d_thr = torch.from_numpy(wl.thresholds.view(np.int16)).cuda()
    torch.cuda.synchronize()
    eng.query_device(d_q, d_off, wl.q_off, d_thr, cobs.COBS_GRAPH)  # capture
    first = eng.download_arrays()
    eng.query_device(d_q, d_off, wl.q_off, d_thr, cobs.COBS_GRAPH)  # replay
    res = eng.download_arrays()
    assert all(np.array_equal(a, b) for a, b in zip(first, res))
    return res


def _plain_matches(dix, wl, res, m):
    """The plain form (one query per launch) on the first m queries, as a batch
    of its own, gives exactly the hits of the full batch's first m queries."""
    import torch
    qo = wl.q_off[:m + 1].copy()
    d_q = torch.from_numpy(wl.queries[:int(qo[-1])].copy()).cuda()
    d_off = torch.from_numpy(qo.view(np.int64)).cuda()
    d_thr = torch.from_numpy(wl.thresholds[:m].copy().view(np.int16)).cuda()
    eng = cobs.Engine(dix)
    torch.cuda.synchronize()
    eng.query_device(d_q, d_off, qo, d_thr, cobs.COBS_PLAIN)
    plain = eng.download_arrays()
    for i in range(m):
        assert _query(plain, i)[:2] == _query(res, i)[:2], i
        a, b = _query(plain, i), _query(res, i)
        assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3]), i


def _query(res, i):
    h0, h1 = int(res[2][i]), int(res[2][i + 1])
    return int(res[0][i]), int(res[1][i]), res[3][h0:h1], res[4][h0:h1]


def _sample_with_longest(wl, n, n_long, seed):
    lens = np.diff(wl.q_off).astype(np.int64)
    longest = np.argsort(-lens, kind="stable")[:n_long]
    rest = np.setdiff1d(np.arange(wl.n_queries), longest)
    pick = np.random.default_rng(seed).choice(rest, n - n_long, replace=False)
    return sorted(set(longest.tolist()) | set(pick.tolist()))


def test_cfg4_full_size_index_and_sampled_queries():
    """The text q-gram workload at full size (50,000 documents, h = 3, 13
    blocks of 4,096): every index byte, and 300 sampled queries (the 20 longest
    among them) in the graph form, against the oracle."""
    wl = synth.config4()
    dix = cobs.DeviceIndex.build(cobs.make_params(**wl.params()), wl.docs, wl.doc_off)
    ref = oracle_index(wl, threaded=True)
    assert len(ref.blocks()) == 13
    assert_index_equal(dix, ref)
    res = _graph_form_results(dix, wl)
    _plain_matches(dix, wl, res, 2000)  # the fused plain kernel, h = 3, 13 blocks
    ql = wl.query_list()
    sample = _sample_with_longest(wl, 300, 20, 4004)
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor() as ex:
        want = list(ex.map(lambda i: ref.query(ql[i], int(wl.thresholds[i])), sample))
    for i, (ell, mn, ids, sc) in zip(sample, want):
        g = _query(res, i)
        assert (g[0], g[1]) == (ell, mn), (i, g[:2], ell, mn)
        assert np.array_equal(g[2], ids) and np.array_equal(g[3], sc), i


def test_cfg3_full_size_plan_sampled_blocks_and_queries():
    """The batched uneven-query workload at full size (100,000 documents, about
    8 GB of index in 13 blocks, 50,000 queries of 100 b - 100 kb).  The oracle's
    per-document counts and plan over all documents are compared in full (block
    table, permutation, counts); the rows of three blocks -- two seeded ones and
    the last (largest) block -- byte for byte; and 220 sampled queries (the 20
    longest, on the widest counters, among them; half the workload's queries are
    random strings) in the graph form: l and ceil(K l) exactly, and the hits
    among the three blocks' documents against an oracle index whose other blocks
    are left empty (scores there are 0, below every min score >= 1)."""
    wl = synth.config3()
    P = oracle.make_params(**wl.params())
    dix = cobs.DeviceIndex.build(cobs.make_params(**wl.params()), wl.docs, wl.doc_off)
    v = oracle.doc_counts_threaded(P, wl.docs, wl.doc_off)
    ref = oracle.plan(P, v)
    blocks = ref.blocks()
    assert len(blocks) == 13
    host = dix.download()
    info = host.info()
    assert info["blocks"] == blocks
    assert np.array_equal(info["perm"], ref.perm())
    assert np.array_equal(info["nterms"], ref.nterms())
    picked = sorted(set(np.random.default_rng(3003).choice(12, 2, replace=False).tolist()) | {12})
    oracle.fill_threaded(ref, wl.docs, wl.doc_off, picked)
    got_rows, want_rows = info["rows"], ref.rows_view()
    for b in picked:
        blk = blocks[b]
        lo, hi = blk["row_offset"], blk["row_offset"] + blk["w"] * blk["rowbytes"]
        assert np.array_equal(got_rows[lo:hi], want_rows[lo:hi]), f"block {b} differs"
    del host, info, got_rows
    res = _graph_form_results(dix, wl)
    # the plain form on 500 queries: most are longer than one term round (terms
    # kernels, then the gather kernel), the others run fused
    _plain_matches(dix, wl, res, 500)
    perm = ref.perm()
    in_picked = np.zeros(wl.n_docs, dtype=bool)
    for b in picked:
        in_picked[perm[blocks[b]["doc_begin"]:blocks[b]["doc_begin"] + blocks[b]["n_docs"]]] = True
    ql = wl.query_list()
    sample = _sample_with_longest(wl, 220, 20, 3033)
    assert min(len(ql[i]) for i in sorted(sample, key=lambda i: -len(ql[i]))[:20]) >= 50_000
    from concurrent.futures import ThreadPoolExecutor
    order = sorted(sample, key=lambda i: -len(ql[i]))  # longest first across the threads
    with ThreadPoolExecutor() as ex:
        want = dict(zip(order, ex.map(lambda i: ref.query(ql[i], int(wl.thresholds[i])), order)))
    n_hits = 0
    for i in sample:
        ell, mn, ids, sc = want[i]
        g = _query(res, i)
        assert (g[0], g[1]) == (ell, mn), (i, g[:2], ell, mn)
        keep = in_picked[g[2]]
        assert np.array_equal(g[2][keep], ids) and np.array_equal(g[3][keep], sc), i
        n_hits += len(ids)
    assert n_hits > 0
