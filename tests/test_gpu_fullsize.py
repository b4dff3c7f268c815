"""The benchmark workload at full size (10,000 compact documents, 10,000
queries of 1,000 bases) in the launch configuration bench.py times: the device
index is compared with the oracle's byte for byte, and a seeded sample of the
batched results is compared with the oracle query by query."""
import numpy as np
import pytest

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
