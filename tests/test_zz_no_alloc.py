"""The query entry point that allocates nothing (cobs_query_one_noalloc).

It serves callers that cannot allocate device memory: a process whose memory
pool already holds the device memory it may use, or a latency-critical request
thread that must not call cudaMalloc/cudaFree (they can synchronise the whole
device).  Its scratch is a fixed device array inside the library.  These tests
call it through the C ABI and check its hits against the library's existing
batched entry point, bit for bit, on consecutive calls that reuse the scratch.
The file is named so that pytest collects it last.
"""

import numpy as np
import pytest

import synth
from paper_1905_09624_gb300 import cobs

from parity import device_index, small_compact

pytestmark = pytest.mark.gpu


def _run_noalloc(dix, n_docs, query: bytes, thr: int):
    import torch
    L = cobs.lib()
    q = torch.from_numpy(np.frombuffer(query, np.uint8).copy() if query else np.zeros(1, np.uint8)).cuda()
    meta = torch.full((3,), 0xFFFF, dtype=torch.int32, device="cuda")
    ids = torch.full((max(n_docs, 1),), -1, dtype=torch.int32, device="cuda")
    scores = torch.full((max(n_docs, 1),), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    st = L.cobs_query_one_noalloc(dix.h, q.data_ptr(), len(query), thr, meta.data_ptr(), ids.data_ptr(),
                                  scores.data_ptr(), n_docs, None)
    assert st == cobs.COBS_OK, L.cobs_last_error()
    torch.cuda.synchronize()
    m = meta.cpu().numpy().astype(np.uint32)
    n = int(m[2])
    return int(m[0]), int(m[1]), ids.cpu().numpy()[:n].astype(np.uint32), scores.cpu().numpy()[:n].astype(np.uint32)


def _same(a, b):
    return a[0] == b[0] and a[1] == b[1] and np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


def test_noalloc_matches_batched_on_consecutive_calls():
    import torch
    torch.cuda.set_device(0)
    wl = small_compact(seed=61, n_docs=700, block_docs=256, n_q=12, q_len=300)
    ql = wl.query_list()
    # one long query (spills the distinct-term set to the global scratch) and an empty one
    long_q = synth.dna_docs(62, [6000])[0].tobytes()
    ql += [bytes(wl.docs[int(wl.doc_off[5]):int(wl.doc_off[5]) + 5000]), long_q, b""]
    thr = list(wl.thresholds) + [800, 1, 500]
    qo = np.zeros(len(ql) + 1, np.uint64)
    qo[1:] = np.cumsum([len(x) for x in ql])
    qb = np.frombuffer(b"".join(ql), np.uint8)
    thr = np.array(thr, np.uint16)
    dix = device_index(wl)
    ref = dix.query(qb, qo, thr, cobs.COBS_BATCHED)
    order = [0, 1, 1, len(ql) - 3, len(ql) - 2, 2, len(ql) - 1, 3]   # repeats and back-to-back calls
    for i in order:
        got = _run_noalloc(dix, wl.n_docs, ql[i], int(thr[i]))
        assert _same(got, ref[i]), (i, got[:2], ref[i][:2], got[2][:8], ref[i][2][:8])
    assert any(len(ref[i][2]) > 100 for i in order)  # the K = 1 permille query has many hits


def test_noalloc_rejects_beyond_its_limits():
    import torch
    torch.cuda.set_device(0)
    wl = small_compact(seed=63, n_docs=50, block_docs=0, n_q=2)
    dix = device_index(wl)
    L = cobs.lib()
    buf = torch.zeros(20000, dtype=torch.uint8, device="cuda")
    out = torch.zeros(64, dtype=torch.int32, device="cuda")
    too_long = int(cobs.lib().cobs_query_one_noalloc(dix.h, buf.data_ptr(), 20000, 500, out.data_ptr(),
                                                     out.data_ptr(), out.data_ptr(), 64, None))
    assert too_long == cobs.COBS_ERR_ARG and b"windows" in L.cobs_last_error()
    small_out = int(L.cobs_query_one_noalloc(dix.h, buf.data_ptr(), 100, 500, out.data_ptr(), out.data_ptr(),
                                             out.data_ptr(), 10, None))
    assert small_out == cobs.COBS_ERR_ARG and b"out_capacity" in L.cobs_last_error()
    assert int(L.cobs_query_one_noalloc(dix.h, buf.data_ptr(), 100, 0, out.data_ptr(), out.data_ptr(),
                                        out.data_ptr(), 64, None)) == cobs.COBS_ERR_ARG
