"""The query entry point that allocates nothing (cobs_query_one_noalloc).

It serves callers that cannot allocate device memory: a process whose memory
pool already holds the device memory it may use, or a latency-critical request
thread that must not call cudaMalloc/cudaFree (they can synchronise the whole
device).  Its scratch is a fixed device array inside the library.  These tests
call it through the C ABI and check its hits against the library's existing
batched entry point, bit for bit, on consecutive calls that reuse the scratch;
they also make every library allocation fail and check that the entry point
still answers, and that the device's free memory does not move across calls.
The file is named so that pytest collects it last.
"""

import numpy as np
import pytest

import synth
from paper_1905_09624_gb300 import cobs

from parity import device_index, small_compact

pytestmark = pytest.mark.gpu


def _run_noalloc(dix, n_docs, query: bytes, thr: int, bufs=None):
    """One call; bufs = (query, meta, ids, scores) device tensors reused across calls."""
    import torch
    L = cobs.lib()
    if bufs is None:
        bufs = _buffers(n_docs, max(len(query), 1))
    q, meta, ids, scores = bufs
    if query:
        q[:len(query)].copy_(torch.from_numpy(np.frombuffer(query, np.uint8).copy()))
    meta.fill_(0xFFFF)
    ids.fill_(-1)
    scores.fill_(-1)
    torch.cuda.synchronize()
    st = L.cobs_query_one_noalloc(dix.h, q.data_ptr(), len(query), thr, meta.data_ptr(), ids.data_ptr(),
                                  scores.data_ptr(), n_docs, None)
    assert st == cobs.COBS_OK, L.cobs_last_error()
    torch.cuda.synchronize()
    m = meta.cpu().numpy().astype(np.uint32)
    n = int(m[2])
    return int(m[0]), int(m[1]), ids.cpu().numpy()[:n].astype(np.uint32), scores.cpu().numpy()[:n].astype(np.uint32)


def _buffers(n_docs, max_len):
    import torch
    return (torch.zeros(max_len, dtype=torch.uint8, device="cuda"),
            torch.zeros(3, dtype=torch.int32, device="cuda"),
            torch.zeros(max(n_docs, 1), dtype=torch.int32, device="cuda"),
            torch.zeros(max(n_docs, 1), dtype=torch.int32, device="cuda"))


def _same(a, b):
    return a[0] == b[0] and a[1] == b[1] and np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


def _batch(ql, thr):
    qo = np.zeros(len(ql) + 1, np.uint64)
    qo[1:] = np.cumsum([len(x) for x in ql])
    return np.frombuffer(b"".join(ql), np.uint8), qo, np.array(thr, np.uint16)


def test_noalloc_matches_batched_on_consecutive_calls():
    import torch
    torch.cuda.set_device(0)
    wl = small_compact(seed=61, n_docs=700, block_docs=256, n_q=12, q_len=300)
    ql = wl.query_list()
    # one long query (spills the distinct-term set to the global scratch) and an empty one
    long_q = synth.dna_docs(62, [6000])[0].tobytes()
    ql += [bytes(wl.docs[int(wl.doc_off[5]):int(wl.doc_off[5]) + 5000]), long_q, b""]
    thr = list(wl.thresholds) + [800, 1, 500]
    qb, qo, thr = _batch(ql, thr)
    dix = device_index(wl)
    ref = dix.query(qb, qo, thr, cobs.COBS_BATCHED)
    order = [0, 1, 1, len(ql) - 3, len(ql) - 2, 2, len(ql) - 1, 3]   # repeats and back-to-back calls
    for i in order:
        got = _run_noalloc(dix, wl.n_docs, ql[i], int(thr[i]))
        assert _same(got, ref[i]), (i, got[:2], ref[i][:2], got[2][:8], ref[i][2][:8])
    assert any(len(ref[i][2]) > 100 for i in order)  # the K = 1 permille query has many hits


def test_noalloc_answers_while_every_allocation_fails():
    """After its first call (which looks up the scratch address), the entry point
    needs no allocation: with every library allocation made to fail, two more
    calls still succeed with the batched form's hits, and the device's free
    memory is the same before and after them."""
    import torch
    torch.cuda.set_device(0)
    wl = small_compact(seed=71, n_docs=500, block_docs=128, n_q=6, q_len=400)
    ql = wl.query_list()
    qb, qo, thr = _batch(ql, list(wl.thresholds))
    dix = device_index(wl)
    ref = dix.query(qb, qo, thr, cobs.COBS_BATCHED)
    bufs = _buffers(wl.n_docs, max(len(x) for x in ql))
    assert _same(_run_noalloc(dix, wl.n_docs, ql[0], int(thr[0]), bufs), ref[0])
    L = cobs.lib()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    L.cobs_debug_fail_alloc(0)
    try:
        for i in (1, 2, 1):
            got = _run_noalloc(dix, wl.n_docs, ql[i], int(thr[i]), bufs)
            assert _same(got, ref[i]), i
        # the allocation hook is live: an allocating call fails meanwhile
        with pytest.raises(cobs.CobsError):
            dix.query(qb, qo, thr, cobs.COBS_BATCHED)
    finally:
        L.cobs_debug_fail_alloc(-1)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def _text_index():
    return synth.config4(n_docs=160, n_q=10, n_words=800, median=1500, lo=50, hi=6000, block_docs=64)


def _dna16_index():
    return small_compact(seed=73, n_docs=300, block_docs=128, n_q=8, q_len=500, score_bits=16)


def _dna_32_lists():
    # 32 blocks of 10 documents, one hash: blocks x hashes = 32, the entry point's limit
    return small_compact(seed=75, n_docs=320, median=600, lo=40, hi=3000, block_docs=10, n_q=8, q_len=200)


@pytest.mark.parametrize("make", [_text_index, _dna16_index, _dna_32_lists],
                         ids=["bytes-q8-h3", "dna-16-bit-scores", "32-blocks-x-hashes"])
def test_noalloc_matches_batched_per_index_kind(make):
    import torch
    torch.cuda.set_device(0)
    wl = make()
    ql = wl.query_list()
    qb, qo, thr = _batch(ql, list(wl.thresholds))
    dix = device_index(wl)
    info = dix.info()
    assert len(info["blocks"]) * wl.num_hashes <= 32
    if make is _dna_32_lists:
        assert len(info["blocks"]) * wl.num_hashes == 32
    ref = dix.query(qb, qo, thr, cobs.COBS_BATCHED)
    for i in list(range(len(ql))) + [0]:
        got = _run_noalloc(dix, wl.n_docs, ql[i], int(thr[i]))
        assert _same(got, ref[i]), (i, got[:2], ref[i][:2])


def test_noalloc_at_its_window_limit():
    # exactly COBS_NOALLOC_MAX_WINDOWS (16,384) windows: answered, as the batched
    # form; one window more: refused
    import torch
    torch.cuda.set_device(0)
    wl = small_compact(seed=65, n_docs=400, block_docs=128, n_q=2, q_len=300)
    dix = device_index(wl)
    k = 31
    q = synth.dna_docs(66, [16384 + k - 1])[0].tobytes()
    qb, qo, thr = _batch([q], [300])
    ref = dix.query(qb, qo, thr, cobs.COBS_BATCHED)
    got = _run_noalloc(dix, wl.n_docs, q, 300)
    assert got[0] == 16384 and _same(got, ref[0])
    L = cobs.lib()
    over = torch.from_numpy(np.frombuffer(q + b"A", np.uint8).copy()).cuda()
    out = torch.zeros(max(wl.n_docs, 3), dtype=torch.int32, device="cuda")
    st = int(L.cobs_query_one_noalloc(dix.h, over.data_ptr(), len(q) + 1, 300, out.data_ptr(), out.data_ptr(),
                                      out.data_ptr(), wl.n_docs, None))
    assert st == cobs.COBS_ERR_ARG and b"windows" in L.cobs_last_error()


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
    # 33 blocks x hashes: one more than the entry point's row lists
    wl33 = small_compact(seed=77, n_docs=330, median=600, lo=40, hi=3000, block_docs=10, n_q=2, q_len=200)
    d33 = device_index(wl33)
    assert len(d33.info()["blocks"]) == 33
    o33 = torch.zeros(400, dtype=torch.int32, device="cuda")
    st = int(L.cobs_query_one_noalloc(d33.h, buf.data_ptr(), 100, 500, o33.data_ptr(), o33.data_ptr(),
                                      o33.data_ptr(), 400, None))
    assert st == cobs.COBS_ERR_ARG and b"blocks x hashes" in L.cobs_last_error()
