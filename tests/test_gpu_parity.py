"""CUDA path vs CPU oracle, element by element, through the C ABI.

Bit-exact: index bytes, block table and permutation; per query the distinct
term count, the threshold, and the sorted (document id, score) hit list.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_1905_09624_gb300 import cobs

from parity import assert_index_equal, assert_results_equal, device_index, oracle_index, small_compact

pytestmark = pytest.mark.gpu

FORMS = [cobs.COBS_PLAIN, cobs.COBS_BATCHED, cobs.COBS_GRAPH]


@pytest.fixture(scope="module")
def cfg1():
    wl = synth.config1()
    return wl, oracle_index(wl), device_index(wl)


def test_cfg1_index_bit_exact(cfg1):
    wl, ref, dix = cfg1
    assert_index_equal(dix, ref)


@pytest.mark.parametrize("flags", FORMS)
def test_cfg1_results_all_forms(cfg1, flags):
    wl, ref, dix = cfg1
    got = dix.query(wl.queries, wl.q_off, wl.thresholds, flags)
    assert_results_equal(got, ref, wl.query_list(), wl.thresholds)
    # every exact substring query finds its source document with score l
    for i in range(100):
        assert wl.src[i] in got[i][2].tolist()


@pytest.fixture(scope="module")
def compact():
    wl = small_compact()
    return wl, oracle_index(wl), device_index(wl)


def test_compact_index_bit_exact(compact):
    wl, ref, dix = compact
    assert len(ref.blocks()) == 3 and ref.blocks()[-1]["n_docs"] == 600 - 512
    assert_index_equal(dix, ref)


@pytest.mark.parametrize("slice_bytes", [32, 64, 128, 256])
def test_compact_batched_slice_widths(compact, slice_bytes):
    wl, ref, dix = compact
    eng = cobs.Engine(dix, slice_bytes=slice_bytes)
    got = eng.query_host(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
    assert_results_equal(got, ref, wl.query_list(), wl.thresholds)


@pytest.mark.parametrize("flags", FORMS)
def test_compact_forms(compact, flags):
    wl, ref, dix = compact
    got = dix.query(wl.queries, wl.q_off, wl.thresholds, flags)
    assert_results_equal(got, ref, wl.query_list(), wl.thresholds)


def test_flat_result_arrays_match_lists(compact):
    wl, ref, dix = compact
    eng = cobs.Engine(dix)
    lists = eng.query_host(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
    ell, mn, off, ids, sc = eng.query_host_arrays(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
    for i, g in enumerate(lists):
        assert (ell[i], mn[i]) == (g[0], g[1])
        assert np.array_equal(ids[off[i]:off[i + 1]], g[2]) and np.array_equal(sc[off[i]:off[i + 1]], g[3])


def test_many_hits_large_segments():
    # K = 1 permille: every document with one matching term is a hit, so hit lists
    # exceed the shared-memory sort and use the global merge passes.
    wl = small_compact(seed=37, n_docs=2500, median=2000, block_docs=1024, n_q=30)
    ref = oracle_index(wl)
    dix = device_index(wl)
    thr = np.full(wl.n_queries, 1, np.uint16)
    got = dix.query(wl.queries, wl.q_off, thr, cobs.COBS_BATCHED)
    assert max(len(g[2]) for g in got) > 1024
    assert_results_equal(got, ref, wl.query_list(), thr, which=range(0, wl.n_queries, 7))


@pytest.mark.parametrize("n_docs", [1024, 1025, 2049, 30000])
def test_many_hits_sort_limits(n_docs):
    # K = 1 permille and 400-base queries: every document is a hit.  1,024 hits
    # is the most one query's shared-memory sort takes; 1,025 goes to the
    # large-segment sort as one chunk; 2,049 is a full 2,048-key chunk, a one-key
    # chunk and a merge pass in global memory; 30,000 is 15 chunks and four passes.
    wl = small_compact(seed=41, n_docs=n_docs, median=300, sigma=0.3, lo=100, hi=1000, block_docs=4096, n_q=6,
                       q_len=400)
    ref = oracle_index(wl)
    dix = device_index(wl)
    thr = np.full(wl.n_queries, 1, np.uint16)
    for flags in (cobs.COBS_BATCHED, cobs.COBS_GRAPH):
        got = dix.query(wl.queries, wl.q_off, thr, flags)
        assert max(len(g[2]) for g in got) == n_docs
        assert_results_equal(got, ref, wl.query_list(), thr)


def test_counter_class_and_round_boundaries():
    # Queries of exactly 1, 255, 256, 2,048, 2,049, 4,095, 4,096, 65,535 and
    # 65,536 windows (random bases: as many distinct terms), each also a document,
    # so the best score of each query is its whole term count: the largest value
    # of the 8-, 12- and 16-level counters (255, 4,095, 65,535) and one more, and
    # the last on-chip term set (2,048 windows) and the first long query's chunks.
    # Every form, K = 1000 and 500 permille.
    k = 31
    windows = [1, 255, 256, 2048, 2049, 4095, 4096, 65535, 65536]
    qs = [synth.dna_docs(95 + i, [w + k - 1])[0].tobytes() for i, w in enumerate(windows)]
    lens = synth.lognormal_lengths(94, 30, 3000, 0.5, 500, 20000)
    docs, off = synth.dna_docs(94, lens)
    db = np.concatenate([docs, np.frombuffer(b"".join(qs), np.uint8)])
    doff = np.concatenate([off, off[-1] + np.cumsum([len(x) for x in qs]).astype(np.uint64)])
    ql = qs + qs
    qo = np.zeros(len(ql) + 1, np.uint64)
    qo[1:] = np.cumsum([len(x) for x in ql])
    qb = np.frombuffer(b"".join(ql), np.uint8)
    thr = np.array([1000] * len(qs) + [500] * len(qs), np.uint16)
    wl = synth.Workload("boundaries", 0, k, 1, 0.3, 16, 32, db, doff, qb, qo, thr, np.full(len(ql), -1))
    ref = oracle_index(wl)
    dix = device_index(wl)
    for i, w in enumerate(windows):
        ell, mn, ids, sc = ref.query(qs[i], 1000)
        assert ell == w and int(sc[0]) == w and len(lens) + i in ids.tolist()
    for flags in FORMS:
        assert_results_equal(dix.query(qb, qo, thr, flags), ref, ql, thr)


def test_long_queries_in_several_set_groups():
    # 130 queries of 40,000 bases: their global distinct-term sets (2 slots per
    # window, 10.4 M slots) exceed the 8 M-slot table region, so the batch
    # inserts them in two groups that reuse the region in turn
    k = 31
    lens = synth.lognormal_lengths(97, 200, 20000, 0.5, 2000, 200000)
    docs, off = synth.dna_docs(97, lens)
    qb, qo, src = synth.dna_queries(98, 130, docs, off, n_tp=80, fixed_len=40000, rate_lo=0.0, rate_hi=0.02)
    ql = [bytes(qb[qo[i]:qo[i + 1]]) for i in range(130)]
    assert sum(2 * (len(x) - k + 1) for x in ql) > (8 << 20)
    thr = synth.choice_u16(99, 130, [300, 700, 1000])
    wl = synth.Workload("long-groups", 0, k, 1, 0.3, 64, 32, docs, off, qb, qo, thr, src)
    ref = oracle_index(wl)
    dix = device_index(wl)
    for flags in (cobs.COBS_BATCHED, cobs.COBS_GRAPH):
        assert_results_equal(dix.query(qb, qo, thr, flags), ref, ql, thr)


def test_hit_capacity_overflow_reruns(compact):
    wl, ref, dix = compact
    eng = cobs.Engine(dix, max_hits=4)
    thr = np.full(wl.n_queries, 1, np.uint16)
    got = eng.query_host(wl.queries, wl.q_off, thr, cobs.COBS_BATCHED)
    assert_results_equal(got, ref, wl.query_list(), thr, which=range(0, wl.n_queries, 11))


def test_uneven_query_lengths_counter_classes():
    # Queries from 0 bytes to 20 kb: empty and shorter-than-k queries (l = 0),
    # lengths spanning the 8-, 12- and 16-level counter kernels, spilled
    # distinct-term sets (> 2048 windows), and windows with non-ACGT bytes.
    lens = synth.lognormal_lengths(91, 80, 30000, 0.4, 25000, 90000)
    docs, off = synth.dna_docs(91, lens)
    qb, qo, src = synth.dna_queries(92, 60, docs, off, n_tp=40, median=2000, sigma=1.5, lo=1, hi=20000,
                                    rate_lo=0.0, rate_hi=0.05)
    ql = [bytes(qb[qo[i]:qo[i + 1]]) for i in range(60)]
    ql[3] = b""
    ql[4] = b"ACGT" * 7          # 28 < k
    ql[5] = ql[5][:200] + b"NNNN" + ql[5][200:] if len(ql[5]) > 300 else b"ACGTN" * 80
    ql[6] = ql[6].lower()        # no valid windows
    qo2 = np.zeros(61, np.uint64)
    qo2[1:] = np.cumsum([len(x) for x in ql])
    qb2 = np.frombuffer(b"".join(ql), np.uint8)
    thr = synth.choice_u16(93, 60, [500, 700, 900, 1000])
    wl = synth.Workload("uneven", 0, 31, 1, 0.3, 32, 32, docs, off, qb2, qo2, thr, src)
    ref = oracle_index(wl)
    dix = device_index(wl)
    assert_index_equal(dix, ref)
    for flags in FORMS:
        got = dix.query(wl.queries, wl.q_off, thr, flags)
        assert_results_equal(got, ref, ql, thr)
        assert got[3][0] == 0 and len(got[3][2]) == 0


@pytest.mark.parametrize("kind,q", [(1, 31), (0, 15), (1, 32), (0, 1)])
def test_dna_kinds_and_lengths(kind, q):
    wl = small_compact(seed=17, n_docs=150, median=1500, block_docs=64, n_q=50, q_len=120, kind=kind, q=q)
    ref = oracle_index(wl)
    dix = device_index(wl)
    assert_index_equal(dix, ref)
    got = dix.query(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
    assert_results_equal(got, ref, wl.query_list(), wl.thresholds)


@pytest.mark.parametrize("q,h", [(8, 3), (5, 2), (3, 1), (6, 4), (8, 5)])
def test_text_qgrams_multi_hash(q, h):
    wl = synth.config4(n_docs=400, n_q=120, n_words=3000, median=3000, lo=50, hi=20000, block_docs=128)
    wl.q, wl.num_hashes = q, h
    ref = oracle_index(wl)
    dix = device_index(wl)
    assert_index_equal(dix, ref)
    for flags in FORMS:
        got = dix.query(wl.queries, wl.q_off, wl.thresholds, flags)
        assert_results_equal(got, ref, wl.query_list(), wl.thresholds)


@pytest.mark.parametrize("slice_bytes", [32, 64, 128])
def test_multi_hash_slice_widths(slice_bytes):
    # h = 3: 128-byte slices run the pipelined kernel, narrower ones the register kernel
    wl = synth.config4(n_docs=300, n_q=80, n_words=2000, median=2500, lo=50, hi=20000, block_docs=128)
    ref = oracle_index(wl)
    dix = device_index(wl)
    eng = cobs.Engine(dix, slice_bytes=slice_bytes)
    for flags in (cobs.COBS_BATCHED, cobs.COBS_GRAPH):
        got = eng.query_host(wl.queries, wl.q_off, wl.thresholds, flags)
        assert_results_equal(got, ref, wl.query_list(), wl.thresholds)


def test_classic_equals_compact_single_block():
    wl = small_compact(seed=23, n_docs=90, block_docs=0, n_q=40)
    ref = oracle_index(wl)
    dix_c = device_index(wl)
    wl.block_docs = 128
    dix_k = device_index(wl)
    a = dix_c.query(wl.queries, wl.q_off, wl.thresholds)
    b = dix_k.query(wl.queries, wl.q_off, wl.thresholds)
    assert_results_equal(a, ref, wl.query_list(), wl.thresholds)
    for x, y in zip(a, b):
        assert x[0] == y[0] and x[1] == y[1] and np.array_equal(x[2], y[2]) and np.array_equal(x[3], y[3])


def test_save_load_roundtrip(compact, tmp_path):
    wl, ref, dix = compact
    hix = dix.download()
    p = str(tmp_path / "i.cobs")
    hix.save(p)
    dix2 = cobs.DeviceIndex.load(cobs.HostIndex.load(p))
    assert_index_equal(dix2, ref)
    got = dix2.query(wl.queries, wl.q_off, wl.thresholds)
    assert_results_equal(got, ref, wl.query_list(), wl.thresholds)


def test_errors():
    wl = small_compact(seed=29, n_docs=20, n_q=4, score_bits=16)
    dix = device_index(wl)
    thr = np.array([0, 500, 500, 500], np.uint16)
    with pytest.raises(cobs.CobsError) as e:
        dix.query(wl.queries, wl.q_off, thr)
    assert e.value.status == cobs.COBS_ERR_ARG
    big = np.frombuffer(b"A" * 70000, np.uint8)
    with pytest.raises(cobs.CobsError) as e:
        dix.query(big, np.array([0, 70000], np.uint64), np.array([500], np.uint16))
    assert e.value.status == cobs.COBS_ERR_OVERFLOW
    res = dix.query(np.zeros(0, np.uint8), np.zeros(1, np.uint64), np.zeros(0, np.uint16))
    assert res == []


def test_score_width_limits():
    """16-bit scores count at most 65,535: a query of exactly 65,535 windows runs in
    every form, and a document that holds it scores 65,535 (the largest 16-bit
    value, nothing wraps); one window more is refused with OVERFLOW, and 2^24
    windows (the batch plan's limit for any score width) with ARG."""
    k = 31
    lens = synth.lognormal_lengths(91, 40, 3000, 0.5, 500, 20000)
    docs, off = synth.dna_docs(91, lens)
    qmax = synth.dna_docs(92, [65535 + k - 1])[0].tobytes()
    extra = [qmax, qmax[:30000] + bytes(docs[:2000])]   # the query itself, and half of it
    db = np.concatenate([docs, np.frombuffer(b"".join(extra), np.uint8)])
    doff = np.concatenate([off, off[-1] + np.cumsum([len(x) for x in extra]).astype(np.uint64)])
    ql = [qmax, qmax[:40000], bytes(docs[int(off[3]):int(off[3]) + 900])]
    qo = np.zeros(len(ql) + 1, np.uint64)
    qo[1:] = np.cumsum([len(x) for x in ql])
    qb = np.frombuffer(b"".join(ql), np.uint8)
    thr = np.array([1000, 300, 500], np.uint16)
    wl = synth.Workload("score-width", 0, k, 1, 0.3, 16, 16, db, doff, qb, qo, thr, np.full(len(ql), -1))
    ref = oracle_index(wl)
    dix = device_index(wl)
    assert_index_equal(dix, ref)
    ell, mn, ids, sc = ref.query(ql[0], 1000)
    assert ell == 65535 and len(ids) >= 1 and int(sc[0]) == 65535 and int(ids[0]) == len(lens)
    for flags in FORMS:
        assert_results_equal(dix.query(qb, qo, thr, flags), ref, ql, thr)
    over = np.frombuffer(qmax + b"A", np.uint8)
    for flags in FORMS:
        with pytest.raises(cobs.CobsError) as e:
            dix.query(over, np.array([0, len(over)], np.uint64), np.array([500], np.uint16), flags)
        assert e.value.status == cobs.COBS_ERR_OVERFLOW
    wl32 = small_compact(seed=93, n_docs=30, n_q=2)
    d32 = device_index(wl32)
    huge = np.zeros((1 << 24) + k - 1, np.uint8)
    huge[:] = ord("A")
    with pytest.raises(cobs.CobsError) as e:
        d32.query(huge, np.array([0, len(huge)], np.uint64), np.array([500], np.uint16), cobs.COBS_BATCHED)
    assert e.value.status == cobs.COBS_ERR_ARG


def test_empty_and_tiny_documents():
    docs = [b"", b"ACG", b"ACGTACGTACGTACGTACGTACGTACGTACGTAC", b"N" * 50, b"GATTACA" * 10]
    off = np.zeros(len(docs) + 1, np.uint64)
    off[1:] = np.cumsum([len(d) for d in docs])
    db = np.frombuffer(b"".join(docs), np.uint8)
    qs = [b"GATTACAGATTACAGATTACAGATTACAGATTACA", b"ACGTACGTACGTACGTACGTACGTACGTACGTA", b"TTTT"]
    qo = np.zeros(4, np.uint64)
    qo[1:] = np.cumsum([len(x) for x in qs])
    qb = np.frombuffer(b"".join(qs), np.uint8)
    thr = np.array([1000, 500, 1000], np.uint16)
    for B in (0, 2):
        wl = synth.Workload("tiny", 0, 31, 1, 0.3, B, 32, db, off, qb, qo, thr, np.full(3, -1))
        ref = oracle_index(wl)
        dix = device_index(wl)
        assert_index_equal(dix, ref)
        for flags in FORMS:
            assert_results_equal(dix.query(qb, qo, thr, flags), ref, qs, thr)


def test_split_long_queries_small_batch():
    # A batch of a few long queries: each query longer than the part size (256 to
    # 4,080 terms, sized from the batch) runs as parts whose partial counts are
    # summed before the threshold.  Edge cases: a periodic query whose distinct
    # terms fill only its first part (the other parts count zero terms), windows
    # with non-ACGT bytes, K = 1 and K = 1000 permille, 4,080 and 4,081 windows.
    lens = synth.lognormal_lengths(61, 400, 25000, 0.5, 5000, 200000)
    docs, off = synth.dna_docs(61, lens)
    qb, qo, src = synth.dna_queries(62, 20, docs, off, n_tp=14, median=12000, sigma=0.8, lo=4000, hi=60000,
                                    rate_lo=0.0, rate_hi=0.005)
    ql = [bytes(qb[qo[i]:qo[i + 1]]) for i in range(20)]
    k = 31
    ql[0] = ql[0][:4080 + k - 1] if len(ql[0]) >= 4081 + k - 1 else ql[0]
    ql[1] = ql[1][:4081 + k - 1] if len(ql[1]) >= 4081 + k - 1 else ql[1]
    ql[2] = ql[2][:60] * 200
    ql[4] = ql[4][:1000] + b"N" * 40 + ql[4][1000:]
    qo2 = np.zeros(21, np.uint64)
    qo2[1:] = np.cumsum([len(x) for x in ql])
    qb2 = np.frombuffer(b"".join(ql), np.uint8)
    thr = synth.choice_u16(63, 20, [1, 300, 700, 1000])
    wl = synth.Workload("split", 0, k, 1, 0.3, 256, 32, docs, off, qb2, qo2, thr, src)
    ref = oracle_index(wl)
    dix = device_index(wl)
    assert_index_equal(dix, ref)
    windows = [max(0, len(x) - k + 1) for x in ql]
    for split in (0, 2, 1):
        eng = cobs.Engine(dix, split=split)
        for flags in (cobs.COBS_BATCHED, cobs.COBS_GRAPH):
            got = eng.query_host(qb2, qo2, thr, flags)
            st = eng.stats()
            if split == 1:
                assert st["split_queries"] == 0 and st["split_part"] == 0
            else:
                P = st["split_part"]
                assert 256 <= P <= 4080 and P % 16 == 0
                assert st["split_queries"] == sum(1 for w in windows if w > P) > 0
            assert_results_equal(got, ref, ql, thr)
    for i in range(5, 20):
        if src[i] >= 0 and thr[i] <= 700:
            assert src[i] in got[i][2].tolist()


def test_all_ones_qgram_short_and_long_queries():
    # The 8-byte q-gram of 0xFF bytes is the one code an open-addressing set
    # cannot hold; it is counted once per query, in short queries (set on chip)
    # and in long ones (one CTA per 2,048-window chunk), as the oracle does.
    rng = np.random.default_rng(11)
    docs = []
    for d in range(40):
        b = rng.integers(0, 256, 4000, dtype=np.uint8)
        if d % 3 == 0:
            b[500:540] = 0xFF
        docs.append(b.tobytes())
    off = np.zeros(len(docs) + 1, np.uint64)
    off[1:] = np.cumsum([len(x) for x in docs])
    db = np.frombuffer(b"".join(docs), np.uint8)
    qs = [docs[0][300:900], docs[3][100:3900] + b"\xff" * 30 + docs[6][0:3000], b"\xff" * 3000, b"\xff" * 9,
          docs[9][480:560], docs[1][0:2055], docs[2][0:2056] + b"\xff" * 8]
    qo = np.zeros(len(qs) + 1, np.uint64)
    qo[1:] = np.cumsum([len(x) for x in qs])
    qb = np.frombuffer(b"".join(qs), np.uint8)
    thr = np.array([500, 300, 1000, 1000, 700, 900, 800], np.uint16)
    for h in (1, 3):
        wl = synth.Workload("ones", 2, 8, h, 0.3, 16, 32, db, off, qb, qo, thr, np.full(len(qs), -1))
        ref = oracle_index(wl)
        dix = device_index(wl)
        assert_index_equal(dix, ref)
        for flags in FORMS:
            got = dix.query(qb, qo, thr, flags)
            assert_results_equal(got, ref, qs, thr)
            assert got[2][0] == 1 and got[3][0] == 1  # one distinct term each


def test_submit_host_pipelined_on_two_engines(compact):
    # Two engines on two streams alternate cobs_engine_submit_host and
    # cobs_engine_download over four sub-batches (one of them from page-locked
    # memory): each batch's results equal the oracle's.
    import torch
    wl, ref, dix = compact
    ql = wl.query_list()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    engs = [cobs.Engine(dix, stream=s1.cuda_stream), cobs.Engine(dix, stream=s2.cuda_stream)]
    cuts = [0, 40, 41, 100, len(ql)]
    batches = []
    for lo, hi in zip(cuts, cuts[1:]):
        qs = ql[lo:hi]
        off = np.zeros(len(qs) + 1, np.uint64)
        off[1:] = np.cumsum([len(x) for x in qs])
        qb = np.frombuffer(b"".join(qs), np.uint8)
        if lo == 41:  # page-locked query bytes: copied by DMA from this buffer
            pin = torch.empty(len(qb), dtype=torch.uint8, pin_memory=True).numpy()
            pin[:] = qb
            qb = pin
        batches.append((qs, qb, off, wl.thresholds[lo:hi]))
    for flags in (cobs.COBS_BATCHED, cobs.COBS_GRAPH):
        engs[0].submit_host(batches[0][1], batches[0][2], batches[0][3], flags)
        for i in range(1, len(batches) + 1):
            if i < len(batches):
                qs, qb, off, thr = batches[i]
                engs[i % 2].submit_host(qb, off, thr, flags)
            qs, qb, off, thr = batches[i - 1]
            assert_results_equal(engs[(i - 1) % 2].download(), ref, qs, thr)


@pytest.mark.parametrize("feed", [1, 2])
def test_gather_feeds_agree_with_the_oracle(compact, feed):
    # the single-hash gather fed by the cp.async ring (1) or by TMA gathers of
    # four indexed rows per copy (2): identical results, every counter class,
    # split parts, batched and graph forms, slice remainders of a ragged block
    wl, ref, dix = compact
    eng = cobs.Engine(dix, gather_feed=feed)
    for flags in (cobs.COBS_BATCHED, cobs.COBS_GRAPH):
        got = eng.query_host(wl.queries, wl.q_off, wl.thresholds, flags)
        assert_results_equal(got, ref, wl.query_list(), wl.thresholds)
    lens = synth.lognormal_lengths(97, 80, 30000, 0.4, 25000, 90000)
    docs, off = synth.dna_docs(97, lens)
    qb, qo, src = synth.dna_queries(98, 40, docs, off, n_tp=30, median=3000, sigma=1.2, lo=1, hi=30000,
                                    rate_lo=0.0, rate_hi=0.02)
    thr = synth.choice_u16(99, 40, [1, 500, 1000])
    wl2 = synth.Workload("feeds", 0, 31, 1, 0.3, 32, 32, docs, off, qb, qo, thr, src)
    ref2 = oracle_index(wl2)
    dix2 = device_index(wl2)
    for split in (0, 1):
        eng2 = cobs.Engine(dix2, gather_feed=feed, split=split)
        got = eng2.query_host(qb, qo, thr, cobs.COBS_BATCHED)
        assert_results_equal(got, ref2, wl2.query_list(), thr)


def test_gather_feed_tma_on_narrow_rows(cfg1):
    # cfg1: one classic block of 64 documents, 16-byte rows inside 128-byte boxes
    wl, ref, dix = cfg1
    eng = cobs.Engine(dix, gather_feed=2)
    got = eng.query_host(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
    assert_results_equal(got, ref, wl.query_list(), wl.thresholds)


def _autotune_and_check(wl, ref, dix):
    import torch
    eng = cobs.Engine(dix)
    dq = torch.from_numpy(wl.queries).cuda()
    do = torch.from_numpy(wl.q_off.view(np.int64)).cuda()
    dt = torch.from_numpy(wl.thresholds.view(np.int16)).cuda()
    cfg = eng.autotune(dq, do, wl.q_off, dt)
    widths = (32, 64, 128, 256) if wl.num_hashes == 1 else (32, 64, 128)
    assert cfg["slice_bytes"] in widths and cfg["ctas_per_sm"] >= 1 and cfg["l2_hints"] in (1, 2, 3, 4)
    assert (cfg["split"], cfg["split_part"]) in ((0, 0), (1, 0), (2, 4080), (2, 1024))
    assert cfg["class_streams"] in (0, 2)
    st = eng.stats()
    assert (st["slice_bytes"], st["ctas_per_sm"]) == (cfg["slice_bytes"], cfg["ctas_per_sm"])
    for flags in (cobs.COBS_BATCHED, cobs.COBS_GRAPH):
        got = eng.query_host(wl.queries, wl.q_off, wl.thresholds, flags)
        assert_results_equal(got, ref, wl.query_list(), wl.thresholds)
    # a second engine on the same index and batch shape takes the cached choice
    again = cobs.Engine(dix).autotune(dq, do, wl.q_off, dt)
    assert again.pop("from_cache")
    cfg.pop("from_cache")
    assert again == cfg


def test_autotune_single_hash(compact):
    # the sweep (slice width, CTAs per SM, L2 hints, term chunk, class streams)
    # ends on one of its shapes and the engine's results stay those of the oracle
    wl, ref, dix = compact
    _autotune_and_check(wl, ref, dix)


def test_autotune_three_hashes():
    wl = synth.config4(n_docs=300, n_q=80, n_words=2000, median=2500, lo=50, hi=20000, block_docs=128)
    _autotune_and_check(wl, oracle_index(wl), device_index(wl))


def test_slice_width_rules(compact):
    # 256-byte slices are the one-hash default when the blocks' rows pad to at
    # most 2 % more bytes than with 128-byte slices (128 otherwise, for the TMA
    # feed and for more hashes); only one hash may use them
    def expected(dix):
        rbs = [b["rowbytes"] for b in dix.info()["blocks"]]
        p128 = sum(-(-r // 128) * 128 for r in rbs)
        p256 = sum(-(-r // 256) * 256 for r in rbs)
        return 256 if p256 * 50 <= p128 * 51 else 128

    lens = np.full(8192, 60, np.uint64)  # one block of 8,192 documents: 1,024-byte rows
    docs, off = synth.dna_docs(401, lens)
    qb, qo, src = synth.dna_queries(402, 20, docs, off, n_tp=20, fixed_len=50, rate_lo=0.0, rate_hi=0.0)
    wide = synth.Workload("wide", 0, 31, 1, 0.3, 8192, 32, docs, off, qb, qo, np.full(20, 1000, np.uint16), src)
    wl, ref, dix = compact
    cases = [(wl, ref, dix), (wide, oracle_index(wide), device_index(wide))]
    assert [expected(c[2]) for c in cases] == [128, 256]
    for w, r, d in cases:
        for feed in (0, 2):
            eng = cobs.Engine(d, gather_feed=feed)
            got = eng.query_host(w.queries, w.q_off, w.thresholds, cobs.COBS_GRAPH)
            assert_results_equal(got, r, w.query_list(), w.thresholds)
            assert eng.stats()["slice_bytes"] == (expected(d) if feed == 0 else 128)
    wl3 = synth.config4(n_docs=40, n_q=5, n_words=500, median=800, lo=50, hi=2000, block_docs=16)
    dix3 = device_index(wl3)
    with pytest.raises(cobs.CobsError) as e:
        cobs.Engine(dix3, slice_bytes=256)
    assert e.value.status == cobs.COBS_ERR_ARG
    eng3 = cobs.Engine(dix3)
    eng3.query_host(wl3.queries, wl3.q_off, wl3.thresholds, cobs.COBS_BATCHED)
    assert eng3.stats()["slice_bytes"] == 128


def test_explicit_release_order(compact):
    # close() / with-blocks free objects at once; a device index refuses to close
    # while an engine, a server or a multi-index view on it is open
    wl, ref, _ = compact
    dix = device_index(wl)
    with cobs.Engine(dix) as eng:
        got = eng.query_host(wl.queries, wl.q_off, wl.thresholds, cobs.COBS_BATCHED)
        assert_results_equal(got, ref, wl.query_list(), wl.thresholds)
        with pytest.raises(RuntimeError):
            dix.close()
    srv = cobs.Server(dix)
    view = cobs.DeviceIndex.multi([dix])
    with pytest.raises(RuntimeError):
        dix.close()
    srv.close()
    with pytest.raises(RuntimeError):
        dix.close()
    view.close()
    dix.close()
    assert dix.h is None
