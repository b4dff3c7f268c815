"""Multi-index querying and merged indexes on the GPU against the CPU oracle: a
view over several resident indexes, and the merged host index loaded back, must
score every document exactly as its own part does (ids shifted by the documents
of the parts before it)."""
import numpy as np
import pytest

import oracle
import synth
from paper_1905_09624_gb300 import cobs

pytestmark = pytest.mark.gpu

FORMS = [cobs.COBS_PLAIN, cobs.COBS_BATCHED, cobs.COBS_GRAPH]


def _expected(parts, query, thr):
    """Per part oracle results, ids shifted, merged by (score desc, id asc)."""
    ids, sc, ell, mn, base = [], [], None, None, 0
    for ref, n in parts:
        e, m, i, s = ref.query(query, thr)
        assert ell is None or (e, m) == (ell, mn)
        ell, mn = e, m
        ids += [int(x) + base for x in i]
        sc += [int(x) for x in s]
        base += n
    order = sorted(range(len(ids)), key=lambda j: (-sc[j], ids[j]))
    return ell, mn, [ids[j] for j in order], [sc[j] for j in order]


def _check(got, parts, queries, thr):
    for i, q in enumerate(queries):
        ell, mn, ids, sc = _expected(parts, q, int(thr[i]))
        g = got[i]
        assert (int(g[0]), int(g[1])) == (ell, mn), i
        assert g[2].tolist() == ids, (i, g[2][:8], ids[:8])
        assert g[3].tolist() == sc, i


@pytest.fixture(scope="module")
def three():
    lens = synth.lognormal_lengths(41, 700, 3000, 0.6, 40, 30000)
    docs, off = synth.dna_docs(41, lens)
    cuts = [0, 300, 550, 700]
    specs = [dict(block_docs=128), dict(block_docs=64, fpr=0.1), dict(block_docs=0)]  # the last is classic
    parts = []
    for (lo, hi), sp in zip(zip(cuts, cuts[1:]), specs):
        d = docs[int(off[lo]):int(off[hi])]
        o = off[lo:hi + 1] - off[lo]
        P = dict(term_kind=0, q=31, num_hashes=1, fpr=0.3, score_bits=32)
        P.update(sp)
        ref = oracle.build_index(oracle.make_params(**P), d, o)
        dix = cobs.DeviceIndex.build(cobs.make_params(**P), d, o)
        parts.append((ref, hi - lo, dix))
    qb, qo, _ = synth.dna_queries(42, 90, docs, off, n_tp=60, fixed_len=400, rate_lo=0.0, rate_hi=0.02)
    thr = synth.choice_u16(43, 90, [1, 300, 700, 1000])
    ql = [bytes(qb[qo[i]:qo[i + 1]]) for i in range(90)]
    return parts, qb, qo, thr, ql


@pytest.mark.parametrize("flags", FORMS)
def test_multi_index_view(three, flags):
    parts, qb, qo, thr, ql = three
    view = cobs.DeviceIndex.multi([p[2] for p in parts])
    info = view.info()
    assert info["n_docs"] == 700 and not info["rows_dev"]
    got = view.query(qb, qo, thr, flags)
    _check(got, [(r, n) for r, n, _ in parts], ql, thr)


def test_nested_view_and_merged_index_agree(three):
    parts, qb, qo, thr, ql = three
    inner = cobs.DeviceIndex.multi([parts[0][2], parts[1][2]])
    view = cobs.DeviceIndex.multi([inner, parts[2][2]])
    merged = parts[0][2].download().merge(parts[1][2].download()).merge(parts[2][2].download())
    # the view's download is the merged host index, byte for byte
    a, b = view.download().info(), merged.info()
    assert a["blocks"] == b["blocks"] and np.array_equal(a["perm"], b["perm"])
    assert np.array_equal(a["rows"], b["rows"]) and np.array_equal(a["nterms"], b["nterms"])
    loaded = cobs.DeviceIndex.load(merged)
    expect = [(r, n) for r, n, _ in parts]
    for dix in (view, loaded):
        eng = cobs.Engine(dix)
        _check(eng.query_host(qb, qo, thr, cobs.COBS_BATCHED), expect, ql, thr)


def test_classic_batches_merge_on_device():
    # classic indexes over batches of documents with one common width merge into
    # the classic index of all documents (the device build, the merge and the
    # oracle's classic index with that width agree byte for byte)
    lens = synth.lognormal_lengths(44, 90, 600, 0.5, 40, 5000)
    docs, off = synth.dna_docs(44, lens)
    W = 4001
    P = dict(term_kind=0, q=31, num_hashes=1, fpr=0.3, block_docs=0, score_bits=32)
    full_ref = oracle.build_index(oracle.make_params(width_override=W, **P), docs, off)
    merged = None
    for lo, hi in [(0, 37), (37, 61), (61, 90)]:
        d = docs[int(off[lo]):int(off[hi])]
        o = off[lo:hi + 1] - off[lo]
        part = cobs.DeviceIndex.build(cobs.make_params(width=W, **P), d, o).download()
        merged = part if merged is None else merged.merge(part)
    m = merged.info()
    assert m["blocks"] == full_ref.blocks()
    assert np.array_equal(m["rows"], full_ref.rows()) and np.array_equal(m["perm"], full_ref.perm())
    full_dev = cobs.DeviceIndex.build(cobs.make_params(width=W, **P), docs, off).download().info()
    assert np.array_equal(full_dev["rows"], m["rows"])


def test_multi_index_errors(three):
    parts, qb, qo, thr, ql = three
    sdix = cobs.DeviceIndex.load_streamed(parts[0][2].download())
    with pytest.raises(cobs.CobsError) as e:
        cobs.DeviceIndex.multi([parts[1][2], sdix])
    assert e.value.status == cobs.COBS_ERR_ARG
    lens = synth.lognormal_lengths(45, 5, 500, 0.3, 100, 1000)
    docs, off = synth.dna_docs(45, lens)
    other = cobs.DeviceIndex.build(cobs.make_params(q=21), docs, off)
    with pytest.raises(cobs.CobsError) as e:
        cobs.DeviceIndex.multi([parts[0][2], other])
    assert e.value.status == cobs.COBS_ERR_ARG
