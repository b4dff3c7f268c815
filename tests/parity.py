"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the CPU oracle on the same seeded inputs, compare element by element."""
import numpy as np

import oracle
import synth
from paper_1905_09624_gb300 import cobs


def small_compact(seed=7, n_docs=600, median=3000, sigma=0.6, lo=40, hi=40000, block_docs=256, n_q=160,
                  q_len=300, kind=0, q=31, h=1, fpr=0.3, score_bits=32):
    """A compact DNA workload that spans several blocks with a ragged last block."""
    lens = synth.lognormal_lengths(seed, n_docs, median, sigma, lo, hi)
    docs, off = synth.dna_docs(seed, lens)
    qb, qo, src = synth.dna_queries(seed + 1, n_q, docs, off, n_tp=n_q // 2, fixed_len=q_len, rate_lo=0.0,
                                    rate_hi=0.03)
    thr = synth.choice_u16(seed + 2, n_q, [1, 500, 800, 1000])
    return synth.Workload("small-compact", kind, q, h, fpr, block_docs, score_bits, docs, off, qb, qo, thr, src)


def oracle_index(wl, threaded=False):
    P = oracle.make_params(**wl.params())
    if threaded:
        return oracle.build_index_threaded(P, wl.docs, wl.doc_off)
    return oracle.build_index(P, wl.docs, wl.doc_off)


def device_index(wl):
    return cobs.DeviceIndex.build(cobs.make_params(**wl.params()), wl.docs, wl.doc_off)


def assert_index_equal(dix, ref):
    info = dix.download().info()
    assert info["blocks"] == ref.blocks()
    assert np.array_equal(info["perm"], ref.perm())
    assert np.array_equal(info["nterms"], ref.nterms())
    got, want = info["rows"], ref.rows()
    assert got.shape == want.shape
    if not np.array_equal(got, want):
        bad = np.nonzero(got != want)[0]
        raise AssertionError(f"{len(bad)} index bytes differ, first at {bad[:8]}")


def assert_results_equal(got, ref, queries, thresholds, which=None):
    idx = range(len(queries)) if which is None else which
    for i in idx:
        ell, mn, ids, sc = ref.query(queries[i], int(thresholds[i]))
        g = got[i]
        assert (int(g[0]), int(g[1])) == (ell, mn), (i, g[0], g[1], ell, mn)
        assert np.array_equal(g[2], ids), (i, g[2][:10], ids[:10])
        assert np.array_equal(g[3], sc), (i, g[3][:10], sc[:10])
