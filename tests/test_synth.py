"""The seeded generators: determinism and workload shapes (no GPU)."""
import numpy as np

import synth


def test_deterministic_and_independent_of_threads():
    a, oa = synth.dna_docs(9, [100, 5000, 7], nthreads=1)
    b, ob = synth.dna_docs(9, [100, 5000, 7], nthreads=4)
    assert np.array_equal(a, b) and np.array_equal(oa, ob)
    assert set(np.unique(a).tolist()) <= set(b"ACGT")
    c, _ = synth.dna_docs(10, [100, 5000, 7])
    assert not np.array_equal(a, c)


def test_lognormal_lengths_clipped():
    L = synth.lognormal_lengths(3, 20000, 100_000, 0.3, 10_000, 1_000_000)
    assert L.min() >= 10_000 and L.max() <= 1_000_000
    assert abs(np.median(L) / 100_000 - 1) < 0.02
    assert abs(np.std(np.log(L)) - 0.3) < 0.01


def test_dna_queries_are_substrings_or_random():
    docs, off = synth.dna_docs(4, synth.lognormal_lengths(4, 50, 3000, 0.3, 1000, 9000))
    qb, qo, src = synth.dna_queries(5, 40, docs, off, n_tp=20, fixed_len=200)
    assert np.all(np.diff(qo) == 200)
    for i in range(20):
        d = src[i]
        assert bytes(qb[qo[i]:qo[i + 1]]) in bytes(docs[off[d]:off[d + 1]])
    assert np.all(src[20:] == -1)
    # substitutions keep the length and change about the requested fraction of bases
    qb2, qo2, src2 = synth.dna_queries(5, 40, docs, off, n_tp=40, fixed_len=2000, rate_lo=0.05, rate_hi=0.05)
    assert np.all(np.diff(qo2) == 2000)


def test_text_workload_shape():
    w = synth.config4(n_docs=300, n_q=200, n_words=5000)
    assert w.term_kind == synth.TERM_BYTES and w.q == 8 and w.num_hashes == 3
    lens = np.diff(w.q_off)
    assert lens.min() >= 50 and lens.max() <= 2 * 512
    assert set(np.unique(w.docs).tolist()) <= set(b"abcdefghijklmnopqrstuvwxyz ")


def test_config_shapes():
    w1 = synth.config1()
    assert w1.n_docs == 64 and w1.n_queries == 200 and np.all(np.diff(w1.doc_off) == 5000)
    assert np.sum(w1.src >= 0) == 100 and np.all(w1.thresholds == 800)


def test_workload_file_matches_the_recipes():
    # the JSON workload file holds exactly the recipes' default parameters, and a
    # workload built from it is the recipe's workload byte for byte
    import inspect
    import json
    table = json.load(open(synth.WORKLOADS_JSON))
    for name in ("cfg1", "cfg2", "cfg3", "cfg4"):
        fn = getattr(synth, table[name]["recipe"])
        defaults = {k: (list(v.default) if isinstance(v.default, tuple) else v.default)
                    for k, v in inspect.signature(fn).parameters.items()}
        assert table[name]["params"] == defaults, name
    sig = inspect.signature(synth.config5_queries)
    assert synth.serving_params() == {k: v.default for k, v in sig.parameters.items() if k != "wl2"}
    a, b = synth.workload("cfg1"), synth.config1()
    assert np.array_equal(a.docs, b.docs) and np.array_equal(a.queries, b.queries)
    assert np.array_equal(a.thresholds, b.thresholds) and a.params() == b.params()
    small = synth.workload("cfg1", n_docs=8, n_q=10)
    assert small.n_docs == 8 and small.n_queries == 10
