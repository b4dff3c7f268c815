"""Pins of the CPU oracle to things other than itself (no GPU needed).

Each test ties one oracle function to the paper (Sec. 2.1-2.3), a closed form,
an independent implementation or brute force, chosen so that a dropped term, a
wrong sign or index, or a transposed operand in the oracle fails one of them.
"""
import ctypes
import ctypes.util
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ XXH64
def _libxxhash():
    for name in ("libxxhash.so.0", "libxxhash.so", ctypes.util.find_library("xxhash")):
        if not name:
            continue
        try:
            lib = ctypes.CDLL(name)
            lib.XXH64.restype = ctypes.c_uint64
            lib.XXH64.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64]
            return lib
        except OSError:
            continue
    return None


def test_xxh64_spec_empty_input():
    # The xxHash specification's published value for the empty input, seed 0.
    assert oracle.xxh64(b"", 0) == 0xEF46DB3751D8E999


def test_xxh64_known_answers_fixture():
    # XXH64 answers written once by the reference xxHash library
    # (tests/golden/make_xxh64_fixture.py): every length 0..72 (stripe loop and
    # all tails), longer inputs and 8-byte term codes, five seeds.  Runs whether
    # or not the library is installed here.
    n = 0
    for ln in open(os.path.join(GOLDEN, "xxh64_known_answers.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        f = ln.split()
        length, seed, want = int(f[0]), int(f[1]), int(f[2], 16)
        data = bytes.fromhex(f[3]) if len(f) > 3 else b""
        assert len(data) == length
        assert oracle.xxh64(data, seed) == want, (length, seed)
        if length == 8 and seed < 8:  # the hashed form of a term, seed = hash index
            assert oracle.hash_term(int.from_bytes(data, "little"), seed) == want
        n += 1
    assert n >= 400


def test_xxh64_against_libxxhash():
    lib = _libxxhash()
    if lib is None:
        pytest.skip("libxxhash not installed")
    rng = np.random.default_rng(7)
    for n in list(range(0, 80)) + [100, 255, 1000]:
        data = rng.integers(0, 256, size=n, dtype=np.uint8).tobytes()
        for seed in (0, 1, 2, 0xFFFFFFFFFFFFFFFF, 12345678901234567):
            buf = ctypes.create_string_buffer(data, max(n, 1))
            assert oracle.xxh64(data, seed) == lib.XXH64(buf, n, seed), (n, seed)


def test_hash_term_is_xxh64_of_le_bytes():
    lib = _libxxhash()
    if lib is None:
        pytest.skip("libxxhash not installed")
    for t in (0, 1, 0x0123456789ABCDEF, (1 << 62) - 1, 0xFFFFFFFFFFFFFFFF):
        le = t.to_bytes(8, "little")
        for i in range(4):
            assert oracle.hash_term(t, i) == lib.XXH64(ctypes.create_string_buffer(le, 8), 8, i)


# ------------------------------------------------------------------ terms
def _code(s):
    v = 0
    for ch in s:
        v = v * 4 + "ACGT".index(ch)
    return v


def _revcomp(s):
    return s[::-1].translate(str.maketrans("ACGT", "TGCA"))


@pytest.mark.parametrize("k", [1, 2, 3, 5, 6])
def test_dna_terms_brute_force(k):
    # Every string of length k: forward code is the base-4 number (first base most
    # significant); canonical = min(code, code(reverse complement)).
    for tup in itertools.product("ACGT", repeat=k):
        s = "".join(tup)
        fwd = oracle.terms(s.encode(), 1, k)
        can = oracle.terms(s.encode(), 0, k)
        assert list(fwd) == [_code(s)]
        assert list(can) == [min(_code(s), _code(_revcomp(s)))]


def test_terms_windows_and_invalid_bytes():
    s = b"ACGTNACGTTA"
    # windows of length 4 containing N are skipped
    got = oracle.terms(s, 1, 4)
    want = [_code(s[j:j + 4].decode()) for j in range(len(s) - 3) if b"N" not in s[j:j + 4]]
    assert list(got) == want
    assert len(oracle.terms(b"ACG", 1, 4)) == 0
    assert len(oracle.terms(b"acgt", 1, 2)) == 0  # lower case is not in the alphabet


def test_byte_qgrams_little_endian():
    s = b"hello world"
    for q in (1, 3, 8):
        got = oracle.terms(s, 2, q)
        want = [int.from_bytes(s[j:j + q], "little") for j in range(len(s) - q + 1)]
        assert list(got) == want


def test_distinct_terms_is_a_set():
    s = b"ACGACGACGACG"
    d = oracle.distinct_terms(s, 1, 3)
    assert list(d) == sorted({_code(s[j:j + 3].decode()) for j in range(len(s) - 2)})


# ------------------------------------------------------- Bloom size formula
@pytest.mark.parametrize("h,p", [(1, 0.3), (3, 0.1), (2, 0.05), (1, 0.01)])
def test_bloom_width_is_smallest_meeting_bound(h, p):
    # Sec. 2.1: the false-positive rate is at most (1 - e^{-hv/w})^h.  The width
    # must be the smallest integer w for which that bound is <= p.
    for v in (1, 2, 7, 100, 4970, 123457, 10_000_000):
        w = oracle.bloom_width(h, v, p)
        assert (1 - math.exp(-h * v / w)) ** h <= p * (1 + 1e-12)
        if w > 1:
            assert (1 - math.exp(-h * v / (w - 1))) ** h > p * (1 - 1e-12)


def test_bloom_width_ratios_and_empty():
    assert oracle.bloom_width(1, 10 ** 7, 0.3) / 10 ** 7 == pytest.approx(2.80367, abs=2e-5)
    assert oracle.bloom_width(3, 10 ** 7, 0.1) / 10 ** 7 == pytest.approx(4.80833, abs=2e-5)
    assert oracle.bloom_width(1, 0, 0.3) == 1


def test_bloom_fpr_exact_vs_bound():
    # Sec. 2.1 prints (1-(1-1/w)^{hv})^h <= (1-e^{-hv/w})^h, but (1-1/w)^x <= e^{-x/w},
    # so the exponential form is the SMALLER one; the gap is O(hv/w^2).  Both forms
    # are checked against their closed forms and the true direction is asserted.
    for h, v, w in [(1, 100, 280), (3, 50, 240), (2, 1, 1), (1, 10 ** 6, 2803670)]:
        exact = oracle.bloom_fpr(h, v, w)
        bound = oracle.bloom_fpr_bound(h, v, w)
        assert exact == pytest.approx((1 - (1 - 1 / w) ** (h * v)) ** h, rel=1e-12)
        assert bound == pytest.approx((1 - math.exp(-h * v / w)) ** h, rel=1e-12)
        assert bound <= exact + 1e-15
        if w > 1:
            assert exact - bound < 2.0 * h * h * v / w ** 2 + 1e-12


# ---------------------------------------------------- Theorem 1 and Chernoff
def _golden_worked_example():
    with open(os.path.join(GOLDEN, "worked_example_theorem1.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    l, p, K, val, digits = rows[0]
    return int(l), float(p), float(K), float(val), int(digits)


def test_theorem1_worked_example():
    l, p, K, printed, digits = _golden_worked_example()
    t = math.floor(K * l) + 1          # "more than floor(K l)" false-positive terms
    got = oracle.binom_tail_ge(l, p, t)
    assert round(got, 6) == printed     # 0.000143
    # the other reading (at least floor(K l)) does not reproduce the printed value
    assert round(oracle.binom_tail_ge(l, p, t - 1), 6) != printed


def test_binomial_tail_exact_rational():
    # exact sums in rational arithmetic on small cases
    for l in (1, 5, 12, 30):
        for p in (Fraction(3, 10), Fraction(1, 7)):
            for t in range(0, l + 2):
                exact = sum(Fraction(math.comb(l, i)) * p ** i * (1 - p) ** (l - i) for i in range(t, l + 1))
                assert oracle.binom_tail_ge(l, float(p), t) == pytest.approx(float(exact), rel=1e-9, abs=1e-300)
                if t <= l:
                    pm = Fraction(math.comb(l, t)) * p ** t * (1 - p) ** (l - t)
                    assert oracle.binom_pmf(l, float(p), t) == pytest.approx(float(pm), rel=1e-9)


def test_chernoff_bounds_tail():
    for l in (31, 70, 100, 1000):
        for K in (0.4, 0.5, 0.8, 1.0):
            p = 0.3
            tail = oracle.binom_tail_ge(l, p, math.floor(K * l) + 1)
            assert tail <= oracle.chernoff(l, K, p) + 1e-300


# ------------------------------------------------------------- index/query
def _small_dna(n_docs, length, seed, k=5):
    docs, off = synth.dna_docs(seed, np.full(n_docs, length, dtype=np.uint64))
    return docs, off


def _brute_scores(docs, off, query, k, kind):
    def tset(s):
        out = set()
        for j in range(len(s) - k + 1):
            w = s[j:j + k]
            if kind == 2:
                out.add(int.from_bytes(w, "little"))
                continue
            if any(c not in b"ACGT" for c in w):
                continue
            ws = w.decode()
            c = _code(ws)
            out.add(min(c, _code(_revcomp(ws))) if kind == 0 else c)
        return out
    T = tset(query)
    return len(T), [len(T & tset(bytes(docs[off[d]:off[d + 1]]))) for d in range(len(off) - 1)]


@pytest.mark.parametrize("block_docs", [0, 3, 4, 64])
@pytest.mark.parametrize("h", [1, 2])
def test_exact_mode_equals_brute_force_containment(block_docs, h):
    # Identity hash and w >= 4^k: every distinct term has its own row, so the
    # bit-sliced Bloom index is an exact inverted index (Sec. 2.2) and the q-gram
    # score equals |G_q(P) & G_q(d)|.
    k = 5
    rng = np.random.default_rng(11)
    lens = rng.integers(40, 200, size=11).astype(np.uint64)
    lens[3] = 4  # a document shorter than k has no terms
    docs, off = synth.dna_docs(5, lens)
    prm = oracle.make_params(term_kind=0, q=k, num_hashes=h, fpr=0.3, block_docs=block_docs,
                             hash_kind=oracle.HASH_IDENTITY, width_override=4 ** k)
    ix = oracle.build_index(prm, docs, off)
    for qi in range(8):
        d = qi % 11 if qi % 11 != 3 else 4
        s = bytes(docs[off[d]:off[d + 1]])
        a = int(rng.integers(0, len(s) - 30))
        query = s[a:a + 30] if qi % 2 == 0 else synth.dna_docs(100 + qi, [30])[0].tobytes()
        l, sc = ix.scores(query)
        bl, bs = _brute_scores(docs, off, query, k, 0)
        assert l == bl
        assert list(sc) == bs
        for thr in (1, 500, 800, 1000):
            ell, mn, ids, scs = ix.query(query, thr)
            assert mn == math.ceil(Fraction(thr * l, 1000))
            want = sorted([(s_, i) for i, s_ in enumerate(bs) if s_ >= mn and l > 0], key=lambda x: (-x[0], x[1]))
            assert list(zip(scs.tolist(), ids.tolist())) == want


def test_exact_mode_bytes_kind():
    q = 3
    docs = np.frombuffer(b"the cat sat on the mat" + b"a dog ate the hat" + b"zzz", dtype=np.uint8)
    off = np.array([0, 22, 39, 42], dtype=np.uint64)
    prm = oracle.make_params(term_kind=2, q=q, num_hashes=1, fpr=0.3, block_docs=2,
                             hash_kind=oracle.HASH_IDENTITY, width_override=1 << 24)
    ix = oracle.build_index(prm, docs, off)
    for query in (b"the mat", b"dog hat", b"zzzz", b"qq"):
        l, sc = ix.scores(query)
        bl, bs = _brute_scores(docs, off, query, q, 2)
        assert (l, list(sc)) == (bl, bs)


def test_superset_and_no_false_negatives_xxh64():
    # Sec. 2.2: Bloom scores can only exceed exact containment; every substring
    # of a document (length >= q) returns that document at K = 1.0 with score l.
    docs, off = synth.dna_docs(21, synth.lognormal_lengths(21, 40, 3000, 0.5, 500, 20000))
    prm = oracle.make_params(term_kind=0, q=31, num_hashes=1, fpr=0.3, block_docs=16)
    ix = oracle.build_index(prm, docs, off)
    rng = np.random.default_rng(3)
    for it in range(12):
        d = int(rng.integers(0, 40))
        s = bytes(docs[off[d]:off[d + 1]])
        L = int(rng.integers(31, 200))
        a = int(rng.integers(0, len(s) - L + 1))
        query = s[a:a + L]
        l, sc = ix.scores(query)
        el, ex = oracle.exact_scores(docs, off, 0, 31, query)
        assert l == el
        assert np.all(sc >= ex)
        ell, mn, ids, scs = ix.query(query, 1000)
        assert mn == l and d in ids.tolist()
        assert scs[ids.tolist().index(d)] == l


def test_classic_equals_compact_single_block():
    # Sec. 2.3: each compact sub-index is a classic index; with one block (B >= |D|)
    # the two return identical results (the column order differs).
    docs, off = synth.dna_docs(31, synth.lognormal_lengths(31, 20, 2000, 0.5, 300, 9000))
    a = oracle.build_index(oracle.make_params(block_docs=0), docs, off)
    b = oracle.build_index(oracle.make_params(block_docs=32), docs, off)
    assert a.blocks()[0]["w"] == b.blocks()[0]["w"]
    assert not np.array_equal(a.perm(), b.perm())
    qb, qo, src = synth.dna_queries(32, 30, docs, off, n_tp=15, fixed_len=120, rate_lo=0.0, rate_hi=0.05)
    for i in range(30):
        query = bytes(qb[qo[i]:qo[i + 1]])
        for thr in (500, 800, 1000):
            ra, rb = a.query(query, thr), b.query(query, thr)
            assert ra[0] == rb[0] and ra[1] == rb[1]
            assert np.array_equal(ra[2], rb[2]) and np.array_equal(ra[3], rb[3])


def test_compact_plan_layout():
    docs, off = synth.dna_docs(41, synth.lognormal_lengths(41, 37, 1500, 0.6, 100, 9000))
    ix = oracle.build_index(oracle.make_params(block_docs=8), docs, off)
    v = ix.nterms()
    perm = ix.perm()
    # stable order by (v, id)
    assert list(perm) == sorted(range(37), key=lambda d: (int(v[d]), d))
    blocks = ix.blocks()
    assert [b["n_docs"] for b in blocks] == [8, 8, 8, 8, 5]
    off_b = 0
    for b in blocks:
        vb = max(int(v[perm[b["doc_begin"] + j]]) for j in range(b["n_docs"]))
        assert b["max_terms"] == vb
        assert b["w"] == oracle.bloom_width(1, vb, 0.3)
        assert b["rowbytes"] == 16
        assert b["row_offset"] == off_b
        off_b += b["w"] * b["rowbytes"]
    rows = ix.rows()
    assert len(rows) == off_b
    # padding columns (j >= n_docs) are never set
    for b in blocks:
        m = rows[b["row_offset"]:b["row_offset"] + b["w"] * 16].reshape(b["w"], 16)
        bits = np.unpackbits(m, axis=1, bitorder="little")
        assert not bits[:, b["n_docs"]:].any()
        # each document's column holds at most v_d set bits and at least one if v_d > 0
        for j in range(b["n_docs"]):
            vd = int(v[perm[b["doc_begin"] + j]])
            assert 1 <= bits[:, j].sum() <= vd


def test_false_positive_statistics_binomial():
    # Sec. 2.1, Theorem 1: for terms absent from a document, lookups are
    # (approximately) independent Bernoulli trials with the filter's fill rate.
    # Random 31-mers are absent from every document with overwhelming probability,
    # so each document's score on a random query ~ Binomial(l, f_d), f_d = the
    # fraction of set bits in its column; f_d itself ~ 1 - (1 - 1/w)^v_d.
    docs, off = synth.dna_docs(51, synth.lognormal_lengths(51, 24, 20000, 0.4, 5000, 60000))
    ix = oracle.build_index(oracle.make_params(block_docs=8), docs, off)
    rows, perm, v = ix.rows(), ix.perm(), ix.nterms()
    fill = np.zeros(24)
    for b in ix.blocks():
        m = rows[b["row_offset"]:b["row_offset"] + b["w"] * b["rowbytes"]].reshape(b["w"], b["rowbytes"])
        bits = np.unpackbits(m, axis=1, bitorder="little")
        for j in range(b["n_docs"]):
            d = int(perm[b["doc_begin"] + j])
            fill[d] = bits[:, j].mean()
            expect = 1 - (1 - 1 / b["w"]) ** int(v[d])
            sd = math.sqrt(expect * (1 - expect) / b["w"])
            assert abs(fill[d] - expect) < 6 * sd + 1e-9
            assert fill[d] <= 0.3 + 6 * sd                     # at most the design rate
    qb, qo, _ = synth.dna_queries(52, 400, docs, off, n_tp=0, fixed_len=100)
    ells, hist = [], np.zeros((24, 71))
    for i in range(400):
        l, sc = ix.scores(bytes(qb[qo[i]:qo[i + 1]]))
        ells.append(l)
        if l == 70:
            for d in range(24):
                hist[d, sc[d]] += 1
    # chi-square of the pooled score distribution against the mixture of binomials
    n70 = hist[0].sum()
    assert n70 > 300
    pooled = hist.sum(0)
    expect = np.zeros(71)
    for d in range(24):
        expect += n70 * np.array([oracle.binom_pmf(70, fill[d], i) for i in range(71)])
    # merge sparse tails
    obs, exp_ = [], []
    acc_o = acc_e = 0.0
    for i in range(71):
        acc_o += pooled[i]
        acc_e += expect[i]
        if acc_e >= 20:
            obs.append(acc_o); exp_.append(acc_e); acc_o = acc_e = 0.0
    obs[-1] += acc_o; exp_[-1] += acc_e
    chi2 = sum((o - e) ** 2 / e for o, e in zip(obs, exp_))
    dof = len(obs) - 1
    from scipy.stats import chi2 as chi2d
    assert chi2d.sf(chi2, dof) > 1e-4, (chi2, dof)
    # mean score matches l * mean fill
    assert pooled @ np.arange(71) / (24 * n70) == pytest.approx(70 * fill.mean(), rel=0.02)


def test_generated_inputs_exact_mode_and_superset():
    # Generated small corpora (ACGT with some N, empty and short documents, k = 1..6,
    # 1-2 hashes, classic and tiny blocks): in exact mode (identity hash, w = 4^k)
    # every score equals brute-force containment; with XXH64 every score is at
    # least the containment (Sec. 2.2: one-sided error).
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=60, deadline=None, derandomize=True)
    @hyp.given(docs=st.lists(st.text(alphabet="ACGTN", max_size=60), min_size=1, max_size=7),
               query=st.text(alphabet="ACGTN", max_size=40), k=st.integers(1, 6), h=st.integers(1, 2),
               block_docs=st.sampled_from([0, 1, 2, 3]), canonical=st.booleans())
    def check(docs, query, k, h, block_docs, canonical):
        raw = [d.encode() for d in docs]
        buf = np.frombuffer(b"".join(raw) or b"\0", dtype=np.uint8)[:sum(len(r) for r in raw)].copy()
        off = np.zeros(len(raw) + 1, np.uint64)
        off[1:] = np.cumsum([len(r) for r in raw])
        kind = 0 if canonical else 1
        q = query.encode()
        bl, bs = _brute_scores(buf, off, q, k, kind)
        exact = oracle.build_index(oracle.make_params(term_kind=kind, q=k, num_hashes=h, fpr=0.3,
                                                      block_docs=block_docs, hash_kind=oracle.HASH_IDENTITY,
                                                      width_override=4 ** k), buf, off)
        l, sc = exact.scores(q)
        assert (l, list(sc)) == (bl, bs)
        bloom = oracle.build_index(oracle.make_params(term_kind=kind, q=k, num_hashes=h, fpr=0.3,
                                                      block_docs=block_docs), buf, off)
        l2, sc2 = bloom.scores(q)
        assert l2 == bl and all(a >= b for a, b in zip(sc2.tolist(), bs))

    check()
