"""Incremental insertion (cobs_index_insert) against the oracle: each new
document goes to the free column of the block whose largest distinct-term count
is the smallest one still at least its own (input order, ties to the lower
block); the rest form new blocks planned like a build over them alone.  Checked
byte for byte: every old block afterwards equals the oracle's classic index of
its documents (old ones in sorted order, then the new ones) at the block's
width, and the new blocks equal the oracle's build over the rest."""
import numpy as np
import pytest

import oracle
import synth
from paper_1905_09624_gb300 import cobs

pytestmark = pytest.mark.gpu

P = dict(term_kind=0, q=31, num_hashes=1, fpr=0.3, block_docs=64, score_bits=32)


def _sub(docs, off, ids):
    parts = [bytes(docs[int(off[i]):int(off[i + 1])]) for i in ids]
    o = np.zeros(len(parts) + 1, np.uint64)
    o[1:] = np.cumsum([len(x) for x in parts])
    return np.frombuffer(b"".join(parts), np.uint8), o


def _expected_assignment(blocks, v_new):
    free = [b["rowbytes"] * 8 - b["n_docs"] for b in blocks]
    where, left = [], []
    for j, vj in enumerate(v_new):
        best = None
        for b, blk in enumerate(blocks):
            if free[b] and blk["max_terms"] >= vj and (best is None or blk["max_terms"] < blocks[best]["max_terms"]):
                best = b
        where.append(best)
        if best is None:
            left.append(j)
        else:
            free[best] -= 1
    return where, left


def test_insert_into_free_columns_and_new_blocks():
    docs_a, off_a = synth.dna_docs(91, synth.lognormal_lengths(91, 300, 3000, 0.6, 100, 20000))
    # new documents: most small enough for an existing block, some larger than any
    lens_e = np.concatenate([synth.lognormal_lengths(92, 70, 1500, 0.8, 40, 8000),
                             synth.lognormal_lengths(93, 10, 40000, 0.2, 30000, 60000)])
    docs_e, off_e = synth.dna_docs(94, lens_e)
    n_a, n_e = 300, len(lens_e)
    ref_a = oracle.build_index(oracle.make_params(**P), docs_a, off_a)
    host_a = cobs.DeviceIndex.build(cobs.make_params(**P), docs_a, off_a).download()
    assert host_a.info()["blocks"] == ref_a.blocks()

    ins = host_a.insert(docs_e, off_e)
    got = ins.info()
    v_new = oracle.doc_counts(docs_e, off_e, 0, n_e, P["term_kind"], P["q"])
    where, left = _expected_assignment(ref_a.blocks(), v_new)
    assert 0 < len(left) < n_e  # both paths are exercised
    assert np.array_equal(got["nterms"], np.concatenate([ref_a.nterms(), v_new]))

    rows = got["rows"]
    perm_a = ref_a.perm()
    pos = 0
    for b, blk in enumerate(ref_a.blocks()):
        mine = [j for j in range(n_e) if where[j] == b]
        g = got["blocks"][b]
        assert (g["n_docs"], g["w"], g["rowbytes"], g["row_offset"], g["max_terms"]) == \
            (blk["n_docs"] + len(mine), blk["w"], blk["rowbytes"], blk["row_offset"], blk["max_terms"])
        ids = list(perm_a[blk["doc_begin"]:blk["doc_begin"] + blk["n_docs"]]) + [n_a + j for j in mine]
        assert g["doc_begin"] == pos and list(got["perm"][pos:pos + len(ids)]) == ids
        pos += len(ids)
        # the block equals the classic index of its documents at its width
        da, oa = _sub(docs_a, off_a, ids[:blk["n_docs"]])
        de, oe = _sub(docs_e, off_e, mine)
        dcat = np.concatenate([da, de])
        ocat = np.concatenate([oa, oa[-1] + oe[1:]])
        cls = oracle.build_index(oracle.make_params(**dict(P, block_docs=0), width_override=blk["w"]), dcat, ocat)
        nbytes = blk["w"] * blk["rowbytes"]
        assert np.array_equal(rows[blk["row_offset"]:blk["row_offset"] + nbytes], cls.rows()), b
    # the rest: a build over them alone
    dl, ol = _sub(docs_e, off_e, left)
    ref_l = oracle.build_index(oracle.make_params(**P), dl, ol)
    base_row = len(ref_a.rows())
    nb_a = len(ref_a.blocks())
    for i, blk in enumerate(ref_l.blocks()):
        g = got["blocks"][nb_a + i]
        assert (g["n_docs"], g["w"], g["rowbytes"], g["max_terms"]) == \
            (blk["n_docs"], blk["w"], blk["rowbytes"], blk["max_terms"])
        assert g["row_offset"] == base_row + blk["row_offset"] and g["doc_begin"] == pos + blk["doc_begin"]
    assert list(got["perm"][pos:]) == [n_a + left[i] for i in ref_l.perm()]
    assert np.array_equal(rows[base_row:], ref_l.rows())

    # the new index answers queries: a document inserted into an old block is
    # found by its own substring at K = 1
    dix = cobs.DeviceIndex.load(ins)
    j = next(j for j in range(n_e) if where[j] is not None and lens_e[j] > 200)
    q = bytes(docs_e[int(off_e[j]) + 10:int(off_e[j]) + 150])
    qo = np.array([0, len(q)], np.uint64)
    res = dix.query(np.frombuffer(q, np.uint8), qo, np.array([1000], np.uint16), cobs.COBS_BATCHED)
    assert n_a + j in res[0][2].tolist()


def test_insert_into_a_classic_index():
    docs_a, off_a = synth.dna_docs(95, synth.lognormal_lengths(95, 50, 2000, 0.3, 500, 5000))
    docs_e, off_e = synth.dna_docs(96, synth.lognormal_lengths(96, 20, 2000, 0.3, 500, 9000))
    Pc = dict(P, block_docs=0)
    host_a = cobs.DeviceIndex.build(cobs.make_params(**Pc), docs_a, off_a).download()
    ref_a = oracle.build_index(oracle.make_params(**Pc), docs_a, off_a)
    got = host_a.insert(docs_e, off_e).info()
    v_new = oracle.doc_counts(docs_e, off_e, 0, 20, 0, 31)
    where, left = _expected_assignment(ref_a.blocks(), v_new)
    assert len(got["blocks"]) == (1 if not left else 2)
    assert got["n_docs"] == 70 and got["blocks"][0]["n_docs"] == 50 + sum(w is not None for w in where)
