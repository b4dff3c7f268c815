"""Index merge (host code of the C ABI, no GPU): classic indexes with one common
Bloom width concatenate into the classic index of all their documents (Sec. 2.3),
pinned against the oracle's classic index built over the whole document list."""
import numpy as np
import pytest

import oracle
import synth
from paper_1905_09624_gb300 import cobs

from test_abi import _write_index_file


def _oracle_to_host(ix, path, **params):
    _write_index_file(path, cobs.make_params(**params), ix.blocks(), ix.perm(), ix.nterms(), ix.rows())
    return cobs.HostIndex.load(path)


def _docs(seed, n):
    lens = synth.lognormal_lengths(seed, n, 400, 0.5, 40, 3000)
    return synth.dna_docs(seed, lens)


def _part(docs, off, lo, hi):
    o = off[lo:hi + 1] - off[lo]
    return docs[int(off[lo]):int(off[hi])], o


@pytest.mark.parametrize("n_a", [8, 13, 130, 1])
def test_classic_merge_equals_classic_index_of_all_documents(tmp_path, n_a):
    docs, off = _docs(5, 150)
    W = 997
    full = oracle.build_index(oracle.make_params(block_docs=0, width_override=W), docs, off)
    da, oa = _part(docs, off, 0, n_a)
    db, ob = _part(docs, off, n_a, 150)
    a = _oracle_to_host(oracle.build_index(oracle.make_params(block_docs=0, width_override=W), da, oa),
                        str(tmp_path / "a.idx"), width=W)
    b = _oracle_to_host(oracle.build_index(oracle.make_params(block_docs=0, width_override=W), db, ob),
                        str(tmp_path / "b.idx"), width=W)
    m = a.merge(b).info()
    assert m["n_docs"] == 150 and len(m["blocks"]) == 1
    assert m["blocks"][0]["w"] == W and m["blocks"][0]["max_terms"] == full.blocks()[0]["max_terms"]
    assert m["blocks"] == full.blocks()
    assert np.array_equal(m["perm"], full.perm()) and np.array_equal(m["nterms"], full.nterms())
    assert np.array_equal(m["rows"], full.rows())


def test_compact_merge_keeps_both_block_lists(tmp_path):
    docs, off = _docs(6, 90)
    da, oa = _part(docs, off, 0, 50)
    db, ob = _part(docs, off, 50, 90)
    ra = oracle.build_index(oracle.make_params(block_docs=16), da, oa)
    rb = oracle.build_index(oracle.make_params(block_docs=8, fpr=0.1), db, ob)
    a = _oracle_to_host(ra, str(tmp_path / "a.idx"), block_docs=16)
    b = _oracle_to_host(rb, str(tmp_path / "b.idx"), block_docs=8, fpr=0.1)
    m = a.merge(b).info()
    assert m["n_docs"] == 90 and len(m["blocks"]) == len(ra.blocks()) + len(rb.blocks())
    # b's documents follow a's: sorted positions and ids shifted by 50, rows appended
    assert m["blocks"][:len(ra.blocks())] == ra.blocks()
    for got, want in zip(m["blocks"][len(ra.blocks()):], rb.blocks()):
        assert got["doc_begin"] == want["doc_begin"] + 50
        assert got["row_offset"] == want["row_offset"] + len(ra.rows())
        assert (got["w"], got["rowbytes"], got["n_docs"]) == (want["w"], want["rowbytes"], want["n_docs"])
    assert list(m["perm"]) == list(ra.perm()) + [p + 50 for p in rb.perm()]
    assert np.array_equal(m["rows"], np.concatenate([ra.rows(), rb.rows()]))
    # the merged file round-trips through the format checks
    p = str(tmp_path / "m.idx")
    a.merge(b).save(p)
    assert cobs.HostIndex.load(p).info()["blocks"] == m["blocks"]


def test_merge_refuses_different_terms(tmp_path):
    docs, off = _docs(7, 10)
    ra = oracle.build_index(oracle.make_params(q=31), docs, off)
    rb = oracle.build_index(oracle.make_params(q=21), docs, off)
    a = _oracle_to_host(ra, str(tmp_path / "a.idx"), q=31)
    b = _oracle_to_host(rb, str(tmp_path / "b.idx"), q=21)
    with pytest.raises(cobs.CobsError) as e:
        a.merge(b)
    assert e.value.status == cobs.COBS_ERR_ARG
