"""Document-block sharding (host code of the C ABI, no GPU): the block planner,
the shard indexes and the merge of per-shard hit lists, pinned against the
oracle's index and results over all documents; and the exchange step of the
sharded bench path between world-size-2 gloo ranks."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_1905_09624_gb300 import cobs

from test_merge import _oracle_to_host


def _workload():
    lens = synth.lognormal_lengths(41, 700, 1200, 0.6, 40, 9000)
    docs, off = synth.dna_docs(41, lens)
    qb, qo, _ = synth.dna_queries(42, 60, docs, off, n_tp=40, fixed_len=0, median=300, sigma=0.8, lo=20, hi=3000,
                                  rate_lo=0.0, rate_hi=0.03)
    thr = synth.choice_u16(43, 60, [1, 300, 700, 1000])
    return docs, off, qb, qo, thr


@pytest.fixture(scope="module")
def indexed(tmp_path_factory):
    docs, off, qb, qo, thr = _workload()
    params = dict(block_docs=64)
    ref = oracle.build_index(oracle.make_params(**params), docs, off)
    host = _oracle_to_host(ref, str(tmp_path_factory.mktemp("shard") / "full.idx"), **params)
    ql = [bytes(qb[int(qo[i]):int(qo[i + 1])]) for i in range(len(qo) - 1)]
    want = [ref.query(q, int(thr[i])) for i, q in enumerate(ql)]
    return host, ref, want


def _bytes(b):
    return b["w"] * b["rowbytes"]


@pytest.mark.parametrize("n_shards", [1, 2, 3, 5, 16])
def test_plan_is_the_greedy_balance_of_block_bytes(indexed, n_shards):
    host, _, _ = indexed
    blocks = host.info()["blocks"]
    plan, load = host.shard_plan(n_shards)
    # the rule restated: blocks by decreasing bytes (stable), each to the least loaded shard (lowest on ties)
    want_load = [0] * n_shards
    want = [0] * len(blocks)
    for b in sorted(range(len(blocks)), key=lambda b: -_bytes(blocks[b])):
        s = min(range(n_shards), key=lambda s: (want_load[s], s))
        want[b] = s
        want_load[s] += _bytes(blocks[b])
    assert plan.tolist() == want and load.tolist() == want_load
    assert sum(load.tolist()) == sum(_bytes(b) for b in blocks)
    if n_shards <= len(blocks):  # LPT: no shard exceeds the mean by more than one block
        assert max(load) - sum(load) / n_shards <= max(_bytes(b) for b in blocks)


def test_shards_hold_the_blocks_their_documents_and_rows(indexed):
    host, ref, _ = indexed
    full = host.info()
    plan, _ = host.shard_plan(3)
    seen = []
    for s in range(3):
        sub, gids = host.shard(plan, s)
        si = sub.info()
        assert np.all(np.diff(gids.astype(np.int64)) > 0)  # increasing ids in the full index
        mine = [b for b in range(len(full["blocks"])) if plan[b] == s]
        assert len(si["blocks"]) == len(mine) and si["n_docs"] == len(gids)
        pos = 0
        for fb, sb in zip(mine, si["blocks"]):
            F = full["blocks"][fb]
            assert (sb["n_docs"], sb["w"], sb["rowbytes"], sb["max_terms"]) == \
                   (F["n_docs"], F["w"], F["rowbytes"], F["max_terms"])
            assert sb["doc_begin"] == pos
            fr = full["rows"][F["row_offset"]:F["row_offset"] + _bytes(F)]
            assert np.array_equal(si["rows"][sb["row_offset"]:sb["row_offset"] + _bytes(sb)], fr)
            # sorted position j of the block is the same document
            assert np.array_equal(gids[si["perm"][pos:pos + sb["n_docs"]]],
                                  full["perm"][F["doc_begin"]:F["doc_begin"] + F["n_docs"]])
            pos += sb["n_docs"]
        assert np.array_equal(si["nterms"], full["nterms"][gids])
        seen += gids.tolist()
    assert sorted(seen) == list(range(full["n_docs"]))


def _split_by_shard(want, plan_gids):
    """The oracle's full hit lists cut into per-shard results with shard-local ids."""
    out = []
    for gids in plan_gids:
        local = {int(g): j for j, g in enumerate(gids)}
        off, ids, sc = [0], [], []
        for _, _, qids, qsc in want:
            for i, v in zip(qids.tolist(), qsc.tolist()):
                if i in local:
                    ids.append(local[i])
                    sc.append(v)
            off.append(len(ids))
        out.append((np.array(off, np.uint64), np.array(ids, np.uint32), np.array(sc, np.uint32)))
    return out


@pytest.mark.parametrize("n_shards", [1, 2, 4])
def test_merge_restores_the_full_order(indexed, n_shards):
    host, _, want = indexed
    plan, _ = host.shard_plan(n_shards)
    gids = [host.shard(plan, s)[1] for s in range(n_shards)]
    parts = _split_by_shard(want, gids)
    # each shard's list keeps the order of the full list (local ids increase with ids)
    off, ids, sc = cobs.hits_merge(parts, gids)
    for q, (_, _, qids, qsc) in enumerate(want):
        assert np.array_equal(ids[off[q]:off[q + 1]], qids) and np.array_equal(sc[off[q]:off[q + 1]], qsc), q
    assert any(len(w[2]) > 50 for w in want)


def test_merge_rejects_bad_input():
    L = cobs.lib()
    assert L.cobs_hits_merge(1, 1, None, None, None, None, None, None, None) == cobs.COBS_ERR_ARG


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _exchange_worker(rank, world, port, parts, gids, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    maps = bench.gather_id_maps(gids[rank], dist)
    merged = bench.exchange_and_merge(parts[rank], maps, dist)
    if rank == 0:
        q.put(tuple(np.asarray(x).tolist() for x in merged))
    dist.barrier()
    dist.destroy_process_group()


def test_exchange_between_two_gloo_ranks(indexed):
    import torch.multiprocessing as mp
    host, _, want = indexed
    plan, _ = host.shard_plan(2)
    gids = [host.shard(plan, s)[1] for s in range(2)]
    parts = _split_by_shard(want, gids)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_exchange_worker, args=(r, 2, port, parts, gids, q)) for r in range(2)]
    for p in procs:
        p.start()
    off, ids, sc = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for k, (_, _, qids, qsc) in enumerate(want):
        assert ids[off[k]:off[k + 1]] == qids.tolist() and sc[off[k]:off[k + 1]] == qsc.tolist(), k
