"""Document-block sharding on one GPU: the index split into two shards by the
block planner, each shard a device index of its own queried in the graph form
(as two devices would), the two hit lists merged on the host; every query's
result equals the oracle's over the whole document list and the unsharded
index's."""
import numpy as np
import pytest

from paper_1905_09624_gb300 import cobs

from parity import device_index, oracle_index, small_compact

pytestmark = pytest.mark.gpu


def _graph(dix, wl):
    import torch
    s = torch.cuda.Stream()
    eng = cobs.Engine(dix, stream=s.cuda_stream)
    d_q = torch.from_numpy(wl.queries).cuda()
    d_off = torch.from_numpy(wl.q_off.view(np.int64)).cuda()
    d_thr = torch.from_numpy(wl.thresholds.view(np.int16)).cuda()
    torch.cuda.synchronize()
    eng.query_device(d_q, d_off, wl.q_off, d_thr, cobs.COBS_GRAPH)
    return eng.download_arrays()


@pytest.mark.parametrize("n_shards", [2, 3])
def test_sharded_queries_equal_the_oracle(n_shards):
    import torch
    torch.cuda.set_device(0)
    wl = small_compact(seed=83, n_docs=900, block_docs=128, n_q=150, q_len=400)
    dix = device_index(wl)
    host = dix.download()
    plan, load = host.shard_plan(n_shards)
    assert len(set(plan.tolist())) == n_shards  # every shard holds blocks
    parts, maps = [], []
    for s in range(n_shards):
        sub, gids = host.shard(plan, s)
        sres = _graph(cobs.DeviceIndex.load(sub), wl)
        # l and ceil(K l) depend on the query alone
        full = _graph(dix, wl) if s == 0 else full
        assert np.array_equal(sres[0], full[0]) and np.array_equal(sres[1], full[1])
        parts.append((sres[2], sres[3], sres[4]))
        maps.append(gids)
    off, ids, sc = cobs.hits_merge(parts, maps)
    assert np.array_equal(off, full[2]) and np.array_equal(ids, full[3]) and np.array_equal(sc, full[4])
    ref = oracle_index(wl)
    for i, q in enumerate(wl.query_list()):
        ell, mn, rids, rsc = ref.query(q, int(wl.thresholds[i]))
        assert (int(full[0][i]), int(full[1][i])) == (ell, mn)
        assert np.array_equal(ids[off[i]:off[i + 1]], rids) and np.array_equal(sc[off[i]:off[i + 1]], rsc), i
