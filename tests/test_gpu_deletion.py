"""Lazy deletion (Sec. 4.6) on the GPU: a set marked deleted is still scored
but never returned by top-k or the search pipeline; restoring it brings it
back; a call with an id out of range changes nothing.  Parity is with the
oracle's top-k over the same scores with the deleted ids excluded (bit-exact
for top-k; the search pipeline under the exhaustive-search tolerances)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gem():
    import paper_2603_20336_b300 as g
    return g


@pytest.fixture(scope="module")
def cfg(gem):
    w = synth.exact_fp32(n_sets=1500, n_queries=8)
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("f32", "bf16"))
    q = w.queries.vecs.cuda()
    qo = torch.from_numpy(w.queries.offsets).cuda()
    ws = gem.Workspace(store, max_queries=8, max_q_rows=int(w.queries.offsets[-1]), max_q_len=128,
                       max_cands=8 * 100, max_k=300)
    S64, L1 = oracle.score_all(w.queries.vecs, w.queries.offsets, w.docs.vecs, w.docs.offsets, with_l1=True)
    yield dict(w=w, store=store, ws=ws, q=q, qo=qo, S64=S64, L1=L1, N=store.n_sets)
    ws.close()
    store.close()


def _dead_set(S64, N, seed):
    """Every query's 3 best sets (so deletion changes every answer) plus a
    random tenth of the rest."""
    rng = np.random.default_rng(seed)
    top = {int(i) for b in range(S64.shape[0]) for i in np.argsort(-S64[b])[:3]}
    return sorted(top | set(rng.choice(N, N // 10, replace=False).tolist()))


def test_topk_skips_deleted_sets_and_restores(gem, cfg):
    N = cfg["N"]
    rng = np.random.default_rng(11)
    s = np.round(rng.standard_normal((4, N)), 2).astype(np.float32)    # heavy ties
    dead = sorted(set(np.argsort(-s[0])[:5].tolist()) | set(rng.choice(N, 200, replace=False).tolist()))
    gem.mark_deleted(cfg["store"], dead)
    try:
        for k in (1, 10, 300):
            ids, sc = gem.topk(cfg["ws"], torch.from_numpy(s).cuda(), k)
            ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
            for r in range(4):
                wi, ws_ = oracle.topk(s[r], k, exclude=set(dead))
                assert ids[r].tolist() == wi.tolist()
                np.testing.assert_array_equal(sc[r].astype(np.float64), ws_)
        # ragged rows with explicit ids: the bitmap is indexed by set id, ids past
        # the store's sets are never deleted
        lens = np.array([0, 9, 700, 40])
        off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        sr = np.round(rng.standard_normal(int(off[-1])), 1).astype(np.float32)
        idr = rng.permutation(2 * N)[: int(off[-1])].astype(np.int64)
        gi, gs = gem.topk(cfg["ws"], torch.from_numpy(sr).cuda(), 25, ids=torch.from_numpy(idr).cuda(),
                          row_offsets=torch.from_numpy(off).cuda())
        gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
        for r in range(4):
            seg = slice(off[r], off[r + 1])
            wi, ws_ = oracle.topk(sr[seg], 25, idr[seg], exclude=set(dead))
            m = len(wi)
            assert gi[r, :m].tolist() == wi.tolist()
            np.testing.assert_array_equal(gs[r, :m].astype(np.float64), ws_)
            assert np.all(gi[r, m:] == -1)
    finally:
        gem.mark_deleted(cfg["store"], dead, deleted=False)
    ids, _ = gem.topk(cfg["ws"], torch.from_numpy(s).cuda(), 10)
    assert ids.cpu().numpy()[0].tolist() == oracle.topk(s[0], 10)[0].tolist()


@pytest.mark.parametrize("compute", ["bf16", "f32"])
def test_search_never_returns_deleted_sets(gem, cfg, compute):
    S64, N = cfg["S64"], cfg["N"]
    dead = _dead_set(S64, N, 5)
    gem.mark_deleted(cfg["store"], dead)
    try:
        ids, sc = gem.search(cfg["store"], cfg["ws"], cfg["q"], cfg["qo"], compute, rerank_depth=100, k=10)
    finally:
        gem.mark_deleted(cfg["store"], dead, deleted=False)
    assert cfg["ws"].status() == 0
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    assert not set(ids.ravel().tolist()) & set(dead)
    for b in range(S64.shape[0]):
        wi, ws_ = oracle.topk(S64[b], 10, exclude=set(dead))
        for x in set(wi.tolist()) ^ set(ids[b].tolist()):
            assert abs(S64[b, x] - ws_[-1]) <= 1e-6 * max(1.0, abs(ws_[-1])), (b, x)
        err = np.abs(sc[b].astype(np.float64) - S64[b, ids[b]])
        assert np.all(err <= 1e-5 * cfg["L1"][b, ids[b]])


def test_deleting_every_set_returns_empty_rows(gem, cfg):
    N = cfg["N"]
    gem.mark_deleted(cfg["store"], np.arange(N))
    try:
        ids, sc = gem.search(cfg["store"], cfg["ws"], cfg["q"], cfg["qo"], "bf16", rerank_depth=20, k=5)
    finally:
        gem.mark_deleted(cfg["store"], np.arange(N), deleted=False)
    assert np.all(ids.cpu().numpy() == -1) and np.all(sc.cpu().numpy() == -np.inf)


def test_mark_deleted_rejects_ids_out_of_range_and_changes_nothing(gem, cfg):
    N = cfg["N"]
    s = np.zeros((1, N), np.float32)
    s[0, 7] = 1.0
    for bad in ([7, N], [-1, 7]):
        with pytest.raises(Exception):
            gem.mark_deleted(cfg["store"], bad)
        ids, _ = gem.topk(cfg["ws"], torch.from_numpy(s).cuda(), 1)
        assert ids.item() == 7
    gem.mark_deleted(cfg["store"], [])             # no ids: a no-op
