"""Threshold top-k of long dense rows (the k-argmax of Eq. 2 over every stored
set) against the oracle's exact sort: bit-exact ids and scores, heavy ties,
signed zeros, explicit ids, deleted sets, and rows whose sample misleads the
threshold (the exact fallback over the whole row)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

N_COLS = 500_000   # the text-corpus row length (one score per stored set)


@pytest.fixture(scope="module")
def gem():
    import paper_2603_20336_b300 as g
    return g


@pytest.fixture(scope="module")
def env(gem):
    w = synth.exact_fp32(n_sets=300, n_queries=1)
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("f32",))
    ws = gem.Workspace(store, max_queries=8, max_q_rows=256, max_q_len=32, max_k=1000)
    yield dict(store=store, ws=ws)
    ws.close()
    store.close()


def _launches(gem, fn):
    n0 = gem.lib.gem_kernel_launches()
    out = fn()
    torch.cuda.synchronize()
    return out, gem.lib.gem_kernel_launches() - n0


def _check_rows(s, ids_got, sc_got, k, ids=None, exclude=None):
    for r in range(s.shape[0]):
        wi, ws_ = oracle.topk(s[r], k, None if ids is None else ids[r], exclude=exclude)
        m = len(wi)
        np.testing.assert_array_equal(ids_got[r, :m], wi)
        np.testing.assert_array_equal(sc_got[r, :m].astype(np.float64), ws_)
        assert np.all(ids_got[r, m:] == -1)


def _sampled_positions(cols, runs=256, run=32):
    q = np.arange(runs)
    starts = q * (cols - run) // (runs - 1)
    return (starts[:, None] + np.arange(run)[None, :]).ravel()


@pytest.mark.parametrize("k", [1, 100, 1000])
def test_threshold_topk_matches_oracle_with_heavy_ties(gem, env, k):
    rng = np.random.default_rng(k)
    s = np.round(rng.standard_normal((5, N_COLS)), 2).astype(np.float32)   # ~800 distinct values
    s[3] = 0.5                                                            # one row of equal scores
    s[4, ::7] = -0.0                                                      # signed zeros
    s[4, 3::7] = 0.0
    (gi, gs), n = _launches(gem, lambda: gem.topk(env["ws"], torch.from_numpy(s).cuda(), k))
    assert n == 3     # sample, filter, select
    _check_rows(s, gi.cpu().numpy(), gs.cpu().numpy(), k)


def test_threshold_topk_explicit_ids_and_deleted_sets(gem, env):
    rng = np.random.default_rng(5)
    s = rng.standard_normal((3, N_COLS)).astype(np.float32)
    ids = np.stack([rng.permutation(1 << 24)[:N_COLS] for _ in range(3)]).astype(np.int64)
    ids[:, 17] = -1                                                       # empty slots
    ids[0, :50] = np.arange(50)                                           # small ids: some deleted
    s[0, :50] = 10.0
    dead = np.array([3, 7, 11, 40], np.int64)
    gem.mark_deleted(env["store"], torch.from_numpy(dead).cuda())
    try:
        (gi, gs), n = _launches(gem, lambda: gem.topk(env["ws"], torch.from_numpy(s).cuda(), 1000,
                                                     ids=torch.from_numpy(ids).cuda()))
    finally:
        gem.mark_deleted(env["store"], torch.from_numpy(dead).cuda(), deleted=False)
    assert n == 3
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
    for r in range(3):
        keep = ids[r] >= 0
        wi, ws_ = oracle.topk(s[r][keep], 1000, ids[r][keep], exclude=set(dead.tolist()))
        np.testing.assert_array_equal(gi[r], wi)
        np.testing.assert_array_equal(gs[r].astype(np.float64), ws_)
    assert not set(dead.tolist()) & set(gi[0].tolist())


def test_threshold_topk_misleading_samples_fall_back_exactly(gem, env):
    """Row 0: every sampled position low, the rest high -- the threshold admits
    nearly the whole row and the candidate buffer overflows.  Row 1: every
    sampled position high, the rest low -- fewer than k keys reach the
    threshold.  Both rows take the exact row path."""
    pos = _sampled_positions(N_COLS)
    s = np.zeros((2, N_COLS), np.float32)
    s[0] = 1.0
    s[0, pos] = -1.0
    s[1] = -1.0
    s[1, pos] = 1.0
    (gi, gs), n = _launches(gem, lambda: gem.topk(env["ws"], torch.from_numpy(s).cuda(), 1000))
    assert n == 3
    _check_rows(s, gi.cpu().numpy(), gs.cpu().numpy(), 1000)


def test_short_rows_take_the_row_path(gem, env):
    rng = np.random.default_rng(9)
    s = np.round(rng.standard_normal((4, 30_000)), 1).astype(np.float32)
    (gi, gs), n = _launches(gem, lambda: gem.topk(env["ws"], torch.from_numpy(s).cuda(), 1000))
    assert n == 1     # 30,000 < 8 * (4 * 1000 + 256)
    _check_rows(s, gi.cpu().numpy(), gs.cpu().numpy(), 1000)
