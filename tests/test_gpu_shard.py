"""Doc-range sharded search on one GPU: a store split into 2 and 3 shard stores
(contiguous set ranges balanced by vector count), run through the exchange
protocol (per-shard first pass with global ids, merge of the shard-major lists
into the rerank pool, exact FP32 rerank of each pool entry by its owner, top-k),
must return gem_search's ids and scores on the whole store bit for bit."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gem():
    import paper_2603_20336_b300 as g
    return g


@pytest.fixture(scope="module")
def data(gem):
    w = synth.text_corpus(seed=77, n_sets=6000, n_queries=24, n_centres=256, device="cuda")
    full = gem.Store(w.docs.vecs, w.docs.offsets, keep=("f32", "bf16", "fp8"))
    C = gem.train_codebook(full, k1=512, iters=4, sample=0, seed=2)
    gem.set_codebook(full, C)
    q = w.queries.vecs
    qo = torch.from_numpy(w.queries.offsets).cuda()
    yield dict(w=w, full=full, C=C, q=q, qo=qo)
    full.close()


@pytest.mark.parametrize("n_shards", [2, 3])
@pytest.mark.parametrize("compute", ["bf16", "fp8", "f32", "codes"])
def test_sharded_search_bit_matches_single_store(gem, data, n_shards, compute):
    from paper_2603_20336_b300 import shard
    w, B, R, K = data["w"], 24, 200, 20
    ws_kw = dict(max_queries=B, max_q_rows=B * 32, max_q_len=32, max_cands=B * R, max_k=R)
    ws = gem.Workspace(data["full"], **ws_kw)
    want_i, want_s = gem.search(data["full"], ws, data["q"], data["qo"], compute, rerank_depth=R, k=K)
    assert ws.status() == 0
    ws.close()
    off = w.docs.offsets
    bounds = shard.shard_ranges(off, n_shards)
    shards = []
    for s in range(n_shards):
        a, b = int(bounds[s]), int(bounds[s + 1])
        st = gem.Store(w.docs.vecs[int(off[a]):int(off[b])], off[a:b + 1] - off[a], keep=("f32", "bf16", "fp8"))
        gem.set_codebook(st, data["C"])     # every shard holds the same codebook
        shards.append(shard.Shard(st, gem.Workspace(st, **ws_kw), a, b - a))
    try:
        got_i, got_s = shard.sharded_search(shard.GemEngine("cuda"), shards, n_shards, data["q"], data["qo"],
                                            compute, R, K)
        for sh in shards:
            assert sh.ws.status() == 0
        assert torch.equal(got_i, want_i)
        assert torch.equal(got_s.view(torch.int32), want_s.view(torch.int32))
        # vector balance of the ranges
        v = np.diff(off[bounds])
        assert v.max() - v.min() <= 2 * np.diff(off).max()
    finally:
        for sh in shards:
            sh.ws.close()
            sh.store.close()


def test_merge_topk_of_shard_major_lists(gem):
    """gem_merge_topk against a sort of the union (ties by lower id, empty slots)."""
    rng = np.random.default_rng(4)
    S, rows, k_in, k = 3, 5, 40, 25
    sc = np.round(rng.standard_normal((S, rows, k_in)), 1).astype(np.float32)
    ids = rng.permutation(10 * S * rows * k_in)[: S * rows * k_in].reshape(S, rows, k_in).astype(np.int64)
    ids[1, 2, :10] = -1
    gi = torch.empty((rows, k), dtype=torch.int64, device="cuda")
    gs = torch.empty((rows, k), dtype=torch.float32, device="cuda")
    scd, idd = torch.from_numpy(sc).cuda(), torch.from_numpy(ids).cuda()
    from paper_2603_20336_b300 import _check, _ptr, _stream, lib
    _check(lib.gem_merge_topk(_ptr(scd), _ptr(idd), S, rows, k_in, k, _ptr(gi), _ptr(gs), _stream()))
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
    import oracle
    for r in range(rows):
        s = sc[:, r].reshape(-1)
        i = ids[:, r].reshape(-1)
        keep = i >= 0
        wi, wsc = oracle.topk(s[keep], k, i[keep])
        np.testing.assert_array_equal(gi[r], wi)
        np.testing.assert_array_equal(gs[r].astype(np.float64), wsc)


@pytest.mark.parametrize("n_shards", [2, 3])
@pytest.mark.parametrize("compute", ["f32", "codes"])
def test_routed_candidate_lists_bit_match_single_store(gem, data, n_shards, compute):
    """Candidate lists of global ids (uneven lengths, an empty list, -1 entries)
    scored by their owner shards and combined by a max: bit-identical to
    gem_score_ids on the whole store."""
    from paper_2603_20336_b300 import shard
    w, B = data["w"], 24
    rng = np.random.default_rng(31)
    lens = rng.integers(0, 400, size=B)
    lens[5] = 0
    co = torch.from_numpy(np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)).cuda()
    ci = torch.from_numpy(rng.integers(-1, w.docs.n_sets, size=int(lens.sum())).astype(np.int64)).cuda()
    n = ci.numel()
    ws_kw = dict(max_queries=B, max_q_rows=B * 32, max_q_len=32, max_cands=n, max_k=16)
    ws = gem.Workspace(data["full"], **ws_kw)
    want = gem.score_ids(data["full"], ws, data["q"], data["qo"], co, ci, compute)
    assert ws.status() == 0
    ws.close()
    off = w.docs.offsets
    bounds = shard.shard_ranges(off, n_shards)
    shards = []
    for s in range(n_shards):
        a, b = int(bounds[s]), int(bounds[s + 1])
        st = gem.Store(w.docs.vecs[int(off[a]):int(off[b])], off[a:b + 1] - off[a], keep=("f32",))
        gem.set_codebook(st, data["C"])
        shards.append(shard.Shard(st, gem.Workspace(st, **ws_kw), a, b - a))
    try:
        got = shard.sharded_score_ids(shard.GemEngine("cuda"), shards, n_shards, data["q"], data["qo"], co, ci,
                                      compute)
        for sh in shards:
            assert sh.ws.status() == 0
        assert torch.equal(got.view(torch.int32), want.view(torch.int32))
    finally:
        for sh in shards:
            sh.ws.close()
            sh.store.close()
