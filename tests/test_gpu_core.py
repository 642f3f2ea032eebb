"""GPU parity of the store, exact scoring (FP32 SIMT and BF16 tensor cores),
id-list scoring, top-k and the search pipeline against the FP64 oracle.

Tolerances (also derived in the design notes):
  FP32 path:  |s - s64| <= 1e-5 * sum_i |max_j <q_i, p_j>|  (relative to the L1
              of the per-query-vector terms; 128-term FMA chains of unit vectors
              carry ~1e-7 relative error per term)
  BF16 path:  |s - s64| <= 2e-2 per score against the FP64 score of the FP32
              inputs (storage rounding), and <= 2e-4 * m_q against the FP64
              score of the bf16-rounded inputs (FP32 accumulation only)
"""
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
def cfg1(gem):
    w = synth.exact_fp32()
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("f32", "bf16", "fp8"))
    q = w.queries.vecs.cuda()
    qo = torch.from_numpy(w.queries.offsets).cuda()
    ws = gem.Workspace(store, max_queries=64, max_q_rows=4096, max_q_len=128, max_cands=64 * 256,
                       max_k=256)
    S64, L1 = oracle.score_all(w.queries.vecs, w.queries.offsets, w.docs.vecs, w.docs.offsets,
                               with_l1=True)
    return dict(w=w, store=store, ws=ws, q=q, qo=qo, S64=S64, L1=L1)


def _padded_source_rows(off):
    """Source row of every padded row: each set rounded up to a multiple of 8
    rows, the extra rows repeating the set's last vector."""
    lens = np.diff(off)
    plens = (lens + 7) // 8 * 8
    src = []
    for d in range(len(lens)):
        r = np.arange(plens[d])
        src.append(off[d] + np.minimum(r, lens[d] - 1))
    return np.concatenate([[0], np.cumsum(plens)]), np.concatenate(src)


def test_store_copies_match_oracle_rounding(gem, cfg1):
    w, store = cfg1["w"], cfg1["store"]
    X = w.docs.vecs.numpy()
    pad_off, src = _padded_source_rows(w.docs.offsets)
    np.testing.assert_array_equal(store.export("pad_offsets").cpu().numpy(), pad_off)
    assert store.n_pad_vecs == pad_off[-1]
    bits = store.export("bf16").cpu().numpy().view(np.uint16)
    want = oracle.bf16_round(X[src]).view(np.uint32) >> 16
    np.testing.assert_array_equal(bits.astype(np.uint32), want.astype(np.uint32))
    codes, scale = oracle.fp8_e4m3_quantize(X[src])
    got_scale = store.export("fp8_scale").cpu().numpy()
    np.testing.assert_array_equal(got_scale, scale)
    got_codes = store.export("fp8").cpu().view(torch.float8_e4m3fn).float().numpy()
    np.testing.assert_array_equal(got_codes.astype(np.float64), codes)
    np.testing.assert_array_equal(store.export("offsets").cpu().numpy(), w.docs.offsets)


def test_score_all_f32_matches_oracle(gem, cfg1):
    S = gem.score_all(cfg1["store"], cfg1["ws"], cfg1["q"], cfg1["qo"], "f32").cpu().numpy()
    err = np.abs(S.astype(np.float64) - cfg1["S64"])
    assert np.all(err <= 1e-5 * cfg1["L1"]), err.max()
    assert cfg1["ws"].status() == 0


def test_score_all_bf16_matches_oracle(gem, cfg1):
    w = cfg1["w"]
    S = gem.score_all(cfg1["store"], cfg1["ws"], cfg1["q"], cfg1["qo"], "bf16").cpu().numpy()
    assert cfg1["ws"].status() == 0
    err = np.abs(S.astype(np.float64) - cfg1["S64"])
    assert err.max() <= 2e-2, err.max()
    # against the FP64 score of the bf16-rounded inputs only FP32 accumulation remains
    Sq = oracle.score_all(oracle.bf16_round(w.queries.vecs.numpy()), w.queries.offsets,
                          oracle.bf16_round(w.docs.vecs.numpy()), w.docs.offsets)
    err2 = np.abs(S.astype(np.float64) - Sq)
    assert err2.max() <= 2e-4 * 32, err2.max()


def _fp8_dequantised(X):
    codes, scale = oracle.fp8_e4m3_quantize(np.asarray(X, np.float32))
    return codes * scale[:, None].astype(np.float64)


@pytest.mark.parametrize("lens", [[32] * 10, [1, 5, 17, 32, 33, 64, 100, 7]])
def test_score_all_fp8_matches_oracle_on_dequantised_inputs(gem, cfg1, lens):
    """E4M3 path: per-vector scales on both sides; against the FP64 score of the
    oracle's own E4M3 rounding of the same inputs only FP32 accumulation and the
    two scale multiplies remain."""
    w = cfg1["w"]
    lens = np.array(lens)
    qs = synth.vector_sets(lens, synth.centres(64, 1235), 777)
    S = gem.score_all(cfg1["store"], cfg1["ws"], qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda(),
                      "fp8").cpu().numpy()
    assert cfg1["ws"].status() == 0
    Sq = oracle.score_all(_fp8_dequantised(qs.vecs.numpy()), qs.offsets,
                          _fp8_dequantised(w.docs.vecs.numpy()), w.docs.offsets)
    err = np.abs(S - Sq)
    assert np.all(err <= 2e-4 * lens[:, None]), err.max()
    S64 = oracle.score_all(qs.vecs, qs.offsets, w.docs.vecs, w.docs.offsets)
    print("fp8 max |err| vs fp64 of fp32 inputs: %.3e" % np.abs(S - S64).max())


@pytest.mark.parametrize("lens", [
    [1, 2, 3, 5, 8, 13, 21, 32],          # every slot size, single pass
    [33, 64, 40, 7, 100, 128, 31, 65],    # multi-part queries (up to 4 passes)
    [32] * 19,                            # several query blocks
])
def test_score_all_bf16_query_length_mix(gem, cfg1, lens):
    w = cfg1["w"]
    lens = np.array(lens)
    qs = synth.vector_sets(lens, synth.centres(64, 1235), 4242)
    q = qs.vecs.cuda()
    qo = torch.from_numpy(qs.offsets).cuda()
    S = gem.score_all(cfg1["store"], cfg1["ws"], q, qo, "bf16").cpu().numpy()
    assert cfg1["ws"].status() == 0
    Sq = oracle.score_all(oracle.bf16_round(qs.vecs.numpy()), qs.offsets,
                          oracle.bf16_round(w.docs.vecs.numpy()), w.docs.offsets)
    tol = 2e-4 * lens[:, None]
    assert np.all(np.abs(S - Sq) <= tol), np.abs(S - Sq).max()


@pytest.mark.parametrize("compute", ["bf16", "fp8"])
def test_score_all_rows_beyond_unit_scale(gem, cfg1, compute):
    """Queries scaled by 0.5 .. 3: slots whose row maxima reach 2 in magnitude
    are summed in floating point, the others in fixed point; both agree with the
    oracle on the same rounded inputs."""
    w = cfg1["w"]
    lens = np.array([32, 32, 32, 32, 16, 32])
    qs = synth.vector_sets(lens, synth.centres(64, 1235), 9191)
    scale = np.repeat([1.0, 3.0, 0.5, 2.5, 3.0, 1.9], lens)[:, None].astype(np.float32)
    Xq = qs.vecs.numpy() * scale
    S = gem.score_all(cfg1["store"], cfg1["ws"], torch.from_numpy(Xq).cuda(),
                      torch.from_numpy(qs.offsets).cuda(), compute).cpu().numpy()
    assert cfg1["ws"].status() == 0
    rnd = oracle.bf16_round if compute == "bf16" else _fp8_dequantised
    Sq = oracle.score_all(rnd(Xq), qs.offsets, rnd(w.docs.vecs.numpy()), w.docs.offsets)
    tol = 2e-4 * (lens * np.array([1.0, 3.0, 0.5, 2.5, 3.0, 1.9]))[:, None]
    assert np.all(np.abs(S - Sq) <= tol), np.abs(S - Sq).max()


def test_score_ids_f32_matches_oracle(gem, cfg1):
    w = cfg1["w"]
    rng = np.random.default_rng(5)
    B = 10
    lens = rng.integers(0, 40, size=B)
    co = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    ids = rng.integers(-1, w.docs.n_sets, size=int(co[-1])).astype(np.int64)
    S = gem.score_ids(cfg1["store"], cfg1["ws"], cfg1["q"], cfg1["qo"], torch.from_numpy(co).cuda(),
                      torch.from_numpy(ids).cuda(), "f32").cpu().numpy()
    assert cfg1["ws"].status() == 0
    want = oracle.score_ids(w.queries.vecs, w.queries.offsets, w.docs.vecs, w.docs.offsets, co, ids)
    for t in range(len(ids)):
        if ids[t] < 0:
            assert S[t] == -np.inf
        else:
            b = int(np.searchsorted(co, t, side="right") - 1)
            assert abs(S[t] - want[t]) <= 1e-5 * cfg1["L1"][b, ids[t]]
            # bit-identical to the all-sets FP32 form (same arithmetic order)
    S_all = gem.score_all(cfg1["store"], cfg1["ws"], cfg1["q"], cfg1["qo"], "f32").cpu().numpy()
    for t in range(len(ids)):
        if ids[t] >= 0:
            b = int(np.searchsorted(co, t, side="right") - 1)
            assert S[t] == S_all[b, ids[t]]


def test_score_ids_streamed_rerank_bit_matches(gem, cfg1):
    """The exact id-list path streams the set vectors of a warp's whole range
    (gathered ahead across pairs, chunks and queries).  Query sets of 1 .. 128
    vectors take 1 to 4 groups of 32 rows per chunk of pairs; 60,000 pairs, so
    every warp crosses chunk and query boundaries; -1 ids and an empty list.
    Scores bit-identical to the all-sets FP32 form (the per-pair routine) and
    within 1e-5 of the L1 of the terms of the oracle."""
    w = cfg1["w"]
    rng = np.random.default_rng(11)
    q_lens = np.array([1, 5, 31, 32, 33, 64, 65, 100, 128, 7])
    qs = synth.vector_sets(q_lens, synth.centres(64, 1235), 991)
    q, qo = qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda()
    B = len(q_lens)
    lens = rng.integers(0, 12000, size=B)
    lens[3] = 0
    co = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    ids = rng.integers(-1, w.docs.n_sets, size=int(co[-1])).astype(np.int64)
    for mq in (128, 256):
        ws = gem.Workspace(cfg1["store"], max_queries=64, max_q_rows=4096, max_q_len=mq, max_cands=int(co[-1]))
        S = gem.score_ids(cfg1["store"], ws, q, qo, torch.from_numpy(co).cuda(), torch.from_numpy(ids).cuda(),
                          "f32").cpu().numpy()
        S_all = gem.score_all(cfg1["store"], ws, q, qo, "f32").cpu().numpy()
        assert ws.status() == 0
        ws.close()
        b_of = np.repeat(np.arange(B), lens)
        ok = ids >= 0
        np.testing.assert_array_equal(S[ok].view(np.uint32), S_all[b_of[ok], ids[ok]].view(np.uint32))
        assert np.all(S[~ok] == -np.inf)
    S64, L1 = oracle.score_all(qs.vecs, qs.offsets, w.docs.vecs, w.docs.offsets, with_l1=True)
    for t in rng.choice(np.nonzero(ids >= 0)[0], size=300, replace=False):
        assert abs(S[t] - S64[b_of[t], ids[t]]) <= 1e-5 * L1[b_of[t], ids[t]]


def test_rerank_pool_bit_matches_score_ids(gem, cfg1):
    """gem_rerank_pool on a pool of n_queries x depth ids: from 65,536 entries it
    scores the pool in the order of its set ids (ranges of ids, then query),
    below that in query order.  Pools of 64 x 1,200 (64 ranges) and 10 x 300
    with repeated ids and -1 entries: scores bit-identical to score_ids over the
    same rows as per-query lists, -1 entries -inf; an id past the store reads
    NaN with GEM_ERR_BOUNDS."""
    w, store = cfg1["w"], cfg1["store"]
    rng = np.random.default_rng(17)
    for nq, depth in ((64, 1200), (10, 300)):
        qs = synth.vector_sets(rng.integers(1, 129, size=nq), synth.centres(64, 1235), 993 + nq)
        q, qo = qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda()
        ws = gem.Workspace(store, max_queries=nq, max_q_rows=int(qs.offsets[-1]), max_q_len=128,
                           max_cands=nq * depth, max_k=256)
        # a shared pool: many queries name the same sets, as a top-R pool does
        pool = rng.integers(0, w.docs.n_sets, size=(nq, depth))
        shared = rng.integers(0, 40, size=(nq, depth))
        pool = np.where(rng.random((nq, depth)) < 0.5, shared, pool).astype(np.int64)
        pool[rng.random((nq, depth)) < 0.02] = -1
        pid = torch.from_numpy(pool).cuda()
        got = gem.rerank_pool(store, ws, q, qo, pid)
        assert ws.status() == 0
        co = torch.arange(0, nq * depth + 1, depth, dtype=torch.int64, device="cuda")
        ref = gem.score_ids(store, ws, q, qo, co, pid.view(-1), "f32").view(nq, depth)
        assert ws.status() == 0
        assert torch.equal(got.view(torch.int32), ref.view(torch.int32)), (nq, depth)
        assert torch.all(got[pid < 0] == -float("inf"))
        if nq == 10:
            pid[3, 7] = w.docs.n_sets
            got = gem.rerank_pool(store, ws, q, qo, pid)
            assert ws.status() == 7                # GEM_ERR_BOUNDS
            assert torch.isnan(got[3, 7]).item()
            keep = torch.ones_like(got, dtype=torch.bool)
            keep[3, 7] = False
            assert torch.equal(got[keep].view(torch.int32), ref[keep].view(torch.int32))
        ws.close()


def test_score_ids_query_longer_than_workspace_limit(gem, cfg1):
    """A query set longer than the workspace's max_q_len: its pairs score NaN and
    the status reads GEM_ERR_INVALID; the other queries' pairs are unaffected."""
    w = cfg1["w"]
    qs = synth.vector_sets(np.array([20, 40, 20]), synth.centres(64, 1235), 992)
    q, qo = qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda()
    co = torch.tensor([0, 3, 6, 9], dtype=torch.int64, device="cuda")
    ids = torch.tensor([0, 1, 2] * 3, dtype=torch.int64, device="cuda")
    ws = gem.Workspace(cfg1["store"], max_queries=8, max_q_rows=256, max_q_len=32, max_cands=64)
    S = gem.score_ids(cfg1["store"], ws, q, qo, co, ids, "f32").cpu().numpy()
    assert ws.status() == 1                # GEM_ERR_INVALID
    ws.close()
    assert np.all(np.isnan(S[3:6])) and np.all(np.isfinite(S[:3])) and np.all(np.isfinite(S[6:]))
    want = oracle.score_ids(qs.vecs, qs.offsets, w.docs.vecs, w.docs.offsets, co.cpu().numpy(), ids.cpu().numpy())
    assert np.all(np.abs(S[[0, 1, 2, 6, 7, 8]] - want[[0, 1, 2, 6, 7, 8]]) <= 1e-5 * 40)


def test_score_ids_out_of_range_id_sets_status(gem, cfg1):
    co = torch.tensor([0, 2] + [2] * 9, dtype=torch.int64, device="cuda")
    ids = torch.tensor([0, 10**6], dtype=torch.int64, device="cuda")
    S = gem.score_ids(cfg1["store"], cfg1["ws"], cfg1["q"], cfg1["qo"], co, ids, "f32")
    assert cfg1["ws"].status() == 7          # GEM_ERR_BOUNDS
    assert torch.isnan(S[1]).item() and torch.isfinite(S[0]).item()
    assert cfg1["ws"].status() == 0          # cleared after the read


def _check_topk(ids, sc, want_ids, want_sc):
    np.testing.assert_array_equal(ids, want_ids)
    np.testing.assert_array_equal(sc.astype(np.float64), want_sc)


@pytest.mark.parametrize("n,k", [(1, 1), (5, 10), (1000, 10), (4099, 1000), (70000, 2000), (300, 300)])
def test_topk_matches_oracle(gem, cfg1, n, k):
    rng = np.random.default_rng(n + k)
    s = np.round(rng.standard_normal((3, n)), 2).astype(np.float32)   # heavy ties
    ids, sc = gem.topk(cfg1["ws"], torch.from_numpy(s).cuda(), k)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    for r in range(3):
        wi, ws_ = oracle.topk(s[r], k)
        m = len(wi)
        _check_topk(ids[r, :m], sc[r, :m], wi, ws_)
        assert np.all(ids[r, m:] == -1) and np.all(sc[r, m:] == -np.inf)


def test_topk_signed_zeros_tie(gem, cfg1):
    """-0.0 and +0.0 are equal scores, so the lower id comes first."""
    s = np.array([[-0.0, 0.0, -0.0, 0.0, 1.0, -1.0]], np.float32)
    ids, _ = gem.topk(cfg1["ws"], torch.from_numpy(s).cuda(), 6)
    wi, _ = oracle.topk(s[0], 6)
    assert wi.tolist() == [4, 0, 1, 2, 3, 5]
    assert ids.cpu().numpy()[0].tolist() == wi.tolist()


def test_topk_explicit_ids_ragged_and_all_equal(gem, cfg1):
    rng = np.random.default_rng(3)
    lens = np.array([0, 7, 500, 3])
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    s = np.full(int(off[-1]), 0.5, np.float32)
    s[7:507] = np.round(rng.standard_normal(500), 1)
    ids = rng.permutation(100000)[: int(off[-1])].astype(np.int64)
    ids[2] = -1                                        # empty slot is skipped
    gi, gs = gem.topk(cfg1["ws"], torch.from_numpy(s).cuda(), 20, ids=torch.from_numpy(ids).cuda(),
                      row_offsets=torch.from_numpy(off).cuda())
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
    for r in range(4):
        seg = slice(off[r], off[r + 1])
        keep = ids[seg] >= 0
        wi, ws_ = oracle.topk(s[seg][keep], 20, ids[seg][keep])
        m = len(wi)
        _check_topk(gi[r, :m], gs[r, :m], wi, ws_)
        assert np.all(gi[r, m:] == -1)


@pytest.mark.parametrize("compute", ["bf16", "fp8", "f32"])
def test_search_pipeline_matches_exact_top10(gem, cfg1, compute):
    ids, sc = gem.search(cfg1["store"], cfg1["ws"], cfg1["q"], cfg1["qo"], compute, rerank_depth=200, k=10)
    assert cfg1["ws"].status() == 0
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    S64 = cfg1["S64"]
    for b in range(S64.shape[0]):
        wi, ws_ = oracle.topk(S64[b], 10)
        got = set(ids[b].tolist())
        for x in set(wi.tolist()) ^ got:
            # a swap is accepted only between ids whose exact scores tie within 1e-6
            assert abs(S64[b, x] - ws_[-1]) <= 1e-6 * max(1.0, abs(ws_[-1])), (b, x)
        err = np.abs(sc[b].astype(np.float64) - S64[b, ids[b]])
        assert np.all(err <= 1e-5 * cfg1["L1"][b, ids[b]])


def test_search_large_pool_grouped_by_set_bit_matches_query_order(gem, cfg1):
    """A rerank pool of 72 x 1,000 entries (past the size where the pool is
    taken grouped by set id) and queries of 1..64 vectors: the search's ids and
    scores equal the top-k of gem_score_ids over the same pool in query order,
    bit for bit, and the reranked scores stay within the FP32 bound of the
    oracle."""
    w = cfg1["w"]
    B, R, K = 72, 1000, 10
    lens = np.random.default_rng(23).integers(1, 65, size=B)
    qs = synth.vector_sets(lens, synth.centres(64, 1235), 4321)
    q, qo = qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda()
    ws = gem.Workspace(cfg1["store"], max_queries=B, max_q_rows=int(lens.sum()), max_q_len=64,
                       max_cands=B * R, max_k=R)
    pool, _ = gem.search(cfg1["store"], ws, q, qo, "bf16", rerank_depth=0, k=R)
    co = torch.arange(0, B * R + 1, R, dtype=torch.int64, device="cuda")
    ref = gem.score_ids(cfg1["store"], ws, q, qo, co, pool.reshape(-1).contiguous(), "f32")
    want_i, want_s = gem.topk(ws, ref.view(B, R), K, ids=pool.contiguous())
    got_i, got_s = gem.search(cfg1["store"], ws, q, qo, "bf16", rerank_depth=R, k=K)
    assert ws.status() == 0
    ws.close()
    assert torch.equal(got_i, want_i)
    assert torch.equal(got_s.view(torch.int32), want_s.view(torch.int32))
    S64, L1 = oracle.score_all(qs.vecs, qs.offsets, w.docs.vecs, w.docs.offsets, with_l1=True)
    gi, gs = got_i.cpu().numpy(), got_s.cpu().numpy().astype(np.float64)
    for b in range(B):
        assert np.all(np.abs(gs[b] - S64[b, gi[b]]) <= 1e-5 * L1[b, gi[b]])


def test_search_host_buffers(gem, cfg1):
    w = cfg1["w"]
    q = w.queries.vecs.pin_memory()
    qo = torch.from_numpy(w.queries.offsets)
    ids_h, sc_h = gem.search_host(cfg1["store"], cfg1["ws"], q, qo, "bf16", rerank_depth=100, k=10)
    ids_d, sc_d = gem.search(cfg1["store"], cfg1["ws"], cfg1["q"], cfg1["qo"], "bf16", rerank_depth=100, k=10)
    assert torch.equal(ids_h, ids_d.cpu()) and torch.equal(sc_h, sc_d.cpu())


def test_edge_cases_single_set_single_vector_and_long_set(gem):
    rng = np.random.default_rng(9)
    # one set of one vector; one long set spanning several chunks; short sets
    lens = np.array([1, 70000, 1, 3, 200])
    X = rng.standard_normal((int(lens.sum()), 128))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    X = X.astype(np.float32)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    store = gem.Store(torch.from_numpy(X).cuda(), off, keep=("f32", "bf16"))
    ws = gem.Workspace(store, max_queries=4, max_q_rows=256, max_q_len=64)
    qlens = np.array([1, 32, 64])
    Q = rng.standard_normal((int(qlens.sum()), 128))
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    Q = Q.astype(np.float32)
    qo = np.concatenate([[0], np.cumsum(qlens)]).astype(np.int64)
    S64, L1 = oracle.score_all(Q, qo, X, off, with_l1=True)
    Sf = gem.score_all(store, ws, torch.from_numpy(Q).cuda(), torch.from_numpy(qo).cuda(), "f32").cpu().numpy()
    assert np.all(np.abs(Sf - S64) <= 1e-5 * L1)
    Sb = gem.score_all(store, ws, torch.from_numpy(Q).cuda(), torch.from_numpy(qo).cuda(), "bf16").cpu().numpy()
    Sq = oracle.score_all(oracle.bf16_round(Q), qo, oracle.bf16_round(X), off)
    assert np.all(np.abs(Sb - Sq) <= 2e-4 * qlens[:, None])
    assert ws.status() == 0


def test_invalid_arguments_are_rejected_before_launch(gem, cfg1):
    with pytest.raises(gem.GemError) as e:
        gem.score_all(cfg1["store"], cfg1["ws"], cfg1["q"], cfg1["qo"], 7)
    assert e.value.code == 1
    with pytest.raises(gem.GemError):
        gem.search(cfg1["store"], cfg1["ws"], cfg1["q"], cfg1["qo"], "bf16", rerank_depth=5, k=10)
    # device-resident offsets that are not monotone are caught on the device
    bad = cfg1["qo"].clone()
    bad[3] = bad[2]
    out = torch.full((10, cfg1["store"].n_sets), 7.0, device="cuda")
    gem.score_all(cfg1["store"], cfg1["ws"], cfg1["q"], bad, "bf16", out=out)
    assert cfg1["ws"].status() == 1
    assert torch.all(out == 7.0)             # nothing was scored


def test_longest_query_sets_every_path(gem, cfg1):
    """Query sets of 200..256 vectors (up to 8 passes of the tensor-core plan,
    8 row groups of the streamed scorer) next to sets of 1 and 32 vectors: BF16
    all-sets within 2e-4 m_q of the FP64 score of the rounded inputs, FP32
    all-sets and id lists within 1e-5 of the L1 of the terms, the id-list scores
    bit-identical to the all-sets FP32 form."""
    w = cfg1["w"]
    lens = np.array([256, 1, 200, 32, 255, 129])
    qs = synth.vector_sets(lens, synth.centres(64, 1235), 6060)
    q, qo = qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda()
    B = len(lens)
    rng = np.random.default_rng(61)
    cl = rng.integers(50, 300, size=B)
    co = np.concatenate([[0], np.cumsum(cl)]).astype(np.int64)
    ids = rng.integers(0, w.docs.n_sets, size=int(co[-1])).astype(np.int64)
    ws = gem.Workspace(cfg1["store"], max_queries=B, max_q_rows=int(lens.sum()), max_q_len=256,
                       max_cands=int(co[-1]), max_k=16)
    Sb = gem.score_all(cfg1["store"], ws, q, qo, "bf16").cpu().numpy()
    Sf = gem.score_all(cfg1["store"], ws, q, qo, "f32").cpu().numpy()
    Si = gem.score_ids(cfg1["store"], ws, q, qo, torch.from_numpy(co).cuda(), torch.from_numpy(ids).cuda(),
                       "f32").cpu().numpy()
    assert ws.status() == 0
    ws.close()
    Sq = oracle.score_all(oracle.bf16_round(qs.vecs.numpy()), qs.offsets,
                          oracle.bf16_round(w.docs.vecs.numpy()), w.docs.offsets)
    assert np.all(np.abs(Sb - Sq) <= 2e-4 * lens[:, None]), np.abs(Sb - Sq).max()
    S64, L1 = oracle.score_all(qs.vecs, qs.offsets, w.docs.vecs, w.docs.offsets, with_l1=True)
    assert np.all(np.abs(Sf - S64) <= 1e-5 * L1)
    b_of = np.repeat(np.arange(B), cl)
    np.testing.assert_array_equal(Si.view(np.uint32), Sf[b_of, ids].view(np.uint32))
