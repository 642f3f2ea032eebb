"""Batched candidate scoring (one persistent, graph-replayed launch per
expansion round): bit-identical FP32 scores to the per-query gem_score_ids path,
parity with the FP64 oracle, several rounds, and the codes form."""
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
def beam(gem):
    seed = 1238
    cents = synth.centres(256, seed)
    docs = synth.vector_sets(synth.lengths_lognormal(3000, 70.0, 0.5, 20, 180, seed), cents, seed)
    store = gem.Store(docs.vecs.cuda(), docs.offsets, keep=("f32", "bf16"))
    C = gem.train_codebook(store, k1=512, iters=4, sample=0, seed=3)
    gem.set_codebook(store, C)
    ws = gem.Workspace(store, max_queries=256, max_q_rows=256 * 64, max_q_len=64, max_cands=256 * 64)
    return dict(docs=docs, cents=cents, store=store, ws=ws, C=C)


def _round(beam, rnd, n_queries=200):
    qs, co, ci = synth.beam_batch(beam["docs"], beam["cents"], seed=1238, n_queries=n_queries, len_lo=16,
                                  len_hi=64, shared_frac=0.3, pool_size=100, rnd=rnd)
    return qs, co, ci


def _per_query(gem, beam, qs, co, ci, compute):
    out = []
    for b in range(len(co) - 1):
        qv = qs.vecs[qs.offsets[b]:qs.offsets[b + 1]].cuda()
        qo = torch.tensor([0, qs.offsets[b + 1] - qs.offsets[b]], dtype=torch.int64, device="cuda")
        c = torch.tensor([0, co[b + 1] - co[b]], dtype=torch.int64, device="cuda")
        ids = torch.from_numpy(ci[co[b]:co[b + 1]]).cuda()
        out.append(gem.score_ids(beam["store"], beam["ws"], qv, qo, c, ids, compute))
    return torch.cat(out)


def test_batched_f32_bit_matches_per_query_path_over_rounds(gem, beam):
    bt = gem.Batch(beam["store"], "f32", max_queries=256, max_q_rows=256 * 64, max_q_len=64,
                   max_cands=256 * 64, seg=16)
    docs = beam["docs"]
    for rnd in range(3):
        qs, co, ci = _round(beam, rnd)
        args = (qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda(), torch.from_numpy(co).cuda(),
                torch.from_numpy(ci).cuda())
        s_graph = bt.run(*args).clone()
        s_direct = bt.run(*args, use_graph=False).clone()
        assert bt.status() == 0
        s_ref = _per_query(gem, beam, qs, co, ci, "f32")
        assert torch.equal(s_graph, s_direct)
        assert torch.equal(s_graph, s_ref)
        if rnd == 0:
            want = oracle.score_ids(qs.vecs, qs.offsets, docs.vecs, docs.offsets, co, ci)
            Q = qs.vecs.numpy().astype(np.float64)
            for t in range(0, len(ci), 7):
                b = int(np.searchsorted(co, t, side="right") - 1)
                P = docs.vecs[docs.offsets[ci[t]]:docs.offsets[ci[t] + 1]].numpy().astype(np.float64)
                l1 = np.abs((Q[qs.offsets[b]:qs.offsets[b + 1]] @ P.T).max(axis=1)).sum()
                assert abs(s_graph[t].item() - want[t]) <= 1e-5 * l1
    bt.close()


def test_batched_codes_bit_matches_and_equals_oracle_estimate(gem, beam):
    """The codes form assigns each round's query rows on the tensor cores with
    the row count read on the device (16,384 rows of room here); the per-query
    path assigns the same rows with the SIMT kernel.  Rounds of 1, 50 and 200
    queries (ragged last 128-row unit) in the graph and directly: bit-identical
    to it, and the 50-query round within 1e-5·m_q of the oracle's qCH."""
    bt = gem.Batch(beam["store"], "codes", max_queries=256, max_q_rows=256 * 64, max_q_len=64,
                   max_cands=256 * 64, seg=32)
    for rnd, nq in ((8, 200), (9, 1)):
        qs, co, ci = _round(beam, rnd, n_queries=nq)
        args = (qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda(), torch.from_numpy(co).cuda(),
                torch.from_numpy(ci).cuda())
        s_graph = bt.run(*args).clone()
        s_direct = bt.run(*args, use_graph=False).clone()
        assert bt.status() == 0
        assert torch.equal(s_graph, s_direct), nq
        assert torch.equal(s_graph, _per_query(gem, beam, qs, co, ci, "codes")), nq
    qs, co, ci = _round(beam, 7, n_queries=50)
    q, qo = qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda()
    s = bt.run(q, qo, torch.from_numpy(co).cuda(), torch.from_numpy(ci).cuda()).clone()
    assert bt.status() == 0
    assert torch.equal(s, _per_query(gem, beam, qs, co, ci, "codes"))
    Cn = beam["C"].cpu().numpy()
    pcodes = beam["store"].export("codes").cpu().numpy()
    qcodes = gem.assign_codes(q, beam["C"]).cpu().numpy()
    want = oracle.qch_score_ids(qcodes, qs.offsets, pcodes, beam["docs"].offsets, co, ci, Cn)
    m_q = np.diff(qs.offsets)
    for t in range(len(ci)):
        b = int(np.searchsorted(co, t, side="right") - 1)
        assert abs(s[t].item() - want[t]) <= 1e-5 * m_q[b]
    bt.close()


def test_batched_rejects_inconsistent_offsets(gem, beam):
    bt = gem.Batch(beam["store"], "f32", max_queries=8, max_q_rows=512, max_q_len=64, max_cands=64, seg=8)
    q = torch.randn(64, 128, device="cuda")
    qo = torch.tensor([0, 32, 64], dtype=torch.int64, device="cuda")
    co = torch.tensor([0, 5, 3], dtype=torch.int64, device="cuda")      # last offset != n_cands
    ids = torch.zeros(4, dtype=torch.int64, device="cuda")
    bt.run(q, qo, co, ids)
    assert bt.status() == 1
    co = torch.tensor([0, 2, 4], dtype=torch.int64, device="cuda")
    ids = torch.tensor([0, 1, 2, 10**7], dtype=torch.int64, device="cuda")
    s = bt.run(q, qo, co, ids)
    assert bt.status() == 7 and torch.isnan(s[3]).item()
    bt.close()


def test_batched_short_groups_bit_match_on_boundary_lengths(gem):
    """The batch scorer splits a row group of at most 16 query rows over both
    half-warps (alternate 8-vector blocks).  Query lengths on every side of the
    16 / 32 / 48 boundaries and sets of 1..20 vectors (one block, an odd or an
    even number of blocks) score bit-identically to the id-list path, which
    keeps whole 32-row groups, and within 1e-5·L1 of FP64."""
    seed = 77
    cents = synth.centres(64, seed)
    lens = np.random.default_rng(seed).integers(1, 21, size=400)
    docs = synth.vector_sets(lens.astype(np.int64), cents, seed)
    store = gem.Store(docs.vecs.cuda(), docs.offsets, keep=("f32",))
    qlens = np.array([1, 2, 8, 15, 16, 17, 31, 32, 33, 40, 47, 48, 49, 63, 64], dtype=np.int64)
    qs = synth.vector_sets(qlens, cents, seed + 1)
    rng = np.random.default_rng(seed + 2)
    counts = rng.integers(1, 40, size=len(qlens))
    co = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    ci = rng.integers(0, 400, size=int(co[-1])).astype(np.int64)
    bt = gem.Batch(store, "f32", max_queries=len(qlens), max_q_rows=int(qlens.sum()), max_q_len=64,
                   max_cands=len(ci), seg=8)
    args = (qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda(), torch.from_numpy(co).cuda(),
            torch.from_numpy(ci).cuda())
    got = bt.run(*args).clone()
    assert bt.status() == 0
    ws = gem.Workspace(store, max_queries=len(qlens), max_q_rows=int(qlens.sum()), max_q_len=64)
    ref = gem.score_ids(store, ws, *args, "f32")
    assert torch.equal(got.view(torch.int32), ref.view(torch.int32))
    want = oracle.score_ids(qs.vecs, qs.offsets, docs.vecs, docs.offsets, co, ci)
    Q = qs.vecs.numpy().astype(np.float64)
    for t in range(len(ci)):
        b = int(np.searchsorted(co, t, side="right") - 1)
        P = docs.vecs[docs.offsets[ci[t]]:docs.offsets[ci[t] + 1]].numpy().astype(np.float64)
        l1 = np.abs((Q[qs.offsets[b]:qs.offsets[b + 1]] @ P.T).max(axis=1)).sum()
        assert abs(got[t].item() - want[t]) <= 1e-5 * l1
    ws.close()
    bt.close()
    store.close()


def test_batched_codes_below_tensor_core_size_uses_simt_assignment(gem, beam):
    """A codes-form batch with less than 16,384 query rows of room assigns its
    query codes with the SIMT kernel (row count read on the device): scores
    bit-identical to the per-query path over two rounds of different sizes."""
    bt = gem.Batch(beam["store"], "codes", max_queries=200, max_q_rows=200 * 64 - 1, max_q_len=64,
                   max_cands=200 * 64, seg=16)
    for rnd, nq in ((11, 150), (12, 7)):
        qs, co, ci = _round(beam, rnd, n_queries=nq)
        assert int(qs.offsets[-1]) < 200 * 64 - 1
        args = (qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda(), torch.from_numpy(co).cuda(),
                torch.from_numpy(ci).cuda())
        s_graph = bt.run(*args).clone()
        assert bt.status() == 0
        assert torch.equal(s_graph, _per_query(gem, beam, qs, co, ci, "codes")), nq
    bt.close()
