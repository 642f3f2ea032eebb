"""Full-size parity of the text-corpus configuration, the bench's workload:
500,000 sets (lognormal lengths, 34.7M unit vectors of 128 components from a
4,096-centre mixture) and 1,000 queries of 32 vectors, in the bench's launch
configuration (default tensor-core schedule; the autotuner's other schedules are
bit-identical to it, `test_gpu_autotune.py`).

- Sampled (query, set) pairs of the BF16 first pass against the FP64 oracle:
  within 2e-4·m_q of the exact score of the bf16-rounded inputs (only FP32
  accumulation remains) and within 2e-2 of the exact score of the FP32 inputs.
  The same pairs through the FP32 id-list scorer are within 1e-5·L1.
- The whole search step (BF16 first pass, top-1,000, FP32 Kahan rerank, top-100)
  against the exact FP64 top-100 of every query stored in
  `tests/golden/text500k_truth.npz` (written by the oracle alone): recall@100 of
  at least 0.99 over all 1,000 queries, every id outside the exact top-100 tied
  with its 100th score within 1e-6, and the returned scores of sampled queries
  within 1e-5·L1 of FP64.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TRUTH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "text500k_truth.npz")


@pytest.fixture(scope="module")
def gem():
    import paper_2603_20336_b300 as g
    return g


@pytest.fixture(scope="module")
def text(gem):
    w = synth.text_corpus(device=torch.device("cuda", 0))
    store = gem.Store(w.docs.vecs, w.docs.offsets, keep=("f32", "bf16"))
    ws = gem.Workspace(store, max_queries=1000, max_q_rows=32_000, max_q_len=32, max_cands=1000 * 1000,
                       max_k=1000)
    q, qo = w.queries.vecs, torch.from_numpy(w.queries.offsets).cuda()
    yield w, store, ws, q, qo
    ws.close()
    store.close()


def _rows(w, b, s):
    off = w.docs.offsets
    Q = w.queries.vecs[32 * b: 32 * (b + 1)].cpu().numpy().astype(np.float64)
    P = w.docs.vecs[int(off[s]): int(off[s + 1])].cpu().numpy().astype(np.float64)
    return Q, P


def _l1(Q, P):
    return float(np.abs((Q @ P.T).max(axis=1)).sum())


def test_text500k_sampled_pairs_bf16_and_f32(gem, text):
    w, store, ws, q, qo = text
    S = gem.score_all(store, ws, q, qo, "bf16")
    assert ws.status() == 0
    rng = np.random.default_rng(31)
    qs = rng.integers(0, 1000, size=48)
    ss = rng.integers(0, store.n_sets, size=48)
    # and each sampled query's best set by the first pass: the pairs that decide the ranking
    best = torch.argmax(S[torch.from_numpy(qs).cuda()], dim=1).cpu().numpy()
    pairs = list(zip(qs.tolist(), ss.tolist())) + list(zip(qs.tolist(), best.tolist()))
    Sb = S.cpu().numpy()
    for b, s in pairs:
        Q, P = _rows(w, b, s)
        exact = oracle.chamfer(Q, P)
        on_bf16 = oracle.chamfer(oracle.bf16_round(Q), oracle.bf16_round(P))
        assert abs(Sb[b, s] - on_bf16) <= 2e-4 * 32, (b, s)
        assert abs(Sb[b, s] - exact) <= 2e-2, (b, s)
    # the same pairs in FP32 through the id-list scorer (each query with its own candidates)
    qb = np.array([b for b, _ in pairs])
    order = np.argsort(qb, kind="stable")
    ids = np.array([s for _, s in pairs])[order]
    counts = np.bincount(qb, minlength=1000)
    co = torch.from_numpy(np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)).cuda()
    F = gem.score_ids(store, ws, q, qo, co, torch.from_numpy(ids).cuda(), "f32").cpu().numpy()
    assert ws.status() == 0
    for (b, s), f in zip([pairs[i] for i in order], F):
        Q, P = _rows(w, b, s)
        assert abs(f - oracle.chamfer(Q, P)) <= 1e-5 * _l1(Q, P), (b, s)


def test_text500k_search_against_stored_exact_top100(gem, text):
    w, store, ws, q, qo = text
    d = np.load(TRUTH)
    assert str(d["fingerprint"]) == synth.fingerprint(w.docs, w.queries), "stored truth is of other data"
    t_ids, t_sc = d["ids"].astype(np.int64), d["scores"]
    ids, sc = gem.search(store, ws, q, qo, "bf16", rerank_depth=1000, k=100)
    assert ws.status() == 0
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy().astype(np.float64)
    recall = np.mean([len(set(ids[b].tolist()) & set(t_ids[b, :100].tolist())) / 100.0 for b in range(1000)])
    assert recall >= 0.99, recall
    for b in range(1000):
        extra = set(ids[b].tolist()) - set(t_ids[b, :100].tolist())
        for s in extra:          # only ties at the exact 100th place may differ
            Q, P = _rows(w, b, s)
            assert oracle.chamfer(Q, P) >= t_sc[b, 99] - 1e-6 * max(1.0, abs(t_sc[b, 99])), (b, s)
    for b in np.random.default_rng(4).choice(1000, size=6, replace=False):
        for s, f in zip(ids[b].tolist(), sc[b].tolist()):
            Q, P = _rows(w, b, s)
            assert abs(f - oracle.chamfer(Q, P)) <= 1e-5 * _l1(Q, P), (b, s)


def test_beam_batch_4096_queries_on_the_full_store(gem, text):
    """Config 4 at full size: 4,096 queries of 8..64 vectors, candidate lists of
    64..512 ids (30% from a 10,000-id pool) over the 500,000-set store, two
    graph-replayed rounds (the second with its ids mapped by the round shift):
    every score bit-identical to the non-batched id-list path over the same
    lists, and sampled pairs within 1e-5·L1 of FP64."""
    w, store = text[0], text[1]
    dev = torch.device("cuda", 0)
    nq = 4096
    qs = synth.vector_sets(synth.lengths_uniform(nq, 8, 64, 1238 + 7919), synth.centres(4096, 1236),
                           1238 + 7919, dev)
    co, ci0 = synth.candidate_lists(nq, store.n_sets, 64, 512, 0.3, 10_000, 1238)
    qv, qoff, co_d = qs.vecs, torch.from_numpy(qs.offsets).to(dev), torch.from_numpy(co).to(dev)
    bt = gem.Batch(store, "f32", max_queries=nq, max_q_rows=qv.shape[0], max_q_len=64, max_cands=len(ci0), seg=16)
    ws64 = gem.Workspace(store, max_queries=nq, max_q_rows=qv.shape[0], max_q_len=64)
    for rnd in range(2):
        ci = torch.from_numpy(synth.shift_lists(ci0, rnd, store.n_sets)).to(dev)
        got = bt.run(qv, qoff, co_d, ci).clone()
        assert bt.status() == 0
        ref = gem.score_ids(store, ws64, qv, qoff, co_d, ci, "f32")
        assert ws64.status() == 0
        assert torch.equal(got.view(torch.int32), ref.view(torch.int32)), rnd
    cih = ci.cpu().numpy()
    off = w.docs.offsets
    for t in np.random.default_rng(8).choice(len(cih), size=48, replace=False):
        b = int(np.searchsorted(co, t, side="right") - 1)
        Q = qv[int(qs.offsets[b]): int(qs.offsets[b + 1])].cpu().numpy().astype(np.float64)
        s = int(cih[t])
        P = w.docs.vecs[int(off[s]): int(off[s + 1])].cpu().numpy().astype(np.float64)
        assert abs(got[t].item() - oracle.chamfer(Q, P)) <= 1e-5 * _l1(Q, P), (b, s)
    ws64.close()
    bt.close()
