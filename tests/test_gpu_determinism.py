"""Run-to-run bit identity: every scoring path, given the same inputs twice,
returns the same bits.  With the sanitizers closed on this pool this is the race
check: a missing barrier or a data race between warps shows up as scores that
change from one run to the next.  (The backward's atomic path for sets named by
several pairs is the one place where the order of additions, and so the last
bits, may legitimately vary; here every pair names its own set.)"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gem():
    import paper_2603_20336_b300 as g
    return g


def _same(a, b):
    a, b = a.contiguous(), b.contiguous()
    if a.dtype == torch.float32:
        return torch.equal(a.view(torch.int32), b.view(torch.int32))
    return torch.equal(a, b)


def test_every_scoring_path_is_bit_reproducible(gem):
    w = synth.exact_fp32(n_sets=2000, n_queries=10)
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("f32", "bf16", "fp8", "fp8_set"))
    C = gem.train_codebook(store, k1=256, iters=3, sample=0, seed=3)
    gem.set_codebook(store, C)
    ws = gem.Workspace(store, max_queries=10, max_q_rows=320, max_q_len=32, max_cands=10 * 300, max_k=300)
    q, qo = w.queries.vecs.cuda(), torch.from_numpy(w.queries.offsets).cuda()

    def twice(fn):
        a = fn()
        a = tuple(x.clone() for x in a) if isinstance(a, tuple) else a.clone()
        b = fn()
        return a, b

    for compute in ("bf16", "fp8", "fp8_set", "f32"):
        a, b = twice(lambda: gem.score_all(store, ws, q, qo, compute))
        assert _same(a, b), compute
    rng = np.random.default_rng(5)
    co = torch.arange(0, 10 * 150 + 1, 150, dtype=torch.int64, device="cuda")
    ids = torch.from_numpy(rng.integers(0, 2000, size=10 * 150)).cuda()
    for compute in ("f32", "codes"):
        a, b = twice(lambda: gem.score_ids(store, ws, q, qo, co, ids, compute))
        assert _same(a, b), compute
    a, b = twice(lambda: gem.estimate_codes(store, ws, q, qo))
    assert _same(a, b)
    S = gem.score_all(store, ws, q, qo, "bf16")
    (ia, sa), (ib, sb) = twice(lambda: gem.topk(ws, S, 100))
    assert _same(ia, ib) and _same(sa, sb)
    for compute in ("bf16", "fp8_set", "codes"):
        (ia, sa), (ib, sb) = twice(lambda: gem.search(store, ws, q, qo, compute, rerank_depth=300, k=10))
        assert _same(ia, ib) and _same(sa, sb), compute
    assert ws.status() == 0

    # the backward with every pair naming its own set: dQ (a warp per row) and dP
    # (each row written once by its set's one pair) are both free of atomics
    po = torch.arange(0, 10 * 20 + 1, 20, dtype=torch.int64, device="cuda")
    pid = torch.randperm(2000, device="cuda")[:200].contiguous()
    docs, do = w.docs.vecs.cuda(), torch.from_numpy(w.docs.offsets).cuda()
    (s1, am1), (s2, am2) = twice(lambda: gem.maxsim_fwd(q, qo, docs, do, po, pid, max_q_len=32))
    assert _same(s1, s2) and _same(am1, am2)
    g = torch.linspace(-1.0, 1.0, 200, device="cuda")
    (dq1, dp1), (dq2, dp2) = twice(lambda: gem.maxsim_bwd(q, qo, docs, do, po, pid, am1, g))
    assert _same(dq1, dq2) and _same(dp1, dp2)
    ws.close()
    store.close()
