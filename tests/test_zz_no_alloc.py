"""gem_score_ids_noalloc, the id-list scorer for callers that cannot allocate
device memory (their device memory belongs to another allocator, so they cannot
create a workspace or a batch).  Its scratch is a fixed device array shared by
every call, so two calls in a row must each give what the allocating entry point
gem_score_ids gives.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_score_ids_on_two_calls():
    import paper_2603_20336_b300 as gem
    w = synth.exact_fp32(n_sets=500, n_queries=1)
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("f32",))
    ws = gem.Workspace(store, max_queries=64, max_q_rows=64 * 64, max_q_len=64)
    X = w.docs.vecs.numpy().astype(np.float64)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (n_q, lo, hi) in enumerate([(40, 8, 64), (7, 1, 33)]):
        rng = np.random.default_rng(100 + call)
        qs = synth.vector_sets(rng.integers(lo, hi + 1, size=n_q), synth.centres(64, 1235), 50 + call)
        lens = rng.integers(0, 70, size=n_q)
        co = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        ids = rng.integers(0, w.docs.n_sets, size=int(co[-1])).astype(np.int64)
        q, qo = qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda()
        co_d, ids_d = torch.from_numpy(co).cuda(), torch.from_numpy(ids).cuda()
        want = gem.score_ids(store, ws, q, qo, co_d, ids_d, "f32")
        out = torch.full_like(want, float("nan"))
        rc = gem.lib.gem_score_ids_noalloc(store.handle, _ptr(q), _ptr(qo), n_q, q.shape[0], 64, _ptr(co_d),
                                           _ptr(ids_d), ids_d.numel(), _ptr(out), stream)
        assert rc == 0, gem.lib.gem_last_error_message()
        torch.cuda.synchronize()
        # the tolerance of the FP32 id-list tests (1e-5 of the L1 of the terms) ...
        Q = qs.vecs.numpy().astype(np.float64)
        for t in range(len(ids)):
            b = int(np.searchsorted(co, t, side="right") - 1)
            P = X[w.docs.offsets[ids[t]]:w.docs.offsets[ids[t] + 1]]
            l1 = np.abs((Q[qs.offsets[b]:qs.offsets[b + 1]] @ P.T).max(axis=1)).sum()
            assert abs(out[t].item() - want[t].item()) <= 1e-5 * l1
        # ... and, since both run the same per-pair arithmetic, identical bits
        assert torch.equal(out, want)
    # more queries than the fixed scratch holds is refused up front
    big = torch.zeros(16386, dtype=torch.int64, device="cuda")
    rc = gem.lib.gem_score_ids_noalloc(store.handle, _ptr(q), _ptr(big), 16385, 16385, 64, _ptr(big), _ptr(big), 1,
                                       _ptr(out), stream)
    assert rc == 1 and b"16384" in gem.lib.gem_last_error_message()
