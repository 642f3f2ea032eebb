"""Failure detection on the GPU without a fault: a bounded wait that runs out
(on an mbarrier nothing arrives on) records GEM_ERR_TIMEOUT in the workspace's
status word, the kernel returns, and the context stays usable for the next
scoring call."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

GEM_ERR_TIMEOUT = 4


@pytest.fixture(scope="module")
def gem():
    import paper_2603_20336_b300 as g
    return g


def test_a_wait_that_runs_out_reports_timeout_and_the_context_stays_usable(gem):
    w = synth.exact_fp32(n_sets=80, n_queries=2)
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("f32", "bf16"))
    ws = gem.Workspace(store, max_queries=2, max_q_rows=64, max_q_len=32)
    gem.selftest_wait_timeout(ws, 1 << 20)
    assert ws.status() == GEM_ERR_TIMEOUT
    assert ws.status() == 0                      # read clears the word
    q, qo = w.queries.vecs.cuda(), torch.from_numpy(w.queries.offsets).cuda()
    s = gem.score_all(store, ws, q, qo, "bf16").cpu().numpy()
    assert ws.status() == 0
    S64 = oracle.score_all(w.queries.vecs, w.queries.offsets, w.docs.vecs, w.docs.offsets)
    assert np.abs(s - S64).max() <= 2e-2
    with pytest.raises(Exception):
        gem.selftest_wait_timeout(ws, 0)
    ws.close()
    store.close()
