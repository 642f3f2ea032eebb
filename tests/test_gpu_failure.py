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


def test_a_failed_allocation_is_reported_and_the_context_stays_usable(gem):
    """An allocation the device cannot satisfy (a workspace sized for 2^45
    candidates, 256 TB of ids) fails with GEM_ERR_OOM through the ordinary
    cudaMalloc path, frees what it had allocated, and the next calls work."""
    w = synth.exact_fp32(n_sets=60, n_queries=1)
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("f32",))
    with pytest.raises(gem.GemError) as e:
        gem.Workspace(store, max_queries=1, max_q_rows=32, max_q_len=32, max_cands=1 << 45)
    assert e.value.code == 2                     # GEM_ERR_OOM
    ws = gem.Workspace(store, max_queries=1, max_q_rows=32, max_q_len=32, max_cands=60)
    q, qo = w.queries.vecs.cuda(), torch.from_numpy(w.queries.offsets).cuda()
    s = gem.score_all(store, ws, q, qo, "f32").cpu().numpy()
    assert ws.status() == 0
    S64 = oracle.score_all(w.queries.vecs, w.queries.offsets, w.docs.vecs, w.docs.offsets)
    assert np.abs(s - S64).max() <= 1e-4
    ws.close()
    store.close()


def test_injected_allocation_failures_unwind_cleanly(gem, monkeypatch):
    """Failure injection on the host: GEM_FAULT_INJECT=alloc:N makes the N-th
    device allocation of a creation call fail as if the device were out of
    memory.  Every prefix of the store's and the workspace's allocations is
    unwound with GEM_ERR_OOM and nothing half-built escapes; with the variable
    cleared, the same creation calls succeed and score correctly."""
    w = synth.exact_fp32(n_sets=120, n_queries=2)
    vecs, off = w.docs.vecs.cuda(), w.docs.offsets
    keep = ("f32", "bf16", "fp8", "fp8_set")

    def count_failures(make):
        fails = 0
        for n in range(1, 64):
            monkeypatch.setenv("GEM_FAULT_INJECT", f"alloc:{n}")
            try:
                obj = make()
            except gem.GemError as e:
                assert e.code == 2, e              # GEM_ERR_OOM
                fails += 1
                continue
            obj.close()                            # n is past the call's last allocation
            return fails
        raise AssertionError("an allocation failure at every position up to 63")

    assert count_failures(lambda: gem.Store(vecs, off, keep=keep)) >= 6
    monkeypatch.delenv("GEM_FAULT_INJECT")
    store = gem.Store(vecs, off, keep=keep)
    assert count_failures(lambda: gem.Workspace(store, max_queries=2, max_q_rows=64, max_q_len=32,
                                                max_cands=64, max_k=16)) >= 6
    monkeypatch.delenv("GEM_FAULT_INJECT")
    ws = gem.Workspace(store, max_queries=2, max_q_rows=64, max_q_len=32, max_cands=64, max_k=16)
    q, qo = w.queries.vecs.cuda(), torch.from_numpy(w.queries.offsets).cuda()
    s = gem.score_all(store, ws, q, qo, "f32").cpu().numpy().astype(np.float64)
    S64, L1 = oracle.score_all(w.queries.vecs, w.queries.offsets, w.docs.vecs, w.docs.offsets, with_l1=True)
    assert np.all(np.abs(s - S64) <= 1e-5 * L1)
    assert ws.status() == 0
    ws.close()
    store.close()
