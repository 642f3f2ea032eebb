"""GPU parity of qEMD (Sec. 4.2.2, Eq. 14) against the oracle's exact linear
program on the GPU's own codes and the same FP32 centroids.

The optimal cost of a transportation problem is unique, so values are compared
(the plans may differ where optima tie).  Tolerance: the GPU's costs are FP32
dots of unit centroids (error <= 128 * 2^-24 < 1e-5 each, far less typically)
and its shortest paths compare FP32 sums, so |qemd - oracle| <= 2e-5.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
TOL = 2e-5


@pytest.fixture(scope="module")
def gem():
    import paper_2603_20336_b300 as g
    return g


@pytest.fixture(scope="module")
def cfg(gem):
    seed = 77
    cents = synth.centres(48, seed)
    lens = synth.lengths_uniform(400, 1, 128, seed)
    lens[:3] = [1, 128, 2]
    docs = synth.vector_sets(lens, cents, seed)
    store = gem.Store(docs.vecs.cuda(), docs.offsets, keep=("f32",))
    C = gem.train_codebook(store, k1=256, iters=4, sample=0, seed=3)
    gem.set_codebook(store, C)
    ws = gem.Workspace(store, max_queries=4, max_q_rows=512, max_q_len=128)
    yield dict(gem=gem, store=store, ws=ws, C=C.cpu().numpy(), codes=store.export("codes").cpu().numpy(),
               off=docs.offsets, lens=lens)
    ws.close()
    store.close()


def _run(gem, cfg, a, b):
    out = gem.qemd(cfg["store"], cfg["ws"], torch.tensor(a, dtype=torch.int64).cuda(),
                   torch.tensor(b, dtype=torch.int64).cuda())
    return out.cpu().numpy(), cfg["ws"].status()


def _want(cfg, a, b):
    off, codes = cfg["off"], cfg["codes"]
    return oracle.qemd(codes[off[a]:off[a + 1]], codes[off[b]:off[b + 1]], cfg["C"].astype(np.float64))


def test_qemd_matches_oracle_lp(gem, cfg):
    rng = np.random.default_rng(5)
    a = rng.integers(0, 400, 60).tolist() + [0, 1, 1, 2, 0, 7]
    b = rng.integers(0, 400, 60).tolist() + [1, 0, 1, 2, 2, 7]   # sizes 1 / 128, a set with itself
    got, st = _run(gem, cfg, a, b)
    assert st == 0
    for p in range(len(a)):
        assert abs(got[p] - _want(cfg, a[p], b[p])) <= TOL, (p, a[p], b[p])
    # a set against itself transports every code onto itself
    assert abs(got[-4]) <= TOL and abs(got[-1]) <= TOL


def test_qemd_symmetric_and_bounds_the_averaged_qch(gem, cfg):
    """qEMD(A, B) = qEMD(B, A), and Eq. 10 with quantized distances: the averaged
    qCH distance (1/m_A) sum_i min_j d_X(NN(a_i), NN(b_j)) never exceeds qEMD."""
    rng = np.random.default_rng(6)
    a, b = rng.integers(0, 400, 200), rng.integers(0, 400, 200)
    g1, s1 = _run(gem, cfg, a.tolist(), b.tolist())
    g2, s2 = _run(gem, cfg, b.tolist(), a.tolist())
    assert s1 == 0 and s2 == 0
    np.testing.assert_allclose(g1, g2, atol=TOL)
    off, codes, C = cfg["off"], cfg["codes"], cfg["C"].astype(np.float64)
    for p in range(len(a)):
        ca, cb = codes[off[a[p]]:off[a[p] + 1]], codes[off[b[p]]:off[b[p] + 1]]
        avg = oracle.qch_distance(ca, cb, C) / len(ca)
        assert avg <= g1[p] + TOL


def test_qemd_rejects_long_sets_and_bad_ids_on_the_device(gem):
    w = synth.exact_fp32(n_sets=40, n_queries=1)
    lens = np.diff(w.docs.offsets)
    long_vecs = synth.vector_sets(np.array([129]), synth.centres(8, 1), 2)
    vecs = torch.cat([w.docs.vecs, long_vecs.vecs])
    off = np.concatenate([w.docs.offsets, [w.docs.offsets[-1] + 129]]).astype(np.int64)
    store = gem.Store(vecs.cuda(), off, keep=("f32",))
    gem.set_codebook(store, gem.train_codebook(store, k1=64, iters=2, sample=0, seed=1))
    ws = gem.Workspace(store, max_queries=1, max_q_rows=64, max_q_len=64)
    n = len(lens)
    out = gem.qemd(store, ws, torch.tensor([0, n], dtype=torch.int64).cuda(),
                   torch.tensor([1, 0], dtype=torch.int64).cuda()).cpu().numpy()
    assert ws.status() == 1                    # GEM_ERR_INVALID: a set of 129 vectors
    assert np.isfinite(out[0]) and np.isnan(out[1])
    out = gem.qemd(store, ws, torch.tensor([0], dtype=torch.int64).cuda(),
                   torch.tensor([n + 5], dtype=torch.int64).cuda()).cpu().numpy()
    assert ws.status() == 7 and np.isnan(out[0])   # GEM_ERR_BOUNDS
    ws.close()
    store.close()
