"""GPU parity of nearest-centroid codes, the stage-1 k-means and the qCH
estimate against the FP64 oracle.

Codes are integers decided by floating point: the GPU decides in FP32 (one FMA
chain per dot product), the oracle in FP64.  A code must equal the oracle's
wherever the oracle's top-2 margin exceeds 2 * EPS (EPS bounds the FP32 error of
a 128-term dot product of unit vectors, 128 * 2^-24 < 1e-5); inside that band the
GPU's choice must be within 2 * EPS of the best FP64 inner product.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
EPS = 1e-5


@pytest.fixture(scope="module")
def gem():
    import paper_2603_20336_b300 as g
    return g


def _unit(rng, n, d=128):
    x = rng.standard_normal((n, d))
    return (x / np.linalg.norm(x, axis=1, keepdims=True)).astype(np.float32)


def _check_codes(X, C, codes):
    sims = X.astype(np.float64) @ C.astype(np.float64).T
    want = np.argmax(sims, axis=1)
    if sims.shape[1] > 1:
        top2 = np.sort(sims, axis=1)[:, -2:]
        margin = top2[:, 1] - top2[:, 0]
    else:
        margin = np.full(len(X), np.inf)
    clear = margin > 2 * EPS
    np.testing.assert_array_equal(codes[clear], want[clear])
    got_sim = sims[np.arange(len(X)), codes]
    assert np.all(got_sim >= sims.max(axis=1) - 2 * EPS)
    return int((~clear).sum())


@pytest.mark.parametrize("n,k1", [(1, 1), (100, 7), (5000, 1024), (777, 4099)])
def test_assign_codes_match_oracle(gem, n, k1):
    rng = np.random.default_rng(n + k1)
    cents = synth.centres(64, 5)
    X = synth.draw_vectors(n, cents, 11).numpy()
    C = _unit(rng, k1)
    codes, best = gem.assign_codes(torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda(), with_best=True)
    codes = codes.cpu().numpy().astype(np.int64)
    _check_codes(X, C, codes)
    sims = X.astype(np.float64) @ C.astype(np.float64).T
    np.testing.assert_allclose(best.cpu().numpy(), sims[np.arange(n), codes], atol=EPS)


def test_assign_codes_centroid_maps_to_itself_and_ties_go_low(gem):
    rng = np.random.default_rng(3)
    C = _unit(rng, 300)
    codes = gem.assign_codes(torch.from_numpy(C).cuda(), torch.from_numpy(C).cuda()).cpu().numpy()
    np.testing.assert_array_equal(codes, np.arange(300))
    Cdup = np.vstack([C[:10], C[4:5], C[10:]])          # row 10 repeats row 4
    codes = gem.assign_codes(torch.from_numpy(C[4:5]).cuda(), torch.from_numpy(Cdup).cuda()).cpu().numpy()
    assert codes.tolist() == [4]


def test_train_codebook_fixed_point_invariants(gem):
    """k-means is a heuristic (parity unpinned); its fixed point is checked:
    unit centroids, each the normalised mean of the vectors coded to it."""
    w = synth.exact_fp32(n_sets=120, n_queries=1)
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("f32",))
    C = gem.train_codebook(store, k1=32, iters=40, sample=0, seed=7)
    X = w.docs.vecs.numpy()
    codes = gem.assign_codes(w.docs.vecs.cuda(), C).cpu().numpy()
    Cn = C.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(Cn, axis=1), 1.0, atol=1e-5)
    for c in range(32):
        mem = X[codes == c].astype(np.float64)
        if len(mem):
            m = mem.sum(0)
            np.testing.assert_allclose(Cn[c], m / np.linalg.norm(m), atol=2e-4)
    # a second training with the same seed is identical up to summation order
    C2 = gem.train_codebook(store, k1=32, iters=40, sample=0, seed=7)
    assert torch.allclose(C, C2, atol=1e-5)


def test_qch_lossless_codes_equal_exact_chamfer(gem):
    """With C_quant holding every stored and query vector exactly, NN is the
    identity and the estimate equals exact CH (the lossless invariant)."""
    w = synth.exact_fp32(n_sets=60, n_queries=4)
    X, Q = w.docs.vecs.numpy(), w.queries.vecs.numpy()
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("f32", "bf16"))
    C = np.vstack([X, Q])
    gem.set_codebook(store, torch.from_numpy(C).cuda())
    codes = store.export("codes").cpu().numpy()
    np.testing.assert_array_equal(codes, np.arange(len(X)))
    ws = gem.Workspace(store, max_queries=4, max_q_rows=128, max_q_len=32)
    est = gem.estimate_codes(store, ws, w.queries.vecs.cuda(), torch.from_numpy(w.queries.offsets).cuda())
    assert ws.status() == 0
    S64, L1 = oracle.score_all(Q, w.queries.offsets, X, w.docs.offsets, with_l1=True)
    assert np.all(np.abs(est.cpu().numpy() - S64) <= 1e-5 * L1 + 1e-6)


@pytest.mark.parametrize("qlens", [[32] * 5, [1, 7, 33, 64, 100, 20]])
def test_qch_matches_oracle_given_gpu_codes(gem, qlens):
    w = synth.exact_fp32(n_sets=300, n_queries=1)
    qs = synth.vector_sets(np.array(qlens), synth.centres(64, 1235), 99)
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("f32",))
    C = gem.train_codebook(store, k1=256, iters=5, sample=0, seed=1)
    gem.set_codebook(store, C)
    ws = gem.Workspace(store, max_queries=8, max_q_rows=512, max_q_len=128, max_cands=1000)
    q, qo = qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda()
    est = gem.estimate_codes(store, ws, q, qo).cpu().numpy()
    assert ws.status() == 0
    Cn = C.cpu().numpy()
    pcodes = store.export("codes").cpu().numpy()
    qcodes = gem.assign_codes(q, C).cpu().numpy()
    _check_codes(w.docs.vecs.numpy(), Cn, pcodes.astype(np.int64))
    _check_codes(qs.vecs.numpy(), Cn, qcodes.astype(np.int64))
    want = oracle.qch_score_all(qcodes, qs.offsets, pcodes, w.docs.offsets, Cn)
    lens = np.array(qlens)[:, None]
    assert np.all(np.abs(est - want) <= 1e-5 * lens), np.abs(est - want).max()
    # qsim = m_q - qCH (the distance form of Eq. 16)
    b, n = 1, 17
    d = oracle.qch_distance(qcodes[qs.offsets[b]:qs.offsets[b + 1]],
                            pcodes[w.docs.offsets[n]:w.docs.offsets[n + 1]], Cn)
    assert abs((qlens[b] - d) - est[b, n]) <= 1e-5 * qlens[b]
    # id-list form: same arithmetic, bit-identical to the all-sets form
    rng = np.random.default_rng(2)
    lens = rng.integers(0, 30, size=len(qlens))
    co = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    ids = rng.integers(0, 300, size=int(co[-1])).astype(np.int64)
    est_ids = gem.estimate_codes(store, ws, q, qo, torch.from_numpy(co).cuda(),
                                 torch.from_numpy(ids).cuda()).cpu().numpy()
    for t in range(len(ids)):
        b = int(np.searchsorted(co, t, side="right") - 1)
        assert est_ids[t] == est[b, ids[t]]


def test_asymmetric_qch_lossless_on_the_stored_side(gem):
    """Asymmetric form: with C_quant holding every stored vector (and none of the
    query vectors), the estimate is exact CH; the symmetric form is not."""
    w = synth.exact_fp32(n_sets=60, n_queries=4)
    X, Q = w.docs.vecs.numpy(), w.queries.vecs.numpy()
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("f32",))
    gem.set_codebook(store, torch.from_numpy(X.copy()).cuda())
    ws = gem.Workspace(store, max_queries=4, max_q_rows=128, max_q_len=32)
    gem.set_qch_form(ws, "asymmetric")
    q, qo = w.queries.vecs.cuda(), torch.from_numpy(w.queries.offsets).cuda()
    est = gem.estimate_codes(store, ws, q, qo).cpu().numpy()
    assert ws.status() == 0
    S64, L1 = oracle.score_all(Q, w.queries.offsets, X, w.docs.offsets, with_l1=True)
    assert np.all(np.abs(est - S64) <= 1e-5 * L1 + 1e-6)
    gem.set_qch_form(ws, "symmetric")
    sym = gem.estimate_codes(store, ws, q, qo).cpu().numpy()
    assert np.abs(sym - S64).max() > 1e-3
    ws.close()
    store.close()


@pytest.mark.parametrize("qlens", [[32] * 5, [1, 7, 33, 64, 100, 20]])
def test_asymmetric_qch_matches_oracle_given_gpu_codes(gem, qlens):
    """Tables <q_i, C_c> and lookups: the all-sets form, the id-list form (bit
    identical to it) and score_ids in the codes form (the SIMT arithmetic) all
    within 1e-5 * m_q of the FP64 asymmetric estimate on the GPU's stored codes."""
    w = synth.exact_fp32(n_sets=300, n_queries=1)
    qs = synth.vector_sets(np.array(qlens), synth.centres(64, 1235), 98)
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("f32",))
    C = gem.train_codebook(store, k1=256, iters=5, sample=0, seed=1)
    gem.set_codebook(store, C)
    ws = gem.Workspace(store, max_queries=8, max_q_rows=512, max_q_len=128, max_cands=1000)
    gem.set_qch_form(ws, "asymmetric")
    q, qo = qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda()
    est = gem.estimate_codes(store, ws, q, qo).cpu().numpy()
    assert ws.status() == 0
    pcodes = store.export("codes").cpu().numpy()
    want = oracle.qch_asym_score_all(qs.vecs.numpy(), qs.offsets, pcodes, w.docs.offsets, C.cpu().numpy())
    tol = 1e-5 * np.array(qlens)[:, None]
    assert np.all(np.abs(est - want) <= tol), np.abs(est - want).max()
    rng = np.random.default_rng(4)
    lens = rng.integers(0, 30, size=len(qlens))
    co = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    ids = rng.integers(0, 300, size=int(co[-1])).astype(np.int64)
    co_d, ids_d = torch.from_numpy(co).cuda(), torch.from_numpy(ids).cuda()
    est_ids = gem.estimate_codes(store, ws, q, qo, co_d, ids_d).cpu().numpy()
    simt = gem.score_ids(store, ws, q, qo, co_d, ids_d, "codes").cpu().numpy()
    assert ws.status() == 0
    for t in range(len(ids)):
        b = int(np.searchsorted(co, t, side="right") - 1)
        assert est_ids[t] == est[b, ids[t]]
        assert abs(simt[t] - want[b, ids[t]]) <= 1e-5 * qlens[b]
    ws.close()
    store.close()


def test_qch_with_a_codebook_of_ragged_size_matches_oracle(gem):
    """k1 = 1,000 (not a multiple of the 64-centroid tile): the query rows are coded
    with the centroids split over CTAs; the estimate must equal the oracle's on the
    codes of the row-parallel assignment (gem.assign_codes) within 1e-5 * m_q."""
    rng = np.random.default_rng(12)
    w = synth.exact_fp32(n_sets=200, n_queries=1)
    qs = synth.vector_sets(np.array([32, 32, 17, 32]), synth.centres(64, 1235), 5)
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("f32",))
    C = _unit(rng, 1000)
    gem.set_codebook(store, torch.from_numpy(C).cuda())
    ws = gem.Workspace(store, max_queries=4, max_q_rows=128, max_q_len=32)
    q, qo = qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda()
    est = gem.estimate_codes(store, ws, q, qo).cpu().numpy()
    assert ws.status() == 0
    qcodes = gem.assign_codes(q, torch.from_numpy(C).cuda()).cpu().numpy()
    pcodes = store.export("codes").cpu().numpy()
    want = oracle.qch_score_all(qcodes, qs.offsets, pcodes, w.docs.offsets, C)
    assert np.all(np.abs(est - want) <= 1e-5 * np.array([32, 32, 17, 32])[:, None])
    ws.close()
    store.close()
