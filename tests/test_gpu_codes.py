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


@pytest.mark.parametrize("k1", [4099, 300])
def test_assign_codes_tensor_core_path_equals_simt_path(gem, k1):
    """From 16,384 rows the codes come from the tensor cores (three bf16
    products per dot, six candidates per row, an FP32 recheck by the SIMT
    kernel's own FMA chain, the SIMT kernel for the rows the candidates cannot
    decide).  The same rows in slices of 8,192 take the SIMT kernel.  Codes and
    best values must be bit-identical, on data with dense near-ties (centroids
    that are perturbed rows of the data), exact ties (a duplicated centroid), a
    NaN centroid, a zero row, a NaN row and a k1 that is not a multiple of the
    128-centroid tile."""
    rng = np.random.default_rng(k1)
    n = 40_000
    X = synth.draw_vectors(n, synth.centres(64, 8), 21).numpy().copy()
    C = X[rng.choice(n, k1, replace=False)] + rng.normal(0, 0.01, (k1, 128)).astype(np.float32)
    C /= np.linalg.norm(C, axis=1, keepdims=True)
    C[k1 - 1] = C[5]                      # exact tie: index 5 must win
    C[17] = np.nan                        # never chosen (a NaN dot counts as -inf)
    X[100] = 0.0                          # every dot 0: code 0
    X[200] = np.nan                       # every dot NaN: code 0
    X[300] = C[5]                         # ties 5 / k1-1 exactly
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
    codes, best = gem.assign_codes(Xd, Cd, with_best=True)
    parts = [gem.assign_codes(Xd[a:a + 8192], Cd, with_best=True) for a in range(0, n, 8192)]
    codes_s = torch.cat([p[0] for p in parts]).cpu().numpy()
    best_s = torch.cat([p[1] for p in parts]).cpu().numpy()
    codes, best = codes.cpu().numpy(), best.cpu().numpy()
    np.testing.assert_array_equal(codes, codes_s)
    np.testing.assert_array_equal(best.view(np.uint32), best_s.view(np.uint32))
    assert codes[100] == 0 and codes[200] == 0 and codes[300] == 5
    assert codes.min() >= 0 and codes.max() < k1 and not np.any(codes == 17)
    # against FP64 (the NaN centroid is never the nearest): exact outside the
    # 2 * EPS band, within it a valid choice
    ok = np.isfinite(X).all(axis=1) & (np.abs(X).sum(axis=1) > 0)
    Cf = np.nan_to_num(C.astype(np.float64))
    sims = X[ok].astype(np.float64) @ Cf.T
    sims[:, 17] = -np.inf
    top2 = np.sort(sims, axis=1)[:, -2:]
    clear = top2[:, 1] - top2[:, 0] > 2 * EPS
    np.testing.assert_array_equal(codes[ok][clear], np.argmax(sims, axis=1)[clear])
    got = sims[np.arange(len(sims)), codes[ok]]
    assert np.all(got >= sims.max(axis=1) - 2 * EPS)


def test_assign_codes_centroid_maps_to_itself_and_ties_go_low(gem):
    rng = np.random.default_rng(3)
    C = _unit(rng, 300)
    codes = gem.assign_codes(torch.from_numpy(C).cuda(), torch.from_numpy(C).cuda()).cpu().numpy()
    np.testing.assert_array_equal(codes, np.arange(300))
    Cdup = np.vstack([C[:10], C[4:5], C[10:]])          # row 10 repeats row 4
    codes = gem.assign_codes(torch.from_numpy(C[4:5]).cuda(), torch.from_numpy(Cdup).cuda()).cpu().numpy()
    assert codes.tolist() == [4]


def test_train_codebook_fixed_point_invariants(gem):
    """After many Lloyd steps the trained codebook is a fixed point of the
    update: unit centroids, each the normalised mean of the vectors coded to it.
    (A single step against the oracle's update is in test_gpu_cluster.py.)"""
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
    S64 = oracle.score_all(Q, w.queries.offsets, X, w.docs.offsets)
    # each table entry is one 128-term FP32 FMA chain of unit vectors (absolute
    # error <= 128 * 2^-24 < 7.7e-6 per term, whatever the term's size), the
    # per-set sum a 5-level butterfly (<= 5 * 2^-24 relative): < 1e-5 per query vector
    m_q = np.diff(w.queries.offsets)[:, None]
    assert np.all(np.abs(est.cpu().numpy() - S64) <= 1e-5 * m_q)


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
    S64 = oracle.score_all(Q, w.queries.offsets, X, w.docs.offsets)
    # the bound of the symmetric lossless test: < 1e-5 per query vector
    assert np.all(np.abs(est - S64) <= 1e-5 * np.diff(w.queries.offsets)[:, None])
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


def test_query_codes_split_tie_break_and_nan_rows(gem):
    """Query codes with the centroids split over CTAs (k1 = 1,000, few rows).
    Centroid 4 = e_1 and centroid 700 = e_1 + e_2 (another 64-centroid span) both
    give exactly 1.0 against a query row e_1: the lower index, 4, must win the
    merge across CTAs.  The two choices give different estimates (the table rows
    <C_4, C_c> and <C_700, C_c> differ), so the estimate shows which one won.  A
    query row of NaNs gets code 0 (every dot counts as -inf, the lowest index
    wins) and a stored NaN row also gets a code in range."""
    rng = np.random.default_rng(31)
    k1 = 1000
    C = _unit(rng, k1)
    C[:, 0] *= 0.05                        # no other centroid comes near e_1
    C /= np.linalg.norm(C, axis=1, keepdims=True)
    C[4] = 0.0
    C[4, 0] = 1.0
    C[700] = 0.0
    C[700, 0] = 1.0
    C[700, 1] = 1.0
    w = synth.exact_fp32(n_sets=150, n_queries=1)
    X = w.docs.vecs.numpy().copy()
    X[5] = np.nan                          # one stored row of NaNs (set 0)
    store = gem.Store(torch.from_numpy(X).cuda(), w.docs.offsets, keep=("f32",))
    gem.set_codebook(store, torch.from_numpy(C).cuda())
    pcodes = store.export("codes").cpu().numpy()
    assert pcodes.min() >= 0 and pcodes.max() < k1 and pcodes[5] == 0
    qs = synth.vector_sets(np.array([32, 32, 20]), synth.centres(64, 1235), 77)
    Q = qs.vecs.numpy().copy()
    Q[[0, 33, 40, 70]] = 0.0
    Q[[0, 33, 40, 70], 0] = 1.0            # rows equal to e_1: ties 4 / 700
    Q[50] = np.nan                         # a NaN query row (query 1)
    q, qo = torch.from_numpy(Q).cuda(), torch.from_numpy(qs.offsets).cuda()
    qcodes = gem.assign_codes(q, torch.from_numpy(C).cuda()).cpu().numpy().astype(np.int64)
    assert qcodes[[0, 33, 40, 70]].tolist() == [4, 4, 4, 4] and qcodes[50] == 0
    ok = np.isfinite(Q).all(axis=1)
    _check_codes(Q[ok], C, qcodes[ok])
    ws = gem.Workspace(store, max_queries=3, max_q_rows=96, max_q_len=32)
    est = gem.estimate_codes(store, ws, q, qo).cpu().numpy()
    assert ws.status() == 0
    live = np.arange(1, 150)               # set 0 holds the NaN row
    want = oracle.qch_score_all(qcodes, qs.offsets, pcodes, w.docs.offsets, C)
    m_q = np.diff(qs.offsets)[:, None]
    assert np.all(np.abs(est[:, live] - want[:, live]) <= 1e-5 * m_q)
    # with code 700 in place of 4 the estimate moves by far more than the tolerance
    alt = qcodes.copy()
    alt[[0, 33, 40, 70]] = 700
    moved = oracle.qch_score_all(alt, qs.offsets, pcodes, w.docs.offsets, C)
    assert np.abs(moved[:, live] - want[:, live]).max() > 1e-2
    ws.close()
    store.close()


@pytest.mark.parametrize("form", ["symmetric", "asymmetric"])
def test_search_codes_first_pass_then_exact_rerank(gem, form):
    """gem_search with GEM_CODES (Algorithm 5's order): the qCH estimate of every
    set, its top-R, the exact FP32 rerank of that pool and the top-k of it, in one
    call.  The pool must be the oracle's top-R of the FP64 estimate on the GPU's
    codes wherever the R-th and (R+1)-th estimates are apart by more than twice
    the estimate's tolerance; the result must then be the oracle's rerank of that
    pool (exact-score swaps within 1e-6 allowed)."""
    w = synth.exact_fp32(n_sets=400, n_queries=12)
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("f32",))
    C = gem.train_codebook(store, k1=256, iters=5, sample=0, seed=3)
    gem.set_codebook(store, C)
    R, K = 60, 10
    ws = gem.Workspace(store, max_queries=12, max_q_rows=12 * 32, max_q_len=32, max_cands=12 * R, max_k=R)
    gem.set_qch_form(ws, form)
    q, qo = w.queries.vecs.cuda(), torch.from_numpy(w.queries.offsets).cuda()
    ids, sc = gem.search(store, ws, q, qo, "codes", rerank_depth=R, k=K)
    ids0, _ = gem.search(store, ws, q, qo, "codes", rerank_depth=0, k=K)
    assert ws.status() == 0
    ids, sc, ids0 = ids.cpu().numpy(), sc.cpu().numpy(), ids0.cpu().numpy()
    Cn = C.cpu().numpy()
    pcodes = store.export("codes").cpu().numpy()
    Q, X = w.queries.vecs.numpy(), w.docs.vecs.numpy()
    if form == "symmetric":
        qcodes = gem.assign_codes(q, C).cpu().numpy()
        est = oracle.qch_score_all(qcodes, w.queries.offsets, pcodes, w.docs.offsets, Cn)
    else:
        est = oracle.qch_asym_score_all(Q, w.queries.offsets, pcodes, w.docs.offsets, Cn)
    S64, L1 = oracle.score_all(Q, w.queries.offsets, X, w.docs.offsets, with_l1=True)
    tol = 1e-5 * 32
    checked = 0
    for b in range(12):
        order = np.lexsort((np.arange(400), -est[b]))
        if est[b, order[R - 1]] - est[b, order[R]] <= 2 * tol:
            continue                       # pool boundary inside the estimate's tolerance
        checked += 1
        pool = order[:R]
        want_ids, want_sc = oracle.rerank(Q[w.queries.offsets[b]:w.queries.offsets[b + 1]], np.array([0, 32]),
                                          X, w.docs.offsets, pool[None, :], K)
        want_ids, want_sc = want_ids[0], want_sc[0]
        for x in set(want_ids.tolist()) ^ set(ids[b].tolist()):
            assert abs(S64[b, x] - want_sc[-1]) <= 1e-6 * max(1.0, abs(want_sc[-1])), (b, x)
        assert set(ids[b].tolist()) <= set(pool.tolist())
        assert np.all(np.abs(sc[b] - S64[b, ids[b]]) <= 1e-5 * L1[b, ids[b]])
        # rerank_depth 0: the estimate's own top-k
        top0 = order[:K]
        if est[b, order[K - 1]] - est[b, order[K]] > 2 * tol:
            assert set(ids0[b].tolist()) == set(top0.tolist())
    assert checked >= 8, checked
    ws.close()
    store.close()


def test_assign_partial_last_unit_costs_no_more_than_whole_units(gem):
    """The tensor cores take rows in units of 256; a unit that runs past the
    last row holds zero-filled rows.  Those rows track no candidates: 148,000
    rows (a last unit of 32 live rows) cost about as much as 147,712 (whole
    units) against 65,536 centroids.  When every column of the dead rows tied
    the running maximum, the first took 55 ms and the second 4.4 ms."""
    rng = np.random.default_rng(12)
    X = rng.normal(size=(148_000, 128)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    C = rng.normal(size=(65_536, 128)).astype(np.float32)
    C /= np.linalg.norm(C, axis=1, keepdims=True)
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()

    def ms(n):
        gem.assign_codes(Xd[:n], Cd)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            gem.assign_codes(Xd[:n], Cd)
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / 3

    whole, partial = ms(147_712), ms(148_000)
    assert partial <= 2.0 * whole + 0.5, (partial, whole)
    # and the codes of the shared rows agree
    a = gem.assign_codes(Xd[:147_712], Cd)
    b = gem.assign_codes(Xd, Cd)[:147_712]
    assert torch.equal(a, b)
