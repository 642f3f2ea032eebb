"""Pins for the FP64 oracle: brute force, closed forms, invariants and the paper's
worked example.  Nothing here touches the CUDA library."""
import itertools
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _unit(rng, n, d):
    x = rng.standard_normal((n, d))
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def _brute_ch(A, B):
    """Eq. 1 with pure-Python loops (inputs are small integers, so FP64 is exact)."""
    total = 0.0
    for a in A:
        best = None
        for b in B:
            s = sum(float(x) * float(y) for x, y in zip(a, b))
            best = s if best is None or s > best else best
        total += best
    return total


# --------------------------------------------------------------------------- CH

def test_intro_worked_example():
    g = json.load(open(os.path.join(GOLD, "intro_example.json")))
    Q = np.array(g["sims"])
    P = np.eye(4)                      # <q_i, e_j> = sims[i][j]
    assert oracle.chamfer(Q, P) == pytest.approx(g["ch"], abs=1e-12)
    _, _, jstar = oracle.maxsim_grad(Q, P)
    assert list(jstar) == g["argmax"]


@pytest.mark.parametrize("seed", range(6))
def test_chamfer_matches_brute_force_on_integers(seed):
    rng = np.random.default_rng(seed)
    d = int(rng.integers(1, 9))
    lens = rng.integers(1, 5, size=5)
    X = rng.integers(-3, 4, size=(int(lens.sum()), d)).astype(np.float64)
    off = np.concatenate([[0], np.cumsum(lens)])
    mq = rng.integers(1, 5, size=3)
    q = rng.integers(-3, 4, size=(int(mq.sum()), d)).astype(np.float64)
    qo = np.concatenate([[0], np.cumsum(mq)])
    S = oracle.score_all(q, qo, X, off)
    for b in range(3):
        for n in range(5):
            want = _brute_ch(q[qo[b]:qo[b + 1]], X[off[n]:off[n + 1]])
            assert S[b, n] == want
            assert oracle.chamfer(q[qo[b]:qo[b + 1]], X[off[n]:off[n + 1]]) == want
    co = np.array([0, 2, 2, 5])
    ids = np.array([4, 0, 1, 1, 3])
    got = oracle.score_ids(q, qo, X, off, co, ids)
    want = [S[0, 4], S[0, 0], S[2, 1], S[2, 1], S[2, 3]]
    assert list(got) == want


def test_single_pair_is_dot_product():
    rng = np.random.default_rng(1)
    q, p = rng.standard_normal((1, 128)), rng.standard_normal((1, 128))
    assert oracle.chamfer(q, p) == pytest.approx(math.fsum(q[0] * p[0]), rel=1e-14)


def test_single_doc_vector_closed_form():
    # m_p = 1: every query vector's max is the one product, so CH = <sum_i q_i, p>.
    rng = np.random.default_rng(2)
    Q, p = rng.standard_normal((7, 16)), rng.standard_normal((1, 16))
    assert oracle.chamfer(Q, p) == pytest.approx(float(Q.sum(0) @ p[0]), rel=1e-13)


def test_unit_set_against_itself_equals_cardinality():
    rng = np.random.default_rng(3)
    for m in (1, 5, 33):
        P = _unit(rng, m, 128)
        assert oracle.chamfer(P, P) == pytest.approx(m, abs=1e-12)


def test_permutation_invariance_and_asymmetry():
    rng = np.random.default_rng(4)
    Q, P = _unit(rng, 6, 32), _unit(rng, 9, 32)
    base = oracle.chamfer(Q, P)
    assert oracle.chamfer(Q[rng.permutation(6)], P) == pytest.approx(base, abs=1e-13)
    assert oracle.chamfer(Q, P[rng.permutation(9)]) == pytest.approx(base, abs=1e-13)
    # the operands are not interchangeable: a transposed implementation fails here
    assert abs(oracle.chamfer(P, Q) - base) > 1e-3


def test_superset_monotone_and_query_additive():
    rng = np.random.default_rng(5)
    Q1, Q2, P, P2 = _unit(rng, 4, 16), _unit(rng, 3, 16), _unit(rng, 5, 16), _unit(rng, 4, 16)
    assert oracle.chamfer(Q1, np.vstack([P, P2])) >= oracle.chamfer(Q1, P) - 1e-15
    assert oracle.chamfer(np.vstack([Q1, Q2]), P) == pytest.approx(
        oracle.chamfer(Q1, P) + oracle.chamfer(Q2, P), abs=1e-13)


def test_terms_bounded_by_single_pair_products():
    rng = np.random.default_rng(6)
    Q, P = _unit(rng, 8, 64), _unit(rng, 11, 64)
    sims = Q @ P.T
    ch = oracle.chamfer(Q, P)
    assert sims.min(1).sum() - 1e-12 <= ch <= sims.max(1).sum() + 1e-12
    assert abs(ch) <= len(Q) + 1e-12
    # dropping one query vector removes exactly its best single-pair product
    assert ch - oracle.chamfer(Q[1:], P) == pytest.approx(sims[0].max(), abs=1e-13)


def test_score_all_on_generated_workload():
    w = synth.exact_fp32(n_sets=40, n_queries=2)
    S = oracle.score_all(w.queries.vecs, w.queries.offsets, w.docs.vecs, w.docs.offsets)
    qv, dv = w.queries.vecs.numpy(), w.docs.vecs.numpy()
    for b in range(2):
        for n in (0, 17, 39):
            Q = qv[w.queries.offsets[b]:w.queries.offsets[b + 1]].astype(np.float64)
            P = dv[w.docs.offsets[n]:w.docs.offsets[n + 1]].astype(np.float64)
            want = sum(max(float(np.dot(a, p)) for p in P) for a in Q)
            assert S[b, n] == pytest.approx(want, abs=1e-12)


# --------------------------------------------------------------------------- top-k

def _brute_topk(scores, k, ids):
    pairs = sorted(zip(scores, ids), key=lambda t: (-t[0], t[1]))
    return [p[1] for p in pairs[:k]], [p[0] for p in pairs[:k]]


@pytest.mark.parametrize("seed", range(4))
def test_topk_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300))
    s = np.round(rng.standard_normal(n), 1)           # many ties
    ids = rng.permutation(10 * n)[:n]
    for k in (1, 5, n, n + 3):
        got_i, got_s = oracle.topk(s, k, ids)
        want_i, want_s = _brute_topk(s.tolist(), k, ids.tolist())
        assert got_i.tolist() == want_i
        assert got_s.tolist() == want_s


def test_topk_all_equal_and_full_sort():
    got_i, _ = oracle.topk(np.full(50, 0.25), 7)
    assert got_i.tolist() == list(range(7))
    s = np.array([3.0, 1.0, 2.0])
    got_i, got_s = oracle.topk(s, 10)
    assert got_i.tolist() == [0, 2, 1] and got_s.tolist() == [3.0, 2.0, 1.0]


def test_rerank_is_topk_of_exact_scores_over_pool():
    w = synth.exact_fp32(n_sets=30, n_queries=2)
    S = oracle.score_all(w.queries.vecs, w.queries.offsets, w.docs.vecs, w.docs.offsets)
    pool = np.array([[3, 7, 1, 22, 9, -1], [0, 1, 2, 3, 4, 5]])
    ids, sc = oracle.rerank(w.queries.vecs, w.queries.offsets, w.docs.vecs, w.docs.offsets, pool, 4)
    for b in range(2):
        p = pool[b][pool[b] >= 0]
        want_i, want_s = _brute_topk(S[b, p].tolist(), 4, p.tolist())
        assert ids[b].tolist() == want_i
        assert sc[b] == pytest.approx(want_s, abs=1e-12)
    ids, sc = oracle.rerank(w.queries.vecs, w.queries.offsets[:2], w.docs.vecs, w.docs.offsets,
                            np.array([[5, -1, -1]]), 2)
    assert ids.tolist() == [[5, -1]] and sc[0, 1] == -np.inf


# --------------------------------------------------------------------------- codes / qCH

def test_assign_codes_brute_force_self_and_ties():
    rng = np.random.default_rng(7)
    C = _unit(rng, 20, 8)
    X = _unit(rng, 50, 8)
    codes = oracle.assign_codes(X, C)
    for x, c in zip(X, codes):
        sims = [float(np.dot(x, cc)) for cc in C]
        assert c == max(range(20), key=lambda t: (sims[t], -t))
    assert oracle.assign_codes(C, C).tolist() == list(range(20))
    Cdup = np.vstack([C[:5], C[3:4], C[5:]])      # row 5 duplicates row 3
    assert oracle.assign_codes(C[3:4], Cdup).tolist() == [3]


def test_qch_lossless_codes_equal_exact_chamfer():
    """With a codebook holding every vector exactly, NN is the identity and qCH is CH."""
    rng = np.random.default_rng(8)
    Q, P = _unit(rng, 6, 32), _unit(rng, 9, 32)
    C = np.vstack([Q, P])
    qc, pc = oracle.assign_codes(Q, C), oracle.assign_codes(P, C)
    assert qc.tolist() == list(range(6)) and pc.tolist() == list(range(6, 15))
    ch = oracle.chamfer(Q, P)
    assert oracle.qch_similarity(qc, pc, C) == pytest.approx(ch, abs=1e-13)
    assert oracle.qch_distance(qc, pc, C) == pytest.approx(len(Q) - ch, abs=1e-13)


def test_qch_brute_force_and_batched_forms():
    rng = np.random.default_rng(9)
    C = _unit(rng, 16, 8)
    lens = np.array([3, 1, 4, 2])
    off = np.concatenate([[0], np.cumsum(lens)])
    pc = rng.integers(0, 16, size=int(lens.sum()))
    qc = rng.integers(0, 16, size=5)
    qo = np.array([0, 2, 5])
    S = oracle.qch_score_all(qc, qo, pc, off, C)
    for b in range(2):
        for n in range(4):
            a = qc[qo[b]:qo[b + 1]]
            bb = pc[off[n]:off[n + 1]]
            dist = sum(min(1.0 - float(np.dot(C[x], C[y])) for y in bb) for x in a)
            assert oracle.qch_distance(a, bb, C) == pytest.approx(dist, abs=1e-13)
            assert S[b, n] == pytest.approx(len(a) - dist, abs=1e-13)
    got = oracle.qch_score_ids(qc, qo, pc, off, np.array([0, 1, 3]), np.array([2, 0, 3]), C)
    assert got.tolist() == pytest.approx([S[0, 2], S[1, 0], S[1, 3]], abs=1e-13)


def test_asymmetric_qch_pins():
    """Asymmetric qCH (stored side quantized only): brute force; a codebook holding
    every stored vector makes it the exact CH whatever the query vectors are; with
    the query vectors themselves centroids it equals the symmetric estimate."""
    rng = np.random.default_rng(21)
    Q, P = _unit(rng, 5, 16), _unit(rng, 7, 16)
    C = np.vstack([_unit(rng, 3, 16), P])
    pc = oracle.assign_codes(P, C)
    assert pc.tolist() == list(range(3, 10))
    assert oracle.qch_asym_similarity(Q, pc, C) == pytest.approx(oracle.chamfer(Q, P), abs=1e-13)
    C2 = _unit(rng, 12, 16)
    pc2 = rng.integers(0, 12, size=7)
    brute = sum(max(float(np.dot(q, C2[c])) for c in pc2) for q in Q)
    assert oracle.qch_asym_similarity(Q, pc2, C2) == pytest.approx(brute, abs=1e-13)
    qc = np.array([4, 0, 11])
    assert oracle.qch_asym_similarity(C2[qc], pc2, C2) == pytest.approx(oracle.qch_similarity(qc, pc2, C2),
                                                                       abs=1e-13)
    lens = np.array([3, 4])
    off = np.concatenate([[0], np.cumsum(lens)])
    S = oracle.qch_asym_score_all(Q, np.array([0, 2, 5]), pc2, off, C2)
    for b, (q0, q1) in enumerate([(0, 2), (2, 5)]):
        for n in range(2):
            want = oracle.qch_asym_similarity(Q[q0:q1], pc2[off[n]:off[n + 1]], C2)
            assert S[b, n] == pytest.approx(want, abs=1e-13)


def test_l2_chamfer_pins():
    """Sim = -||a - b||: brute force on a hand example; zero on a set against
    itself; invariant under a common translation and 1-homogeneous under a common
    scale (the inner-product form is neither); on unit vectors the closed form
    -sum_i sqrt(2 - 2 max_j <a_i, b_j>) links it to the inner-product maxima."""
    A = np.array([[0.0, 0.0], [3.0, 4.0]])
    B = np.array([[0.0, 1.0], [6.0, 8.0], [3.0, 0.0]])
    # nearest of (0,0): (0,1) at 1; nearest of (3,4): (3,0) at 4 (vs (6,8) at 5)
    assert oracle.chamfer_l2(A, B) == -5.0
    rng = np.random.default_rng(31)
    X, Y = rng.standard_normal((6, 9)), rng.standard_normal((4, 9))
    assert oracle.chamfer_l2(X, X) == 0.0
    t = rng.standard_normal(9) * 5
    assert oracle.chamfer_l2(X + t, Y + t) == pytest.approx(oracle.chamfer_l2(X, Y), rel=1e-12)
    assert oracle.chamfer_l2(2.5 * X, 2.5 * Y) == pytest.approx(2.5 * oracle.chamfer_l2(X, Y), rel=1e-12)
    U, V = _unit(rng, 5, 9), _unit(rng, 7, 9)
    closed = -np.sqrt(np.maximum(0.0, 2.0 - 2.0 * (U @ V.T).max(axis=1))).sum()
    assert oracle.chamfer_l2(U, V) == pytest.approx(closed, abs=1e-12)
    lens = np.array([2, 3])
    off = np.concatenate([[0], np.cumsum(lens)])
    P = np.vstack([Y[:2], Y[1:]])
    S, L1 = oracle.score_all_l2(X, np.array([0, 4, 6]), P, off, with_l1=True)
    for b, (q0, q1) in enumerate([(0, 4), (4, 6)]):
        for n in range(2):
            assert S[b, n] == oracle.chamfer_l2(X[q0:q1], P[off[n]:off[n + 1]])
    np.testing.assert_array_equal(L1, -S)


def _w1_1d(x, y):
    """Closed form of the 1-D Wasserstein-1 distance between uniform point masses:
    the integral over u in (0, 1) of |F^-1(u) - G^-1(u)|, by merging the quantile
    breakpoints of the two sorted samples."""
    x, y = np.sort(x), np.sort(y)
    cuts = np.union1d(np.arange(len(x) + 1) / len(x), np.arange(len(y) + 1) / len(y))
    total = 0.0
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        mid = 0.5 * (lo + hi)
        total += (hi - lo) * abs(x[int(mid * len(x))] - y[int(mid * len(y))])
    return total


def test_emd_solver_pins():
    """The LP of Eq. 11-12 against: the 1-D closed form (unequal sizes); the
    assignment problem for equal sizes (Birkhoff: an optimal plan is a
    permutation / m, solved by scipy's linear_sum_assignment, another routine);
    a single source (the only feasible plan); symmetry; zero on a set with itself."""
    rng = np.random.default_rng(41)
    for m1, m2 in ((3, 5), (7, 4), (6, 6), (1, 9)):
        x, y = rng.standard_normal(m1), rng.standard_normal(m2)
        D = np.abs(x[:, None] - y[None, :])
        assert oracle.emd_cost(D) == pytest.approx(_w1_1d(x, y), abs=1e-9)
    from scipy.optimize import linear_sum_assignment
    D = rng.uniform(0, 2, size=(8, 8))
    r, c = linear_sum_assignment(D)
    assert oracle.emd_cost(D) == pytest.approx(D[r, c].sum() / 8, abs=1e-9)
    D1 = rng.uniform(0, 2, size=(1, 6))
    assert oracle.emd_cost(D1) == pytest.approx(D1.mean(), abs=1e-12)
    P, Q = _unit(rng, 5, 16), _unit(rng, 9, 16)
    assert oracle.emd(P, Q) == pytest.approx(oracle.emd(Q, P), abs=1e-9)
    assert oracle.emd(P, P) == pytest.approx(0.0, abs=1e-9)


def test_chamfer_lower_bounds_emd_and_qemd_reductions():
    """Eq. 10: the averaged Chamfer distance (1/m_q) sum_i min_j d_X(q_i, p_j)
    never exceeds EMD(Q, P); with a codebook holding every vector, qEMD is EMD;
    with both sets coded to the same centroids qEMD is 0 up to rounding."""
    rng = np.random.default_rng(42)
    for _ in range(5):
        Q, P = _unit(rng, int(rng.integers(1, 9)), 16), _unit(rng, int(rng.integers(1, 9)), 16)
        avg_ch = (len(Q) - oracle.chamfer(Q, P)) / len(Q)
        assert avg_ch <= oracle.emd(Q, P) + 1e-9
    Q, P = _unit(rng, 4, 16), _unit(rng, 6, 16)
    C = np.vstack([Q, P])
    qc, pc = oracle.assign_codes(Q, C), oracle.assign_codes(P, C)
    assert oracle.qemd(qc, pc, C) == pytest.approx(oracle.emd(Q, P), abs=1e-9)
    codes = np.array([2, 5, 5, 7])
    assert oracle.qemd(codes, codes[::-1], _unit(rng, 9, 16)) == pytest.approx(0.0, abs=1e-9)


def test_codebook_size_formula_reproduces_paper():
    g = json.load(open(os.path.join(GOLD, "codebook_sizes.json")))
    for c in g["cases"]:
        assert oracle.k1_for(c["vectors"]) == c["k1"], c["dataset"]


# --------------------------------------------------------------------------- formats

def test_bf16_round_matches_torch_and_ties_to_even():
    rng = np.random.default_rng(10)
    x = np.concatenate([rng.standard_normal(10000).astype(np.float32),
                        (rng.standard_normal(1000) * 1e-39).astype(np.float32)])
    want = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    np.testing.assert_array_equal(oracle.bf16_round(x), want)
    # exact halfway cases between 1 and the next bfloat16 (1 + 2^-7)
    half = np.float32(1.0 + 2.0 ** -8)
    assert oracle.bf16_round(np.array([half]))[0] == 1.0                 # ties to even (down)
    half2 = np.float32(1.0 + 3 * 2.0 ** -8)
    assert oracle.bf16_round(np.array([half2]))[0] == np.float32(1.0 + 2 * 2.0 ** -7)  # up


def test_fp8_e4m3_round_matches_torch_in_range():
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.uniform(-448, 448, 5000), rng.standard_normal(5000) * 0.01,
                        rng.standard_normal(1000) * 1e-3]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).float().numpy().astype(np.float64)
    np.testing.assert_array_equal(oracle.fp8_e4m3_round(x), want)
    # every finite E4M3 value maps to itself; saturation at the top
    allv = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).float().numpy()
    allv = allv[np.isfinite(allv)]
    np.testing.assert_array_equal(oracle.fp8_e4m3_round(allv), allv.astype(np.float64))
    assert oracle.fp8_e4m3_round(np.array([1000.0, -500.0])).tolist() == [448.0, -448.0]


def test_fp8_quantize_scales_and_error_bound():
    rng = np.random.default_rng(12)
    X = _unit(rng, 200, 128).astype(np.float32)
    codes, s = oracle.fp8_e4m3_quantize(X)
    assert np.all(np.abs(codes).max(axis=1) == 448.0)
    deq = codes * s[:, None].astype(np.float64)
    # normal range: relative half-spacing 2^-4; below 2^-6 * s the spacing is 2^-9 * s
    bound = np.maximum(np.abs(X) * 2.0 ** -4, s[:, None] * 2.0 ** -10) * (1 + 1e-6)
    assert np.all(np.abs(deq - X) <= bound)
    c0, s0 = oracle.fp8_e4m3_quantize(np.zeros((1, 4), np.float32))
    assert s0[0] == 1.0 and np.all(c0 == 0)


def test_fp8_quantize_sets_scale_rule_and_codes():
    """Per-set power-of-two scales: hand cases at the boundaries of the rule, the
    codes against torch's own E4M3 conversion of x / s, and the scale against a
    search over exponents written with math.ldexp."""
    import math
    rows = np.array([[448.0, -1.0], [3.0, 0.0],          # set 0: max 448 -> s = 1
                     [-449.0, 0.5],                      # set 1: max 449 -> s = 2
                     [224.0, 10.0],                      # set 2: max 224 -> s = 1/2 (224 <= 448/2)
                     [0.0, 0.0], [0.0, -0.0],            # set 3: zero set -> s = 1
                     [1e-40, 0.0],                       # set 4: subnormal max -> s = 2^-126
                     [224.5, 0.0]], np.float32)          # set 5: just above 224 -> s = 1
    off = np.array([0, 2, 3, 4, 6, 7, 8])
    codes, s = oracle.fp8_e4m3_quantize_sets(rows, off)
    assert s.tolist() == [1.0, 2.0, 0.5, 1.0, 2.0 ** -126, 1.0]
    assert codes[2].tolist() == [-224.0, 0.25] and codes[3].tolist() == [448.0, 20.0]
    assert codes[7].tolist() == [224.0, 0.0]            # 224.5 rounds to the E4M3 grid (spacing 32)
    assert np.all(codes[4:6] == 0)
    rng = np.random.default_rng(21)
    lens = rng.integers(1, 40, 300)
    off = np.concatenate([[0], np.cumsum(lens)])
    X = (rng.standard_normal((off[-1], 128)) * np.repeat(10.0 ** rng.uniform(-30, 30, 300), lens)[:, None])
    X = X.astype(np.float32)
    codes, s = oracle.fp8_e4m3_quantize_sets(X, off)
    for n in range(300):
        a = float(np.abs(X[off[n]:off[n + 1]]).max())
        k = next(k for k in range(-126, 129) if a <= 448.0 * math.ldexp(1.0, k))
        assert s[n] == math.ldexp(1.0, k)
        amax_code = np.abs(codes[off[n]:off[n + 1]]).max()
        assert amax_code <= 448.0 and (k == -126 or amax_code > 224.0 - 16.0)
        want = torch.from_numpy(X[off[n]:off[n + 1]] / s[n]).to(torch.float8_e4m3fn).double().numpy()
        np.testing.assert_array_equal(codes[off[n]:off[n + 1]], want)
    # dequantisation error: half a spacing of E4M3 relative to the set's scale
    sv = np.repeat(s, lens)[:, None].astype(np.float64)
    deq = codes * sv
    assert np.all(np.abs(deq - X) <= np.maximum(np.abs(X) * 2.0 ** -4, sv * 2.0 ** -10) * (1 + 1e-12))
    # the common scale leaves the argmax of Eq. 1's inner max unchanged
    q = rng.standard_normal(128)
    for n in range(0, 300, 37):
        blk = codes[off[n]:off[n + 1]]
        assert np.max(blk @ q) * s[n] == np.max((blk * float(s[n])) @ q)


# --------------------------------------------------------------------------- gradients

def test_maxsim_grad_euler_identity_and_finite_differences():
    rng = np.random.default_rng(13)
    Q, P = _unit(rng, 5, 16), _unit(rng, 7, 16)
    dQ, dP, jstar = oracle.maxsim_grad(Q, P)
    ch = oracle.chamfer(Q, P)
    # 1-homogeneous in Q (and in P) for a fixed argmax
    assert float((dQ * Q).sum()) == pytest.approx(ch, abs=1e-13)
    assert float((dP * P).sum()) == pytest.approx(ch, abs=1e-13)
    h = 1e-6
    for (M, G) in ((Q, dQ), (P, dP)):
        for idx in [(0, 0), (2, 5), (4, 15)]:
            Mp, Mm = M.copy(), M.copy()
            Mp[idx] += h
            Mm[idx] -= h
            args_p = (Mp, P) if M is Q else (Q, Mp)
            args_m = (Mm, P) if M is Q else (Q, Mm)
            fd = (oracle.chamfer(*args_p) - oracle.chamfer(*args_m)) / (2 * h)
            assert fd == pytest.approx(G[idx], abs=1e-7)


def test_contrastive_chain_rule_finite_differences_4x4():
    """FD check of dL/dQ and dL/dP through Eq. 1 and the contrastive loss."""
    rng = np.random.default_rng(14)
    tau, B, ND, m, d = 0.05, 4, 4, 3, 8
    Qs = [_unit(rng, m, d) for _ in range(B)]
    Ps = [[_unit(rng, int(rng.integers(2, 5)), d) for _ in range(ND)] for _ in range(B)]

    def loss(Qs, Ps):
        S = np.array([[oracle.chamfer(Qs[b], Ps[b][n]) for n in range(ND)] for b in range(B)])
        return oracle.contrastive_loss(S, tau), S

    L, S = loss(Qs, Ps)
    g = oracle.contrastive_dscores(S, tau)
    dQs = [np.zeros_like(x) for x in Qs]
    dPs = [[np.zeros_like(p) for p in row] for row in Ps]
    for b in range(B):
        for n in range(ND):
            dq, dp, _ = oracle.maxsim_grad(Qs[b], Ps[b][n])
            margin = np.sort(Qs[b] @ Ps[b][n].T, axis=1)
            assert margin.shape[1] < 2 or np.min(margin[:, -1] - margin[:, -2]) > 1e-4
            dQs[b] += g[b, n] * dq
            dPs[b][n] += g[b, n] * dp
    h = 1e-6
    for b, i, k in [(0, 0, 0), (1, 2, 3), (3, 1, 7)]:
        Qp = [x.copy() for x in Qs]
        Qm = [x.copy() for x in Qs]
        Qp[b][i, k] += h
        Qm[b][i, k] -= h
        fd = (loss(Qp, Ps)[0] - loss(Qm, Ps)[0]) / (2 * h)
        assert fd == pytest.approx(dQs[b][i, k], rel=1e-5, abs=1e-7)
    for b, n, j, k in [(0, 0, 0, 1), (2, 3, 1, 4)]:
        Pp = [[p.copy() for p in row] for row in Ps]
        Pm = [[p.copy() for p in row] for row in Ps]
        Pp[b][n][j, k] += h
        Pm[b][n][j, k] -= h
        fd = (loss(Qs, Pp)[0] - loss(Qs, Pm)[0]) / (2 * h)
        assert fd == pytest.approx(dPs[b][n][j, k], rel=1e-5, abs=1e-7)


def test_contrastive_dscores_rows_sum_to_zero():
    rng = np.random.default_rng(15)
    S = rng.standard_normal((5, 6))
    g = oracle.contrastive_dscores(S, 0.05)
    np.testing.assert_allclose(g.sum(axis=1), 0.0, atol=1e-12)
    assert np.all(g[:, 0] <= 0) and np.all(g[:, 1:] >= 0)


# --------------------------------------------------------------------------- k-means (Sec. 4.1.1)

def test_kmeans_update_fixed_point_invariants():
    rng = np.random.default_rng(16)
    X = _unit(rng, 300, 8)
    C = _unit(rng, 10, 8)
    for _ in range(30):
        codes = oracle.assign_codes(X, C)
        C = oracle.kmeans_update(X, codes, C)
    codes = oracle.assign_codes(X, C)
    for c in range(10):
        mem = X[codes == c]
        if len(mem):
            m = mem.sum(0)
            np.testing.assert_allclose(C[c], m / np.linalg.norm(m), atol=1e-9)
    sims = X @ C.T
    assert np.all(sims[np.arange(300), codes] >= sims.max(1) - 1e-15)


def test_kmeans_update_hand_examples():
    """One Lloyd update on hand-computable inputs (Sec. 4.1.1 stage-1 k-means):
    a centroid with members becomes the unit mean of its members, a centroid with
    no member keeps its value, and so does one whose members sum to zero."""
    X = np.array([[3.0, 0.0, 0.0], [0.0, 4.0, 0.0], [2.0, 0.0, 0.0], [-2.0, 0.0, 0.0]])
    C0 = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    # centroid 0 <- rows 0, 1 (sum (3, 4, 0)); centroid 1 <- rows 2, 3 (sum 0);
    # centroid 2 <- nothing
    C = oracle.kmeans_update(X, np.array([0, 0, 1, 1]), C0)
    np.testing.assert_array_equal(C[0], [0.6, 0.8, 0.0])
    np.testing.assert_array_equal(C[1], C0[1])
    np.testing.assert_array_equal(C[2], C0[2])
    # three points, two centroids, one of them empty: the means of 2 and 1 rows
    X = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 2.0]])
    C = oracle.kmeans_update(X, np.array([1, 1, 1]), np.array([[0.0, -1.0], [1.0, 0.0]]))
    np.testing.assert_array_equal(C[0], [0.0, -1.0])
    np.testing.assert_allclose(C[1], np.array([1.0, 3.0]) / np.sqrt(10.0), rtol=0, atol=1e-15)
    # the update does not depend on the order of the rows
    perm = np.array([2, 0, 1])
    np.testing.assert_array_equal(oracle.kmeans_update(X[perm], np.array([0, 1, 1]), C),
                                  oracle.kmeans_update(X, np.array([1, 1, 0]), C))


def test_synthetic_generators_shapes_and_norms():
    w = synth.exact_fp32(n_sets=100, n_queries=3)
    L = w.docs.lengths()
    assert L.min() >= 16 and L.max() <= 64 and len(L) == 100
    norms = torch.linalg.vector_norm(w.docs.vecs.double(), dim=1)
    assert torch.allclose(norms, torch.ones_like(norms), atol=1e-6)
    lens = synth.lengths_lognormal(200000, 70.0, 0.5, 20, 180, 1)
    assert lens.min() >= 20 and lens.max() <= 180 and 65 < lens.mean() < 72
    co, ci = synth.candidate_lists(20, 1000, 64, 128, 0.3, 50, 3)
    for b in range(20):
        row = ci[co[b]:co[b + 1]]
        assert len(set(row.tolist())) == len(row) and 64 <= len(row) <= 128
    w2 = synth.exact_fp32(n_sets=100, n_queries=3)
    assert torch.equal(w.docs.vecs, w2.docs.vecs)


# ---------------------------------------------------------------------------
# Cluster filter (Sec. 4.5.1, Eq. 15): C_query = union of top-t centroids
# ---------------------------------------------------------------------------

def test_cluster_filter_hand_example_and_ties():
    # d = 2: centroids east, north, west; a query vector near east
    C = np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]])
    Q = np.array([[0.9, 0.1]])
    assert oracle.cluster_filter(Q, [0, 1], C, 1)[0].tolist() == [0]
    assert oracle.cluster_filter(Q, [0, 1], C, 2)[0].tolist() == [0, 1]
    # equal inner products with east and north: the lower index wins
    Qt = np.array([[1.0, 1.0]]) / np.sqrt(2.0)
    assert oracle.cluster_filter(Qt, [0, 1], C, 1)[0].tolist() == [0]
    # two query vectors: the union of their choices, sorted
    Q2 = np.array([[0.9, 0.1], [-0.8, 0.3]])
    assert oracle.cluster_filter(Q2, [0, 2], C, 1)[0].tolist() == [0, 2]


def test_cluster_filter_t_equal_k2_selects_every_centroid():
    rng = np.random.default_rng(21)
    C = _unit(rng, 37, 16)
    Q = _unit(rng, 9, 16)
    out = oracle.cluster_filter(Q, [0, 4, 9], C, 37)
    for o in out:
        assert o.tolist() == list(range(37))


def test_cluster_filter_own_rows_are_the_top_1():
    # with the query vectors themselves among the (unit) centroids, each query
    # vector's inner product 1 with its own copy is the unique maximum
    rng = np.random.default_rng(22)
    Q = _unit(rng, 6, 32)
    C = np.concatenate([_unit(rng, 20, 32), Q, _unit(rng, 5, 32)])
    out = oracle.cluster_filter(Q, [0, 3, 6], C, 1)
    assert out[0].tolist() == [20, 21, 22]
    assert out[1].tolist() == [23, 24, 25]


def test_cluster_filter_permutation_equivariant_and_monotone_in_t():
    rng = np.random.default_rng(23)
    C = _unit(rng, 50, 16)
    Q = _unit(rng, 12, 16)
    qo = [0, 5, 12]
    perm = rng.permutation(50)
    inv = np.argsort(perm)
    prev = [set() for _ in qo[1:]]
    for t in range(1, 7):
        base = oracle.cluster_filter(Q, qo, C, t)
        permuted = oracle.cluster_filter(Q, qo, C[perm], t)
        for b in range(len(base)):
            # centroid i of the permuted matrix is centroid perm[i] of the original
            assert sorted(perm[permuted[b]].tolist()) == base[b].tolist()
            assert prev[b] <= set(base[b].tolist())
            prev[b] = set(base[b].tolist())
    assert inv[perm[3]] == 3


# ---------------------------------------------------------------------------
# Multi-entry points (Sec. 4.5.2, Algorithm 5): members per cluster, the draw
# ---------------------------------------------------------------------------

def test_splitmix64_reference_outputs():
    # the generator's published first outputs from state 0
    st, out = 0, []
    for _ in range(3):
        st, o = oracle.splitmix64_next(st)
        out.append(o)
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_cluster_members_hand_example():
    # sets: 0 = vectors 0..2, 1 = vectors 3..4, 2 = vector 5; index codes per vector
    off = np.array([0, 3, 5, 6])
    codes = np.array([2, 0, 2, 2, 3, 0])
    m = oracle.cluster_members(codes, off, 5)
    assert [x.tolist() for x in m] == [[0, 2], [], [0, 1], [1], []]


def test_entry_points_single_member_empty_cluster_and_membership():
    members = [np.array([7]), np.array([], dtype=np.int64), np.array([1, 4, 9, 12])]
    e = oracle.entry_points([np.array([0, 1, 2]), np.array([2])], members, seed=11)
    assert e[0][0] == 7 and e[0][1] == -1
    assert e[0][2] in (1, 4, 9, 12) and e[1][0] in (1, 4, 9, 12)
    # the draw does not depend on the order the members are listed in
    shuffled = [members[0], members[1], np.array([12, 4, 1, 9])]
    assert [x.tolist() for x in oracle.entry_points([np.array([0, 1, 2]), np.array([2])], shuffled, 11)] == \
        [x.tolist() for x in e]


def test_entry_points_draw_is_uniform_over_members():
    members = [np.array([3, 5, 8, 13])]
    picks = [oracle.entry_points([np.array([0])] * 1, members, seed)[0][0] for seed in range(4000)]
    counts = np.array([picks.count(s) for s in (3, 5, 8, 13)])
    # 4000 draws over 4 members: each count within 5 sigma of 1000
    assert np.all(np.abs(counts - 1000) < 5 * np.sqrt(4000 * 0.25 * 0.75)), counts


# ---------------------------------------------------------------------------
# Cluster-guided beam search (Algorithm 5), in rounds
# ---------------------------------------------------------------------------

def _chain(n, extra=()):
    """Bidirectional path graph 0 - 1 - ... - n-1 (plus extra undirected edges) as CSR."""
    nb = [[] for _ in range(n)]
    for i in range(n - 1):
        nb[i].append(i + 1)
        nb[i + 1].append(i)
    for a, b in extra:
        nb[a].append(b)
        nb[b].append(a)
    off = np.concatenate([[0], np.cumsum([len(x) for x in nb])])
    return off, np.array([v for x in nb for v in sorted(x)], dtype=np.int64)


def test_beam_search_walks_a_path_and_keeps_the_best_ef():
    off, nbrs = _chain(10)
    clusters = [{0}] * 10
    R, rounds = oracle.beam_search(lambda s: float(s), off, nbrs, clusters, [0], [0], ef=3)
    assert R == [(9.0, 9), (8.0, 8), (7.0, 7)]
    assert rounds == 10   # one node popped per round, the last pop adds nothing


def test_beam_search_cluster_filter_stops_the_walk():
    off, nbrs = _chain(10)
    clusters = [{0}] * 10
    clusters[5] = {1}     # not in C_query
    R, _ = oracle.beam_search(lambda s: float(s), off, nbrs, clusters, [0], [0], ef=3)
    assert R == [(4.0, 4), (3.0, 3), (2.0, 2)]


def test_beam_search_prunes_a_path_below_tau():
    # two components: 0..4 scoring 10..14, 5..9 scoring 0..4; entries in both
    off, nbrs = _chain(10)
    off2, nbrs2 = [], []
    cut = [[j for j in nbrs[off[i]:off[i + 1]] if (j < 5) == (i < 5)] for i in range(10)]
    off2 = np.concatenate([[0], np.cumsum([len(x) for x in cut])])
    nbrs2 = np.array([v for x in cut for v in x], dtype=np.int64)
    score = {i: (10.0 + i if i < 5 else float(i - 5)) for i in range(10)}
    seen = []

    def sc(s):
        seen.append(s)
        return score[s]

    R, rounds = oracle.beam_search(sc, off2, nbrs2, [{0}] * 10, [0], [0, 5], ef=3)
    assert R == [(14.0, 4), (13.0, 3), (12.0, 2)]
    assert rounds == 5
    # the second path is cut after two expansions: sets 8 and 9 are never scored
    assert 8 not in seen and 9 not in seen and 7 in seen


def test_beam_search_complete_graph_finds_exact_top_ef():
    n = 12
    off = np.arange(0, n * (n - 1) + 1, n - 1)
    nbrs = np.array([j for i in range(n) for j in range(n) if j != i])
    rng = np.random.default_rng(4)
    vals = rng.permutation(n).astype(float)
    R, _ = oracle.beam_search(lambda s: vals[s], off, nbrs, [{2}] * n, [2, 7], [3], ef=5)
    want = sorted(((vals[i], i) for i in range(n)), key=lambda x: (-x[0], x[1]))[:5]
    assert R == want


def test_lazy_deletion_topk_and_beam_search():
    # top-k never returns a deleted set
    s = np.array([0.9, 0.8, 0.95, 0.1])
    ids, _ = oracle.topk(s, 2, exclude={2})
    assert ids.tolist() == [0, 1]
    # a deleted set on the path is still traversed but never placed in R
    off, nbrs = _chain(10)
    R, _ = oracle.beam_search(lambda x: float(x), off, nbrs, [{0}] * 10, [0], [0], ef=3, dead={8})
    assert R == [(9.0, 9), (7.0, 7), (6.0, 6)]
