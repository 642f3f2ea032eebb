"""MaxSim forward (argmax side output) and hand-written backward against the
FP64 oracle: gradients of an in-batch contrastive loss through Eq. 1, a
finite-difference check on a 4 x 4 instance, and the full-size configuration
(256 queries x 64 own sets, sampled outputs)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
TAU = 0.05


@pytest.fixture(scope="module")
def gem():
    import paper_2603_20336_b300 as g
    return g


def _pairs(n_q, per_q):
    po = torch.arange(n_q + 1, dtype=torch.int64) * per_q
    pid = torch.arange(n_q * per_q, dtype=torch.int64)
    return po, pid


def _oracle_grads(Q, qo, D, do, per_q, S, tau, jstar_gpu=None):
    """Chain rule through the contrastive loss with the oracle's per-pair MaxSim gradient."""
    B = len(qo) - 1
    g = oracle.contrastive_dscores(S.reshape(B, per_q), tau).reshape(-1)
    gq = np.zeros_like(Q, dtype=np.float64)
    gd = np.zeros_like(D, dtype=np.float64)
    agree = []
    for b in range(B):
        for n in range(per_q):
            t = b * per_q + n
            d = t
            dq, dp, js = oracle.maxsim_grad(Q[qo[b]:qo[b + 1]], D[do[d]:do[d + 1]])
            if jstar_gpu is not None:
                agree.append(np.array_equal(js, jstar_gpu[t, :qo[b + 1] - qo[b]]))
            gq[qo[b]:qo[b + 1]] += g[t] * dq
            gd[do[d]:do[d + 1]] += g[t] * dp
    return gq, gd, g, agree


def test_forward_scores_and_argmax_match_oracle(gem):
    w = synth.contrastive_batch(n_queries=6, docs_per_query=8, len_lo=4, len_hi=40)
    po, pid = _pairs(6, 8)
    q, qo = w.queries.vecs.cuda(), torch.from_numpy(w.queries.offsets).cuda()
    D, do = w.docs.vecs.cuda(), torch.from_numpy(w.docs.offsets).cuda()
    for compute in ("f32", "bf16"):
        s, am = gem.maxsim_fwd(q, qo, D, do, po.cuda(), pid.cuda(), compute)
        s, am = s.cpu().numpy(), am.cpu().numpy()
        Qn, Dn = w.queries.vecs.numpy(), w.docs.vecs.numpy()
        if compute == "bf16":
            Qn, Dn = oracle.bf16_round(Qn), oracle.bf16_round(Dn)
        for t in range(48):
            b = t // 8
            Qb = Qn[w.queries.offsets[b]:w.queries.offsets[b + 1]].astype(np.float64)
            Pd = Dn[w.docs.offsets[t]:w.docs.offsets[t + 1]].astype(np.float64)
            sims = Qb @ Pd.T
            assert abs(s[t] - sims.max(1).sum()) <= 1e-5 * np.abs(sims.max(1)).sum()
            srt = np.sort(sims, axis=1)
            clear = (srt[:, -1] - srt[:, -2] > 2e-5) if sims.shape[1] > 1 else np.ones(len(Qb), bool)
            np.testing.assert_array_equal(am[t, :len(Qb)][clear], np.argmax(sims, axis=1)[clear])


def test_tensor_core_forward_agrees_with_simt_forward(gem):
    """GEM_BF16 with max_q_len <= 128 runs on the tensor cores, a larger
    max_q_len on the SIMT kernel; both decide on the same bf16-rounded inputs.
    Queries of 1..128 vectors, sets of 1..700 vectors (several 256-row tiles),
    ragged pair lists (a query with none), an out-of-range id: argmax equal
    wherever the FP64 top-2 margin exceeds the FP32 dot bound, scores within
    1e-5 of the L1 of their terms, the bad id scored NaN with GEM_ERR_BOUNDS."""
    rng = np.random.default_rng(8)
    qlens = np.array([1, 32, 128, 77, 5, 64])
    dlens = rng.integers(1, 700, size=40)
    dlens[:4] = [1, 256, 257, 700]
    cents = synth.centres(64, 4)
    qs = synth.vector_sets(qlens, cents, 31)
    ds = synth.vector_sets(dlens, cents, 32)
    counts = np.array([7, 0, 12, 9, 3, 10])
    po = torch.from_numpy(np.concatenate([[0], np.cumsum(counts)]).astype(np.int64))
    pid = torch.from_numpy(rng.integers(0, 40, size=int(counts.sum())).astype(np.int64))
    pid[5] = 40                                            # out of range
    st = gem.Store(ds.vecs.cuda(), ds.offsets, keep=("f32",))
    ws = gem.Workspace(st, max_queries=1, max_q_rows=1)     # for its status word
    q, qo = qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda()
    D, do = ds.vecs.cuda(), torch.from_numpy(ds.offsets).cuda()
    s_tc, am_tc = gem.maxsim_fwd(q, qo, D, do, po.cuda(), pid.cuda(), "bf16", max_q_len=128, ws=ws)
    assert ws.status() == 7
    s_sm, am_sm = gem.maxsim_fwd(q, qo, D, do, po.cuda(), pid.cuda(), "bf16", max_q_len=160, ws=ws)
    assert ws.status() == 7
    s_tc, am_tc, s_sm, am_sm = s_tc.cpu().numpy(), am_tc.cpu().numpy(), s_sm.cpu().numpy(), am_sm.cpu().numpy()
    assert np.isnan(s_tc[5]) and np.isnan(s_sm[5])
    Qr = oracle.bf16_round(qs.vecs.numpy()).astype(np.float64)
    Dr = oracle.bf16_round(ds.vecs.numpy()).astype(np.float64)
    band = 2 * 128 * 2.0 ** -24 * (1 + 2.0 ** -8) ** 2
    for b in range(len(qlens)):
        for t in range(int(po[b]), int(po[b + 1])):
            d = int(pid[t])
            if d >= 40:
                continue
            sims = Qr[qs.offsets[b]:qs.offsets[b + 1]] @ Dr[ds.offsets[d]:ds.offsets[d + 1]].T
            m = qlens[b]
            srt = np.sort(sims, axis=1)
            clear = (srt[:, -1] - srt[:, -2] > band) if sims.shape[1] > 1 else np.ones(m, bool)
            want = np.argmax(sims, axis=1)
            np.testing.assert_array_equal(am_tc[t, :m][clear], want[clear])
            np.testing.assert_array_equal(am_sm[t, :m][clear], want[clear])
            top = sims.max(axis=1)
            assert np.all(sims[np.arange(m), am_tc[t, :m]] >= top - band)
            l1 = np.abs(top).sum()
            assert abs(s_tc[t] - top.sum()) <= 1e-5 * l1 and abs(s_sm[t] - top.sum()) <= 1e-5 * l1


def test_finite_differences_4x4(gem):
    """4 queries x 4 sets, FP32 forward; margins kept away from argmax switches."""
    rng = np.random.default_rng(21)
    for _ in range(50):
        w = synth.contrastive_batch(seed=int(rng.integers(1 << 30)), n_queries=4, docs_per_query=4, m_q=3,
                                    len_lo=2, len_hi=5)
        ok = True
        for t in range(16):
            b = t // 4
            sims = (w.queries.vecs[w.queries.offsets[b]:w.queries.offsets[b + 1]].double()
                    @ w.docs.vecs[w.docs.offsets[t]:w.docs.offsets[t + 1]].double().T).numpy()
            srt = np.sort(sims, axis=1)
            ok &= bool(np.all(srt[:, -1] - srt[:, -2] > 1e-3))
        if ok:
            break
    assert ok
    po, pid = _pairs(4, 4)
    q = w.queries.vecs.cuda().requires_grad_(True)
    D = w.docs.vecs.cuda().requires_grad_(True)
    qo, do = torch.from_numpy(w.queries.offsets).cuda(), torch.from_numpy(w.docs.offsets).cuda()
    s = gem.MaxSimFn.apply(q, D, qo, do, po.cuda(), pid.cuda(), "f32")
    loss = torch.nn.functional.cross_entropy(s.view(4, 4) / TAU, torch.zeros(4, dtype=torch.int64, device="cuda"))
    loss.backward()
    Qn, Dn = w.queries.vecs.numpy().astype(np.float64), w.docs.vecs.numpy().astype(np.float64)

    def L(Qx, Dx):
        S = np.array([oracle.chamfer(Qx[w.queries.offsets[t // 4]:w.queries.offsets[t // 4 + 1]],
                                     Dx[w.docs.offsets[t]:w.docs.offsets[t + 1]]) for t in range(16)])
        return oracle.contrastive_loss(S.reshape(4, 4), TAU)

    h = 1e-6
    for (M, G) in ((Qn, q.grad.cpu().numpy()), (Dn, D.grad.cpu().numpy())):
        for idx in [(0, 0), (2, 5), (len(M) - 1, 127), (len(M) // 2, 64)]:
            Mp, Mm = M.copy(), M.copy()
            Mp[idx] += h
            Mm[idx] -= h
            fd = (L(Mp, Dn) - L(Mm, Dn)) / (2 * h) if M is Qn else (L(Qn, Mp) - L(Qn, Mm)) / (2 * h)
            assert G[idx] == pytest.approx(fd, rel=1e-4, abs=1e-6)


# Near-tie band of the argmax decision.  Both sides decide j* on the
# bf16-rounded inputs; the GPU's dots are FP32 sums of exact bf16 products, each
# within 128 * 2^-24 * sum_k |q_k p_k| <= 128 * 2^-24 * (1 + 2^-8)^2 of the FP64
# value, so two candidates whose FP64 dots differ by more than twice that are
# ordered the same way on both sides.
ARGMAX_BAND = 2 * 128 * 2.0 ** -24 * (1 + 2.0 ** -8) ** 2
# Products below FP32's normal range: FP32 atomic adds flush subnormal values to
# zero, so each of at most 64 summed terms may lose up to 2^-126.
FTZ_FLOOR = 64 * 2.0 ** -126


def test_full_size_gradient_matches_oracle(gem):
    """256 queries x 32 vectors, 64 own sets each (lengths 32..256), BF16 forward,
    FP32 gradients, against the oracle on every 4th query with all 64 of its sets.

    Outside the near-tie band the GPU's argmax must equal the oracle's FP64 argmax
    exactly; inside it the GPU's choice must be a valid one (within the band of the
    maximum) and the oracle's gradient takes that choice.  dQ and dP are then
    compared on every row, within 1e-5 of the L1 of the terms each sums."""
    w = synth.contrastive_batch(device="cuda")
    B, per_q = 256, 64
    po, pid = _pairs(B, per_q)
    q = w.queries.vecs.clone().requires_grad_(True)
    D = w.docs.vecs.clone().requires_grad_(True)
    qo, do = torch.from_numpy(w.queries.offsets).cuda(), torch.from_numpy(w.docs.offsets).cuda()
    s = gem.MaxSimFn.apply(q, D, qo, do, po.cuda(), pid.cuda(), "bf16")
    s.retain_grad()
    loss = torch.nn.functional.cross_entropy(s.view(B, per_q) / TAU, torch.zeros(B, dtype=torch.int64, device="cuda"))
    loss.backward()
    _, am = gem.maxsim_fwd(w.queries.vecs, qo, w.docs.vecs, do, po.cuda(), pid.cuda(), "bf16")
    am = am.cpu().numpy()
    Qf = w.queries.vecs.cpu().numpy()
    Df = w.docs.vecs.cpu().numpy()
    Qn, Dn = Qf.astype(np.float64), Df.astype(np.float64)
    Qr, Dr = oracle.bf16_round(Qf).astype(np.float64), oracle.bf16_round(Df).astype(np.float64)
    # dL/dS: torch's cross-entropy in FP32 (not this library's arithmetic) against
    # the oracle's FP64 chain rule.  The logits s / tau reach about 600, where an
    # FP32 ulp is 6e-5, so each softmax entry is off by up to about 1e-4 of itself
    # (probabilities below FP32's range come out as 0)
    g64 = oracle.contrastive_dscores(s.detach().cpu().numpy().astype(np.float64).reshape(B, per_q), TAU)
    g = s.grad.cpu().numpy().astype(np.float64).reshape(B, per_q)
    assert np.all(np.abs(g - g64) <= 1e-4 * np.abs(g64).max(axis=1, keepdims=True))
    # the backward kernel's own parity: the oracle takes the very upstream
    # gradient the kernel received
    gq_gpu = q.grad.cpu().numpy()
    gd_gpu = D.grad.cpu().numpy()
    n_rows = n_band = 0
    for b in range(0, B, 4):
        qr = slice(w.queries.offsets[b], w.queries.offsets[b + 1])
        m_q = qr.stop - qr.start
        gq = np.zeros((m_q, 128))
        gq_l1 = np.zeros((m_q, 128))
        for n in range(per_q):
            t = b * per_q + n
            dr = slice(w.docs.offsets[t], w.docs.offsets[t + 1])
            sims = Qr[qr] @ Dr[dr].T
            js = np.argmax(sims, axis=1)
            top = sims.max(axis=1)
            srt = np.sort(sims, axis=1)
            margin = srt[:, -1] - srt[:, -2] if sims.shape[1] > 1 else np.full(m_q, np.inf)
            mine = am[t, :m_q]
            clear = margin > ARGMAX_BAND
            np.testing.assert_array_equal(mine[clear], js[clear], err_msg=f"pair {t}")
            # inside the band: a valid choice, which the oracle's gradient then takes
            assert np.all((mine >= 0) & (mine < sims.shape[1])), t
            assert np.all(sims[np.arange(m_q), mine] >= top - ARGMAX_BAND), t
            jstar = np.where(clear, js, mine)
            n_rows += m_q
            n_band += int((~clear).sum())
            dq, dp, js_o = oracle.maxsim_grad(Qn[qr], Dn[dr], decide=(Qr[qr], Dr[dr]))
            np.testing.assert_array_equal(js_o, js)
            if not np.array_equal(jstar, js_o):
                # a near tie the GPU resolved the other way: the gradient at its choice
                dq = Dn[dr][jstar]
                dp = np.zeros_like(Dn[dr])
                np.add.at(dp, jstar, Qn[qr])
            dp_l1 = np.zeros_like(dp)
            np.add.at(dp_l1, jstar, np.abs(Qn[qr]))
            gq += g[b, n] * dq
            gq_l1 += abs(g[b, n]) * np.abs(dq)
            err = np.abs(gd_gpu[dr] - g[b, n] * dp)
            assert np.all(err <= 1e-5 * abs(g[b, n]) * dp_l1 + FTZ_FLOOR), (t, err.max())
        err = np.abs(gq_gpu[qr] - gq)
        assert np.all(err <= 1e-5 * gq_l1 + FTZ_FLOOR), (b, err.max())
    assert n_rows == 64 * per_q * 32
    assert n_band <= 0.01 * n_rows, n_band


def test_backward_shared_sets_and_rows_outside_any_set(gem):
    """Sets named by several pairs (atomic adds), by one pair (rows written by
    their owner) and by none; rows before the first set and after the last; an
    invalid pair id; argmax entries outside their set.  Every row of grad_docs is
    overwritten (the buffers start as NaN).  A set named by one pair is checked
    bit for bit against the same FP32 sums taken on the host (each row: the q_i
    with j* = row added in ascending i, times g_t); the rest against FP64."""
    from paper_2603_20336_b300 import _check, _ptr, _stream, lib
    rng = np.random.default_rng(5)
    lens = rng.integers(3, 21, 10)
    off = 7 + np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    n_rows = int(off[-1]) + 13
    D = rng.standard_normal((n_rows, 128)).astype(np.float32)
    qlens = np.array([5, 32, 1, 17])
    qo = np.concatenate([[0], np.cumsum(qlens)]).astype(np.int64)
    Q = rng.standard_normal((int(qo[-1]), 128)).astype(np.float32)
    lists = [[0, 1, 2], [2, 3, 4, 9], [5], [2, 6, 0, -1]]      # set 2 thrice, set 0 twice; 7, 8 unnamed
    po = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.int64)
    pid = np.concatenate(lists).astype(np.int64)
    n_pairs, mq = len(pid), 32
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    qd, qod, Dd, dod, pod, pidd = dev(Q), dev(qo), dev(D), dev(off), dev(po), dev(pid)
    _, am = gem.maxsim_fwd(qd, qod, Dd, dod, pod, pidd, "f32", max_q_len=mq)
    am = am.cpu().numpy().copy()
    am[4, 3] = lens[3]          # pair 4 (query 1, set 3): row 3 points past the set
    am[9, 0] = -1               # pair 9 (query 3, set 6): row 0 points before it
    g = rng.standard_normal(n_pairs).astype(np.float32)
    gq = torch.full((int(qo[-1]), 128), float("nan"), device="cuda")
    gd = torch.full((n_rows, 128), float("nan"), device="cuda")
    amd, gdev = dev(am), dev(g)     # kept alive until the kernels have run
    _check(lib.gem_maxsim_bwd(_ptr(qd), _ptr(qod), len(qlens), _ptr(Dd), _ptr(dod), len(lens), n_rows, _ptr(pod),
                              _ptr(pidd), n_pairs, _ptr(amd), mq, _ptr(gdev), _ptr(gq), _ptr(gd), _stream()))
    gq, gd = gq.cpu().numpy(), gd.cpu().numpy()
    assert not np.isnan(gq).any() and not np.isnan(gd).any()
    assert np.all(gd[:off[0]] == 0) and np.all(gd[off[-1]:] == 0)
    for d in (7, 8):
        assert np.all(gd[off[d]:off[d + 1]] == 0)
    want_q = np.zeros((int(qo[-1]), 128))
    l1_q = np.zeros_like(want_q)
    want_d = np.zeros((n_rows, 128))
    l1_d = np.zeros_like(want_d)
    owners = {}
    for b in range(len(qlens)):
        for t in range(po[b], po[b + 1]):
            d = pid[t]
            if d < 0:
                continue
            owners.setdefault(d, []).append((t, b))
            for i in range(qlens[b]):
                j = am[t, i]
                if not 0 <= j < lens[d]:
                    continue
                want_q[qo[b] + i] += float(g[t]) * D[off[d] + j]
                l1_q[qo[b] + i] += abs(float(g[t]) * D[off[d] + j])
                want_d[off[d] + j] += float(g[t]) * Q[qo[b] + i]
                l1_d[off[d] + j] += abs(float(g[t]) * Q[qo[b] + i])
    assert np.all(np.abs(gq - want_q) <= 1e-5 * l1_q + FTZ_FLOOR)
    assert np.all(np.abs(gd - want_d) <= 1e-5 * l1_d + FTZ_FLOOR)
    for d, ts in owners.items():
        if len(ts) != 1:
            continue
        (t, b), = ts
        exp = np.zeros((lens[d], 128), np.float32)
        for j in range(lens[d]):
            acc = np.zeros(128, np.float32)
            hit = False
            for i in range(qlens[b]):
                if am[t, i] == j:
                    acc = (acc + Q[qo[b] + i]).astype(np.float32)
                    hit = True
            if hit:
                exp[j] = (np.float32(g[t]) * acc).astype(np.float32)
        np.testing.assert_array_equal(gd[off[d]:off[d + 1]], exp, err_msg=f"set {d}")
