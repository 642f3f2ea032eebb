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


def test_full_size_gradient_matches_oracle(gem):
    """256 queries x 32 vectors, 64 own sets each (lengths 32..256), BF16 forward,
    FP32 gradients; compared with the oracle on the rows whose argmax agrees."""
    w = synth.contrastive_batch(device="cuda")
    B, per_q = 256, 64
    po, pid = _pairs(B, per_q)
    q = w.queries.vecs.clone().requires_grad_(True)
    D = w.docs.vecs.clone().requires_grad_(True)
    qo, do = torch.from_numpy(w.queries.offsets).cuda(), torch.from_numpy(w.docs.offsets).cuda()
    s = gem.MaxSimFn.apply(q, D, qo, do, po.cuda(), pid.cuda(), "bf16")
    loss = torch.nn.functional.cross_entropy(s.view(B, per_q) / TAU, torch.zeros(B, dtype=torch.int64, device="cuda"))
    loss.backward()
    _, am = gem.maxsim_fwd(w.queries.vecs, qo, w.docs.vecs, do, po.cuda(), pid.cuda(), "bf16")
    am = am.cpu().numpy()
    # sampled outputs: 16 queries with all of their 64 sets
    Qn = w.queries.vecs.cpu().numpy().astype(np.float64)
    Dn = w.docs.vecs.cpu().numpy().astype(np.float64)
    g = oracle.contrastive_dscores(s.detach().cpu().numpy().astype(np.float64).reshape(B, per_q), TAU)
    gq_gpu = q.grad.cpu().numpy()
    gd_gpu = D.grad.cpu().numpy()
    Qr, Dr = oracle.bf16_round(Qn.astype(np.float32)), oracle.bf16_round(Dn.astype(np.float32))
    n_rows = n_agree = 0
    for b in range(0, B, 16):
        qr = slice(w.queries.offsets[b], w.queries.offsets[b + 1])
        gq = np.zeros((32, 128))
        rows_ok = np.ones(32, bool)
        for n in range(per_q):
            t = b * per_q + n
            dr = slice(w.docs.offsets[t], w.docs.offsets[t + 1])
            # j* decided on the bf16-rounded inputs, as the BF16 forward decides it
            dq, dp, js = oracle.maxsim_grad(Qn[qr], Dn[dr], decide=(Qr[qr], Dr[dr]))
            same = js == am[t, :32]
            rows_ok &= same
            gq += g[b, n] * dq
            if same.all():
                np.testing.assert_allclose(gd_gpu[dr], g[b, n] * dp, atol=1e-5 * abs(g[b, n]) + 1e-7)
        n_rows += 32
        n_agree += int(rows_ok.sum())
        np.testing.assert_allclose(gq_gpu[qr][rows_ok], gq[rows_ok], rtol=1e-4, atol=1e-6)
    assert n_agree >= 0.97 * n_rows
