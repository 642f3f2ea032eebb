"""Full-size parity of the multi-modal page configuration: 50,000 sets of exactly
1,024 vectors (51.2M vectors, 1,024-centre mixture), 500 queries of 16..32
vectors, the store kept in FP32, BF16 and E4M3 with per-vector scales.

What the FP64 oracle can compute one by one is checked on sampled (query, set)
pairs, per dtype:
  FP32 exhaustive: |s - s64| <= 1e-5 * sum_i |max_j <q_i, p_j>|
  BF16 exhaustive: |s - s64| <= 2e-2 (storage rounding of unit vectors)
  E4M3 exhaustive: against the oracle on the same E4M3-rounded inputs,
                   |s - s64q| <= 2e-4 * m_q (FP32 accumulation and the scales)
What holds at any size is checked on every query: the BF16 and E4M3 pipelines
(top-2,000, exact FP32 rerank, top-100) return the exact FP32 exhaustive top-100,
except for ids whose FP32 scores tie within 1e-6 at the cut.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def gem():
    import paper_2603_20336_b300 as g
    return g


@pytest.fixture(scope="module")
def pages(gem):
    w = synth.multimodal_pages(device="cuda")
    store = gem.Store(w.docs.vecs, w.docs.offsets, keep=("f32", "bf16", "fp8"))
    q = w.queries.vecs
    qo = torch.from_numpy(w.queries.offsets).cuda()
    B = len(w.queries.offsets) - 1
    ws = gem.Workspace(store, max_queries=B, max_q_rows=q.shape[0], max_q_len=32, max_cands=B * 2000,
                       max_k=2000)
    yield dict(w=w, store=store, q=q, qo=qo, ws=ws, B=B)
    ws.close()
    store.close()


def _dequant_e4m3(X):
    codes, scale = oracle.fp8_e4m3_quantize(np.asarray(X, np.float32))
    return codes * scale[:, None].astype(np.float64)


def test_pages_50k_sampled_pairs_per_dtype(gem, pages):
    w, store, ws = pages["w"], pages["store"], pages["ws"]
    S = {dt: gem.score_all(store, ws, pages["q"], pages["qo"], dt) for dt in ("f32", "bf16", "fp8")}
    assert ws.status() == 0
    rng = np.random.default_rng(2024)
    qoff, doff = w.queries.offsets, w.docs.offsets
    errs = {"f32": 0.0, "bf16": 0.0, "fp8_vs_fp32_inputs": 0.0, "fp8_vs_e4m3_inputs": 0.0}
    for _ in range(48):
        b = int(rng.integers(pages["B"]))
        n = int(rng.integers(len(doff) - 1))
        Q = w.queries.vecs[qoff[b]:qoff[b + 1]].cpu().numpy()
        P = w.docs.vecs[doff[n]:doff[n + 1]].cpu().numpy()
        s64, l1 = oracle.score_all(Q, [0, len(Q)], P, [0, len(P)], with_l1=True)
        s64q = oracle.score_all(_dequant_e4m3(Q), [0, len(Q)], _dequant_e4m3(P), [0, len(P)])
        got = {dt: float(S[dt][b, n]) for dt in S}
        e32 = abs(got["f32"] - s64[0, 0])
        assert e32 <= 1e-5 * l1[0, 0], (b, n, e32)
        eb = abs(got["bf16"] - s64[0, 0])
        assert eb <= 2e-2, (b, n, eb)
        e8q = abs(got["fp8"] - s64q[0, 0])
        assert e8q <= 2e-4 * len(Q), (b, n, e8q)
        errs["f32"] = max(errs["f32"], e32)
        errs["bf16"] = max(errs["bf16"], eb)
        errs["fp8_vs_e4m3_inputs"] = max(errs["fp8_vs_e4m3_inputs"], e8q)
        errs["fp8_vs_fp32_inputs"] = max(errs["fp8_vs_fp32_inputs"], abs(got["fp8"] - s64[0, 0]))
    print("pages-50k max |error| vs FP64 per dtype:", errs)


@pytest.mark.parametrize("compute", ["bf16", "fp8"])
def test_pages_50k_rerank_pipeline_matches_exact_fp32_top100(gem, pages, compute):
    store, ws = pages["store"], pages["ws"]
    S32 = gem.score_all(store, ws, pages["q"], pages["qo"], "f32")
    exact_s, exact_i = torch.topk(S32, 100, dim=1)
    ids, sc = gem.search(store, ws, pages["q"], pages["qo"], compute, rerank_depth=2000, k=100)
    assert ws.status() == 0
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    exact_i, exact_s, S32 = exact_i.cpu().numpy(), exact_s.cpu().numpy(), S32.cpu().numpy()
    hits = 0
    for b in range(pages["B"]):
        got, want = set(ids[b].tolist()), set(exact_i[b].tolist())
        hits += len(got & want)
        cut = exact_s[b, -1]
        for x in got ^ want:
            assert abs(S32[b, x] - cut) <= 1e-6 * max(1.0, abs(cut)), (b, x)
        # the reranked scores are the exact FP32 scores of those ids
        np.testing.assert_array_equal(sc[b], S32[b, ids[b]])
    recall = hits / (100 * pages["B"])
    print(f"pages-50k {compute} + FP32 rerank recall@100 vs exact FP32: {recall:.4f}")
    assert recall >= 0.99
