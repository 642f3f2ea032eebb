"""E4M3 storage with one power-of-two scale per stored set (GEM_KEEP_FP8_SET,
GEM_FP8_E4M3_SET): the device copy equals the oracle's per-set quantisation bit
for bit, and the tensor-core scores equal the FP64 Chamfer score (Eq. 1) of the
oracle's dequantised inputs up to FP32 accumulation.

Tolerance: the stored side's scale is exact and common to the set, so it leaves
the inner max unchanged (max_j <q, s c_j> = s max_j <q, c_j>); each query row
carries its per-row E4M3 scale as in GEM_FP8_E4M3.  What remains is FP32
accumulation of 128 products per dot and of m_q maxima, bounded by 2e-4 per
query row for unit-scale rows, the bound the per-vector FP8 path uses."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gem():
    import paper_2603_20336_b300 as g
    return g


def _padded_source_rows(off):
    lens = np.diff(off)
    plens = (lens + 7) // 8 * 8
    src = [off[d] + np.minimum(np.arange(plens[d]), lens[d] - 1) for d in range(len(lens))]
    return np.concatenate([[0], np.cumsum(plens)]), np.concatenate(src)


@pytest.fixture(scope="module")
def cfg(gem):
    w = synth.exact_fp32()
    # a few sets scaled far from unit norm so the scales spread over many exponents
    X = w.docs.vecs.numpy().copy()
    off = w.docs.offsets
    for d, f in [(0, 1e-30), (3, 1e20), (5, 3.0), (7, 0.001)]:
        X[off[d]:off[d + 1]] *= np.float32(f)
    docs = torch.from_numpy(X)
    store = gem.Store(docs.cuda(), off, keep=("f32", "fp8_set"))
    ws = gem.Workspace(store, max_queries=64, max_q_rows=4096, max_q_len=128, max_cands=64 * 256, max_k=256)
    yield dict(w=w, X=X, off=off, store=store, ws=ws)
    ws.close()
    store.close()


def test_fp8_set_copy_matches_oracle(gem, cfg):
    X, off, store = cfg["X"], cfg["off"], cfg["store"]
    codes, scale = oracle.fp8_e4m3_quantize_sets(X, off)
    np.testing.assert_array_equal(store.export("set_scale").cpu().numpy(), scale)
    pad_off, src = _padded_source_rows(off)
    got = store.export("fp8_set").cpu().view(torch.float8_e4m3fn).float().numpy().astype(np.float64)
    np.testing.assert_array_equal(got, codes[src])


def _fp8_rows(X):
    c, s = oracle.fp8_e4m3_quantize(np.asarray(X, np.float32))
    return c * s[:, None].astype(np.float64)


@pytest.mark.parametrize("lens", [[32] * 10, [1, 5, 17, 32, 33, 64, 100, 7, 128]])
def test_score_all_fp8_set_matches_oracle_on_dequantised_inputs(gem, cfg, lens):
    X, off = cfg["X"], cfg["off"]
    lens = np.array(lens)
    qs = synth.vector_sets(lens, synth.centres(64, 1235), 778)
    S = gem.score_all(cfg["store"], cfg["ws"], qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda(),
                      "fp8_set").cpu().numpy().astype(np.float64)
    assert cfg["ws"].status() == 0
    codes, scale = oracle.fp8_e4m3_quantize_sets(X, off)
    deq = codes * np.repeat(scale.astype(np.float64), np.diff(off))[:, None]
    Sq = oracle.score_all(_fp8_rows(qs.vecs.numpy()), qs.offsets, deq, off)
    # error relative to the set's scale: the per-set tolerance is 2e-4 * m_q for
    # unit-scale rows, times the largest stored magnitude of that set
    smax = np.array([np.abs(X[off[d]:off[d + 1]]).max() for d in range(len(off) - 1)])
    tol = 2e-4 * lens[:, None] * np.maximum(smax, 1.0)[None, :]
    assert np.all(np.abs(S - Sq) <= tol), np.abs(S - Sq).max()


def test_search_fp8_set_first_pass_then_exact_rerank(gem, cfg):
    """Search with the per-set-scale first pass: the rerank makes the final
    scores exact FP32 CH, equal to gem_search with the FP32 first pass wherever
    both pools hold the true top k."""
    w = cfg["w"]
    q = w.queries.vecs.cuda()
    qo = torch.from_numpy(w.queries.offsets).cuda()
    k = 10
    i8, s8 = gem.search(cfg["store"], cfg["ws"], q, qo, "fp8_set", rerank_depth=100, k=k)
    i32, s32 = gem.search(cfg["store"], cfg["ws"], q, qo, "f32", rerank_depth=100, k=k)
    assert cfg["ws"].status() == 0
    assert torch.equal(i8, i32)
    assert torch.equal(s8, s32)


def test_fp8_set_needs_its_copy(gem, cfg):
    st = gem.Store(torch.from_numpy(cfg["X"]).cuda(), cfg["off"], keep=("f32",))
    ws = gem.Workspace(st, max_queries=4, max_q_rows=128, max_q_len=32)
    try:
        w = cfg["w"]
        with pytest.raises(gem.GemError):
            gem.score_all(st, ws, w.queries.vecs[:32].cuda(), torch.tensor([0, 32]).cuda(), "fp8_set")
    finally:
        ws.close()
        st.close()
