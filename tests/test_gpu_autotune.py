"""Autotuner: the chosen schedule is one of the candidates, results do not
depend on it (bit-identical scores), and the JSON cache is written and hit."""
import json
import os

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


def test_autotune_score_all_bit_identical_and_cached(gem, tmp_path):
    w = synth.exact_fp32(n_sets=3000, n_queries=40)
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("bf16", "fp8", "fp8_set"))
    ws = gem.Workspace(store, max_queries=64, max_q_rows=64 * 32, max_q_len=32)
    q, qo = w.queries.vecs.cuda(), torch.from_numpy(w.queries.offsets).cuda()
    cache = str(tmp_path / "tune.json")
    for compute in ("bf16", "fp8", "fp8_set"):
        gem.set_schedule(ws, 2, 1 << 16)
        ref = gem.score_all(store, ws, q, qo, compute).clone()
        ch = gem.autotune_score_all(store, ws, q, qo, compute, cache_path=cache)
        assert ch["m_tiles"] in (1, 2, 4) and ch["chunk_rows"] in (1 << 14, 1 << 16, 1 << 18)
        assert not ch["from_cache"] and ch["ms"] > 0
        assert torch.equal(gem.score_all(store, ws, q, qo, compute), ref)
        again = gem.autotune_score_all(store, ws, q, qo, compute, cache_path=cache)
        assert again["from_cache"] and again["m_tiles"] == ch["m_tiles"]
    entries = json.load(open(cache))["entries"]
    assert len(entries) == 3 and all(k.startswith("score_all|") for k in entries)


def test_autotune_batch_choice_bit_matches(gem, tmp_path):
    seed = 1238
    cents = synth.centres(128, seed)
    docs = synth.vector_sets(synth.lengths_lognormal(800, 70.0, 0.5, 20, 180, seed), cents, seed)
    store = gem.Store(docs.vecs.cuda(), docs.offsets, keep=("f32",))
    qs, co, ci = synth.beam_batch(docs, cents, seed=seed, n_queries=64, len_lo=16, len_hi=64, pool_size=50)
    args = (qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda(), torch.from_numpy(co).cuda(),
            torch.from_numpy(ci).cuda())
    ch = gem.autotune_batch(store, *args, mode="f32", max_q_len=64, cache_path=str(tmp_path / "b.json"))
    assert ch["seg"] in (8, 16, 32, 64) and ch["ctas_per_sm"] in (0, 1, 2)
    outs = []
    for seg, ctas in ((ch["seg"], ch["ctas_per_sm"]), (8, 1)):
        bt = gem.Batch(store, "f32", max_queries=64, max_q_rows=64 * 64, max_q_len=64, max_cands=64 * 64,
                       seg=seg, ctas_per_sm=ctas)
        outs.append(bt.run(*args).clone())
        assert bt.status() == 0
        bt.close()
    assert torch.equal(outs[0], outs[1])
    assert gem.autotune_batch(store, *args, mode="f32", max_q_len=64,
                              cache_path=str(tmp_path / "b.json"))["from_cache"]


@pytest.mark.parametrize("qlens", ["32", "mixed"])
def test_every_schedule_bit_identical(gem, qlens):
    """The tensor-core schedules (resident query rows, query rows in tensor
    memory or shared memory, epilogue sets, MMA issuers, chunk size) only
    change the launch shape.  "mixed": queries of 1..100 rows, so slots of every
    size and up to four passes that add onto the previous pass's scores."""
    w = synth.exact_fp32(n_sets=2500, n_queries=37)
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("bf16", "fp8", "fp8_set"))
    if qlens == "mixed":
        lens = np.random.default_rng(3).integers(1, 101, size=37)
        qs = synth.vector_sets(lens, synth.centres(64, 1235), 5150)
        q, qo = qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda()
        ws = gem.Workspace(store, max_queries=64, max_q_rows=int(lens.sum()), max_q_len=128)
    else:
        q, qo = w.queries.vecs.cuda(), torch.from_numpy(w.queries.offsets).cuda()
        ws = gem.Workspace(store, max_queries=64, max_q_rows=64 * 32, max_q_len=32)
    for compute in ("bf16", "fp8", "fp8_set"):
        outs = []
        for mt, var, cr in ((2, "two_sets", 1 << 16), (2, "plain", 1 << 16), (2, "a_tmem", 1 << 16),
                            (1, "two_sets", 1 << 16), (4, "plain", 1 << 14), (1, "plain", 1 << 18),
                            (2, "a_tmem", 1 << 14), (2, "two_sets", 1 << 14)):
            gem.set_schedule(ws, mt, cr, variant=var)
            outs.append(gem.score_all(store, ws, q, qo, compute).clone())
            assert ws.status() == 0
        for o in outs[1:]:
            assert torch.equal(o, outs[0])
        if qlens == "mixed" and compute == "bf16":
            Sq = oracle.score_all(oracle.bf16_round(qs.vecs.numpy()), qs.offsets,
                                  oracle.bf16_round(w.docs.vecs.numpy()), w.docs.offsets)
            assert np.all(np.abs(outs[0].cpu().numpy() - Sq) <= 2e-4 * lens[:, None])
        if qlens == "mixed" and compute == "fp8_set":
            # multi-pass queries with the per-set scale applied at each pass's set end
            c8, s8 = oracle.fp8_e4m3_quantize_sets(w.docs.vecs.numpy(), w.docs.offsets)
            cq, sq = oracle.fp8_e4m3_quantize(qs.vecs.numpy())
            Sq = oracle.score_all(cq * sq[:, None].astype(np.float64), qs.offsets,
                                  c8 * np.repeat(s8.astype(np.float64), np.diff(w.docs.offsets))[:, None],
                                  w.docs.offsets)
            assert np.all(np.abs(outs[0].cpu().numpy() - Sq) <= 2e-4 * lens[:, None])
    with pytest.raises(Exception):
        gem.set_schedule(ws, 4, 1 << 16, variant="a_tmem")
