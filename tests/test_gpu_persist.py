"""Store persistence: a store saved with gem_store_save and read back with
gem_store_load holds bit-identical arrays (FP32 master, bf16 and E4M3 copies,
scales, offsets, codes, C_quant, C_index, index codes, deletions) and answers a
search and a beam search exactly as the original; files that are not stores,
truncated files and stores without the FP32 copy are refused."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gem():
    import paper_2603_20336_b300 as g
    return g


ARRAYS = ("f32", "bf16", "fp8", "fp8_scale", "offsets", "pad_offsets", "codes", "codebook", "index_codes",
          "index_centroids", "deleted")


def _build(gem):
    w = synth.exact_fp32(n_sets=500, n_queries=5)
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("f32", "bf16", "fp8"))
    gem.set_codebook(store, gem.train_codebook(store, k1=128, iters=3, sample=0, seed=2))
    gem.set_index_centroids(store, gem.kmeans(store.export("codebook"), 12, iters=3, seed=4))
    gem.mark_deleted(store, [3, 17, 250, 499])
    return w, store


def test_save_load_round_trip_is_bit_exact(gem, tmp_path):
    w, a = _build(gem)
    path = tmp_path / "store.gem"
    a.save(path)
    b = gem.Store.load(path, keep=("f32", "bf16", "fp8"))
    assert (b.n_sets, b.n_vecs, b.n_pad_vecs, b.k1, b.k2) == (a.n_sets, a.n_vecs, a.n_pad_vecs, a.k1, a.k2)
    for name in ARRAYS:
        x, y = a.export(name), b.export(name)
        assert torch.equal(x.view(torch.uint8) if x.dtype != torch.uint8 else x,
                           y.view(torch.uint8) if y.dtype != torch.uint8 else y), name
    q, qo = w.queries.vecs.cuda(), torch.from_numpy(w.queries.offsets).cuda()
    res = []
    for s in (a, b):
        ws = gem.Workspace(s, max_queries=5, max_q_rows=int(w.queries.offsets[-1]), max_q_len=32,
                           max_cands=5 * 50, max_k=50)
        ids, sc = gem.search(s, ws, q, qo, "bf16", rerank_depth=50, k=10)
        mask, lst, cnt = gem.cluster_filter(q, qo, s.export("index_centroids"), t=2, max_q_len=32)
        ent = gem.entry_points(s, lst, cnt, seed=7)
        go, gn = synth.random_graph(s.n_sets, 6, 3)
        bi, bs, rounds = gem.beam_search(s, ws, q, qo, torch.from_numpy(go).cuda(), torch.from_numpy(gn).cuda(),
                                         mask, ent, ef=12)
        assert ws.status() == 0
        res.append((ids.cpu(), sc.cpu(), ent.cpu(), bi.cpu(), bs.cpu(), rounds))
        ws.close()
    for x, y in zip(*res):
        assert (x == y) if isinstance(x, int) else torch.equal(x, y)
    assert not set(res[0][0].view(-1).tolist()) & {3, 17, 250, 499}
    # a store loaded with fewer copies still scores its FP32 path
    c = gem.Store.load(path, keep=("f32",))
    assert torch.equal(c.export("f32"), a.export("f32")) and torch.equal(c.export("codes"), a.export("codes"))
    for s in (a, b, c):
        s.close()


def test_load_refuses_bad_files_and_save_needs_fp32(gem, tmp_path):
    w, a = _build(gem)
    good = tmp_path / "good.gem"
    a.save(good)
    raw = good.read_bytes()
    (tmp_path / "short.gem").write_bytes(raw[:-20])
    (tmp_path / "long.gem").write_bytes(raw + b"x")
    (tmp_path / "magic.gem").write_bytes(b"NOTASTOR" + raw[8:])
    (tmp_path / "version.gem").write_bytes(raw[:8] + (7).to_bytes(4, "little") + raw[12:])
    for name in ("short", "long", "magic", "version", "missing"):
        with pytest.raises(Exception):
            gem.Store.load(tmp_path / f"{name}.gem", keep=("f32",))
    with pytest.raises(Exception):
        gem.Store.load(good, keep=("bf16",))      # codes need the FP32 copy
    only_bf16 = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("bf16",))
    with pytest.raises(Exception):
        only_bf16.save(tmp_path / "x.gem")
    only_bf16.close()
    a.close()
