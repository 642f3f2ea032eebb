"""GPU parity of the cluster-guided multi-path beam search (Algorithm 5), run in
rounds over a seeded random graph.

The oracle runs the same rounds sequentially with the GPU's own inputs to the
search logic: the qsim score of every (query, set) pair (gem_estimate_codes,
whose values are checked against FP64 under the qCH row), the
clusters of every set (its vectors' nearest C_index centroids), C_query and the
entry sets.  Given those, every decision is exact, so R (ids and scores, best
first) and the number of rounds must match bit for bit.
"""
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


@pytest.fixture(scope="module")
def setup(gem):
    seed = 4321
    cents = synth.centres(96, seed)
    docs = synth.vector_sets(synth.lengths_lognormal(3000, 40.0, 0.5, 8, 120, seed), cents, seed)
    store = gem.Store(docs.vecs.cuda(), docs.offsets, keep=("f32",))
    C = gem.train_codebook(store, k1=256, iters=5, seed=1)
    gem.set_codebook(store, C)
    Ci = gem.kmeans(C, 24, iters=5, seed=2)
    gem.set_index_centroids(store, Ci)
    lens = np.array([32, 20, 32, 9, 32, 27, 32, 1, 32, 16])
    qs = synth.vector_sets(lens, cents, seed + 1)
    q, qo = qs.vecs.cuda(), torch.from_numpy(qs.offsets).cuda()
    ws = gem.Workspace(store, max_queries=len(lens), max_q_rows=int(lens.sum()), max_q_len=32,
                       max_cands=len(lens) * 3000)
    mask, lst, cnt = gem.cluster_filter(q, qo, Ci, t=2, max_q_len=32)
    ent = gem.entry_points(store, lst, cnt, seed=9)
    go, gn = synth.random_graph(3000, 6, seed)
    # the GPU's qsim of every (query, set) pair, by the search's own arithmetic
    # (centroid tables and lookups; the all-sets form is bit-identical to the
    # id-list form the search uses)
    B, N = len(lens), store.n_sets
    allq = gem.estimate_codes(store, ws, q, qo).cpu().numpy()
    codes = store.export("index_codes").cpu().numpy()
    off = docs.offsets
    set_clusters = [set(codes[off[s]:off[s + 1]].tolist()) for s in range(N)]
    yield dict(store=store, ws=ws, q=q, qo=qo, mask=mask, lst=lst.cpu().numpy(), cnt=cnt.cpu().numpy(),
               ent=ent, go=go, gn=gn, allq=allq, set_clusters=set_clusters, B=B)
    ws.close()
    store.close()


@pytest.mark.parametrize("ef,max_rounds", [(16, 1000), (5, 1000), (40, 3), (300, 1000)])
def test_beam_search_matches_oracle_rounds(gem, setup, ef, max_rounds):
    d = setup
    ids, sc, rounds = gem.beam_search(d["store"], d["ws"], d["q"], d["qo"], torch.from_numpy(d["go"]).cuda(),
                                      torch.from_numpy(d["gn"]).cuda(), d["mask"], d["ent"], ef=ef,
                                      max_rounds=max_rounds)
    assert d["ws"].status() == 0
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    ent = d["ent"].cpu().numpy()
    want_rounds = 0
    for b in range(d["B"]):
        qc = d["lst"][b, :d["cnt"][b]]
        R, r = oracle.beam_search(lambda s, b=b: float(d["allq"][b, s]), d["go"], d["gn"], d["set_clusters"], qc,
                                  ent[b], ef=ef, max_rounds=max_rounds)
        want_rounds = max(want_rounds, r)
        n = len(R)
        assert ids[b, :n].tolist() == [i for _, i in R], b
        np.testing.assert_array_equal(sc[b, :n], np.array([s for s, _ in R], dtype=np.float32))
        assert np.all(ids[b, n:] == -1)
    assert rounds == want_rounds


def test_beam_search_rejects_a_neighbour_out_of_range(gem, setup):
    d = setup
    gn = d["gn"].copy()
    gn[:] = 5000           # every neighbour id out of range
    with pytest.raises(Exception):
        gem.beam_search(d["store"], d["ws"], d["q"], d["qo"], torch.from_numpy(d["go"]).cuda(),
                        torch.from_numpy(gn).cuda(), d["mask"], d["ent"], ef=8)


def test_beam_search_rejects_lists_longer_than_max_degree(gem, setup):
    """The round buffer holds max_degree sets per queue; a popped set with more
    neighbours to queue than that stops the walk and the call reports it (the
    writes past the buffer are never made)."""
    d = setup
    with pytest.raises(Exception, match="max_degree"):
        gem.beam_search(d["store"], d["ws"], d["q"], d["qo"], torch.from_numpy(d["go"]).cuda(),
                        torch.from_numpy(d["gn"]).cuda(), d["mask"], d["ent"], ef=8, max_degree=1)
    # the workspace stays usable: the same search with the true degree succeeds
    gem.beam_search(d["store"], d["ws"], d["q"], d["qo"], torch.from_numpy(d["go"]).cuda(),
                    torch.from_numpy(d["gn"]).cuda(), d["mask"], d["ent"], ef=8)
    assert d["ws"].status() == 0


def test_beam_search_with_deleted_sets_matches_oracle(gem, setup):
    """Lazy deletion (Sec. 4.6): deleted sets, among them every entry set of the
    first query and the best sets R held without deletion, are traversed but never
    enter R; the rounds and R match the oracle exactly."""
    d = setup
    args = (d["store"], d["ws"], d["q"], d["qo"], torch.from_numpy(d["go"]).cuda(), torch.from_numpy(d["gn"]).cuda(),
            d["mask"], d["ent"])
    ids0, _, _ = gem.beam_search(*args, ef=16)
    ent = d["ent"].cpu().numpy()
    rng = np.random.default_rng(3)
    dead = set(ids0.cpu().numpy()[:, :4].ravel().tolist()) | {int(e) for e in ent[0] if e >= 0}
    dead |= set(rng.choice(d["store"].n_sets, 300, replace=False).tolist())
    dead.discard(-1)
    gem.mark_deleted(d["store"], sorted(dead))
    try:
        ids, sc, rounds = gem.beam_search(*args, ef=16)
    finally:
        gem.mark_deleted(d["store"], sorted(dead), deleted=False)
    assert d["ws"].status() == 0
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    want_rounds = 0
    for b in range(d["B"]):
        qc = d["lst"][b, :d["cnt"][b]]
        R, r = oracle.beam_search(lambda s, b=b: float(d["allq"][b, s]), d["go"], d["gn"], d["set_clusters"], qc,
                                  ent[b], ef=16, dead=dead)
        want_rounds = max(want_rounds, r)
        n = len(R)
        assert ids[b, :n].tolist() == [i for _, i in R], b
        np.testing.assert_array_equal(sc[b, :n], np.array([s for s, _ in R], dtype=np.float32))
        assert np.all(ids[b, n:] == -1)
    assert rounds == want_rounds
    assert not set(ids.ravel().tolist()) & dead


def test_beam_search_asymmetric_qch_matches_oracle(gem, setup):
    """The search scored by the asymmetric estimate (exact query vectors against
    the stored vectors' centroids): R and the rounds match the oracle run on the
    GPU's asymmetric qsim."""
    d = setup
    gem.set_qch_form(d["ws"], "asymmetric")
    try:
        allq = gem.estimate_codes(d["store"], d["ws"], d["q"], d["qo"]).cpu().numpy()
        ids, sc, rounds = gem.beam_search(d["store"], d["ws"], d["q"], d["qo"], torch.from_numpy(d["go"]).cuda(),
                                          torch.from_numpy(d["gn"]).cuda(), d["mask"], d["ent"], ef=16)
    finally:
        gem.set_qch_form(d["ws"], "symmetric")
    assert d["ws"].status() == 0
    assert np.abs(allq - d["allq"]).max() > 0      # a different estimate
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    ent = d["ent"].cpu().numpy()
    want_rounds = 0
    for b in range(d["B"]):
        qc = d["lst"][b, :d["cnt"][b]]
        R, r = oracle.beam_search(lambda s, b=b: float(allq[b, s]), d["go"], d["gn"], d["set_clusters"], qc,
                                  ent[b], ef=16)
        want_rounds = max(want_rounds, r)
        n = len(R)
        assert ids[b, :n].tolist() == [i for _, i in R], b
        np.testing.assert_array_equal(sc[b, :n], np.array([s for s, _ in R], dtype=np.float32))
    assert rounds == want_rounds


@pytest.mark.parametrize("ef", [16, 300])
def test_beam_search_dense_graph_with_repeated_neighbours(gem, setup, ef):
    """Neighbour lists of about 40 sets, tested 32 at a time on the GPU, with
    repeats inside a group of 32 and across groups (the walk of the oracle queues
    a set once: its second occurrence is visited or fails the same cluster test),
    with R smaller and larger than a round's candidates (ef 16 and 300).
    R and the number of rounds bit-exact against the oracle."""
    d = setup
    go, gn = synth.random_graph(3000, 20, 777)
    gn = gn.copy()
    for node in range(0, 3000, 5):
        lo, hi = int(go[node]), int(go[node + 1])
        if hi - lo >= 36:
            gn[lo + 1] = gn[lo]            # a repeat within the first group
            gn[lo + 34] = gn[lo + 2]       # a repeat in the next group
    ids, sc, rounds = gem.beam_search(d["store"], d["ws"], d["q"], d["qo"], torch.from_numpy(go).cuda(),
                                      torch.from_numpy(gn).cuda(), d["mask"], d["ent"], ef=ef)
    assert d["ws"].status() == 0
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    ent = d["ent"].cpu().numpy()
    want_rounds = 0
    for b in range(d["B"]):
        qc = d["lst"][b, :d["cnt"][b]]
        R, r = oracle.beam_search(lambda s, b=b: float(d["allq"][b, s]), go, gn, d["set_clusters"], qc, ent[b],
                                  ef=ef)
        want_rounds = max(want_rounds, r)
        n = len(R)
        assert ids[b, :n].tolist() == [i for _, i in R], b
        np.testing.assert_array_equal(sc[b, :n], np.array([s for s, _ in R], dtype=np.float32))
    assert rounds == want_rounds
