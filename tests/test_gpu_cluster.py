"""GPU parity of the cluster filter (Sec. 4.5.1, Eq. 15) and of the second-stage
k-means that builds C_index from C_quant (Sec. 4.1.1).

Cluster filter: the GPU union C_query equals the oracle's, except for centroids
whose FP64 score ties (within 2e-6, the FP32 dot's error bound for unit vectors)
with the t-th best score of some vector of that query, on either side.  The
bitmask, the sorted list and the count must describe the same set.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

EPS = 2e-6


@pytest.fixture(scope="module")
def gem():
    import paper_2603_20336_b300 as g
    return g


def _check_against_oracle(Q, qoff, C, t, mask, ids, count, max_q_len):
    want = oracle.cluster_filter(Q, qoff, C, t)
    C64 = C.astype(np.float64)
    W = (len(C) + 31) // 32
    for b, w in enumerate(want):
        bits = mask[b].view(np.uint32)
        in_mask = [c for c in range(len(C)) if (bits[c >> 5] >> (c & 31)) & 1]
        assert count[b] == len(in_mask)
        cap = max_q_len * t
        assert ids[b][:min(cap, count[b])].tolist() == in_mask[:cap]
        got = set(in_mask)
        if got != set(w.tolist()):
            S = Q[qoff[b]:qoff[b + 1]].astype(np.float64) @ C64.T
            kth = np.sort(S, axis=1)[:, ::-1][:, t - 1]
            for c in got ^ set(w.tolist()):
                # a near-tie at the t-th place of some query vector explains it
                assert np.any(np.abs(S[:, c] - kth) <= EPS), (b, c)
        assert W == bits.shape[0]


@pytest.mark.parametrize("t", [1, 2, 4, 8])
@pytest.mark.parametrize("k2", [37, 64, 1000])
def test_cluster_filter_matches_oracle(gem, t, k2):
    rng = np.random.default_rng(100 + t + k2)
    cents = synth.centres(64, 77)
    C = synth.draw_vectors(k2, cents, 31 + k2).numpy()
    lens = np.array([32, 1, 17, 0, 64, 100, 5, 32])
    qs = synth.vector_sets(lens, cents, int(rng.integers(1 << 20)))
    Q, qoff = qs.vecs.numpy(), qs.offsets
    mask, ids, count = gem.cluster_filter(torch.from_numpy(Q).cuda(), torch.from_numpy(qoff).cuda(),
                                          torch.from_numpy(C).cuda(), t=t, max_q_len=128)
    _check_against_oracle(Q, qoff, C, t, mask.cpu().numpy(), ids.cpu().numpy(), count.cpu().numpy(), 128)


def test_cluster_filter_capacity_and_self_centroids(gem):
    """Queries longer than max_q_len keep the full set in the mask and the count;
    the list holds the first max_q_len * t ids.  With the query vectors among the
    centroids, t = 1 selects exactly their own indices."""
    rng = np.random.default_rng(5)
    cents = synth.centres(16, 5)
    qs = synth.vector_sets(np.array([40, 8]), cents, 6)
    Q, qoff = qs.vecs.numpy(), qs.offsets
    other = synth.draw_vectors(100, cents, 7).numpy()
    C = np.concatenate([other[:50], Q, other[50:]])
    mask, ids, count = gem.cluster_filter(torch.from_numpy(Q).cuda(), torch.from_numpy(qoff).cuda(),
                                          torch.from_numpy(C).cuda(), t=1, max_q_len=16)
    count = count.cpu().numpy()
    ids = ids.cpu().numpy()
    assert count.tolist() == [40, 8]
    assert ids[0].tolist() == list(range(50, 66))          # capacity 16 of 40
    assert ids[1][:8].tolist() == list(range(90, 98))
    bits = mask.cpu().numpy().view(np.uint32)[0]
    assert [c for c in range(len(C)) if (bits[c >> 5] >> (c & 31)) & 1] == list(range(50, 90))
    del rng


def test_cluster_filter_rejects_bad_arguments(gem):
    C = torch.zeros((10, 128), device="cuda")
    q = torch.zeros((4, 128), device="cuda")
    qo = torch.tensor([0, 4], dtype=torch.int64, device="cuda")
    for t in (0, 9, 11):
        with pytest.raises(Exception):
            gem.cluster_filter(q, qo, C, t=t)


def test_kmeans_init_and_one_lloyd_step_match_oracle(gem):
    """C_index from C_quant (second clustering stage).  iters = 0 returns k
    distinct rows of x (the seeded initial choice); iters = 1 returns the
    oracle's Lloyd update of those rows (renormalised means of the members),
    except for the few centroids whose member set differs because of an FP32
    near-tie in the assignment; the result is unit-norm."""
    X = synth.draw_vectors(4000, synth.centres(40, 9), 10).numpy()
    k = 64
    C0 = gem.kmeans(torch.from_numpy(X).cuda(), k, iters=0, seed=3).cpu().numpy()
    rows = {tuple(r) for r in X.tolist()}
    assert all(tuple(c) in rows for c in C0.tolist())
    assert len({tuple(c) for c in C0.tolist()}) == k
    C1 = gem.kmeans(torch.from_numpy(X).cuda(), k, iters=1, seed=3).cpu().numpy()
    np.testing.assert_allclose(np.linalg.norm(C1, axis=1), 1.0, atol=1e-5)
    want = oracle.kmeans_update(X, oracle.assign_codes(X, C0), C0)
    close = np.all(np.abs(C1 - want) <= 1e-5, axis=1)
    assert close.mean() >= 0.95, close.mean()
    C8 = gem.kmeans(torch.from_numpy(X).cuda(), k, iters=8, seed=3).cpu().numpy()
    np.testing.assert_allclose(np.linalg.norm(C8, axis=1), 1.0, atol=1e-5)


def test_index_codes_members_and_entry_points_match_oracle(gem):
    """C_index attached to a store: every stored vector's nearest coarse centroid
    agrees with the oracle except FP64 near-ties; given the GPU's codes, the
    oracle's member lists and SplitMix64 draws give exactly the GPU's entry sets,
    for the C_query lists the GPU cluster filter returns (empty clusters give -1)."""
    w = synth.exact_fp32(n_sets=700, n_queries=6)
    store = gem.Store(w.docs.vecs.cuda(), w.docs.offsets, keep=("f32",))
    k2 = 48
    Ci = gem.kmeans(w.docs.vecs.cuda(), k2, iters=3, seed=2)
    Ci[5] = -Ci[5]            # a centroid few vectors choose: likely an empty cluster
    gem.set_index_centroids(store, Ci)
    codes = store.export("index_codes").cpu().numpy()
    X = w.docs.vecs.numpy().astype(np.float64)
    C64 = Ci.cpu().numpy().astype(np.float64)
    want = oracle.assign_codes(X, C64)
    diff = np.nonzero(codes != want)[0]
    for i in diff:
        s = X[i] @ C64.T
        assert s[want[i]] - s[codes[i]] <= EPS, i
    members = oracle.cluster_members(codes, w.docs.offsets, k2)
    q, qo = w.queries.vecs.cuda(), torch.from_numpy(w.queries.offsets).cuda()
    _, ids, count = gem.cluster_filter(q, qo, Ci, t=4, max_q_len=32)
    # add an empty cluster to one query's list to cover the -1 case
    empty = [c for c in range(k2) if len(members[c]) == 0]
    ids_np, count_np = ids.cpu().numpy(), count.cpu().numpy()
    if empty:
        ids_np[0, count_np[0]] = empty[0]
        count_np[0] += 1
    for seed in (0, 12345):
        got = gem.entry_points(store, torch.from_numpy(ids_np).cuda(), torch.from_numpy(count_np).cuda(),
                               seed=seed).cpu().numpy()
        lists = [ids_np[b, :count_np[b]] for b in range(len(count_np))]
        exp = oracle.entry_points(lists, members, seed)
        for b in range(len(lists)):
            assert got[b, :count_np[b]].tolist() == exp[b].tolist()
            assert np.all(got[b, count_np[b]:] == -1)
    store.close()
