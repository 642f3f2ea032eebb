"""Doc-range sharding (Eq. 2 over a store split by set id) on CPU: the shard
boundaries of gem_shard_ranges (exact cover of [0, N), balance by vector count)
and the exchange protocol of paper_2603_20336_b300.shard run by world-size-2 and
-3 gloo ranks, one shard per rank, with the FP64 oracle doing each shard's work:
the all-gathered lists are shard-major, the merge is the whole store's top-R pool,
every pool entry is scored by its owner only, and the answer equals the oracle's
single-store search (exhaustive score -> top-R -> exact rerank -> top-k)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
R, K = 12, 5


def _ranges(off, n):
    from paper_2603_20336_b300 import shard
    return shard.shard_ranges(off, n)


@pytest.mark.parametrize("n_shards", [1, 2, 3, 7, 40])
def test_shard_ranges_cover_and_balance(n_shards):
    lens = synth.lengths_lognormal(40, 70.0, 0.5, 20, 180, 3)
    lens[5] = 2000                       # one set far longer than the rest
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    b = _ranges(off, n_shards)
    assert b[0] == 0 and b[-1] == 40 and len(b) == n_shards + 1
    assert np.all(np.diff(b) >= 1)       # every shard non-empty, exact cover, in order
    V = off[-1]
    for s in range(1, n_shards):
        # the boundary is the set boundary closest to s/n of the vectors, unless
        # keeping every shard non-empty moved it
        target = V * s / n_shards
        best = np.argmin(np.abs(off - target))
        assert b[s] == best or b[s] == b[s - 1] + 1 or b[s] == 40 - (n_shards - s)
    if n_shards == 2:
        v = [off[b[s + 1]] - off[b[s]] for s in range(2)]
        assert abs(v[0] - v[1]) <= lens.max()


def test_shard_ranges_rejects_bad_input():
    from paper_2603_20336_b300 import GemError
    off = np.array([0, 3, 5, 9], np.int64)
    with pytest.raises(GemError):
        _ranges(off, 4)                 # more shards than sets
    with pytest.raises(GemError):
        _ranges(np.array([0, 3, 3, 9], np.int64), 2)   # an empty set


class OracleEngine:
    """The protocol's per-shard operations in FP64 on the host (test double of
    GemEngine): first pass = exact CH of the shard's sets and their top R."""

    def __init__(self, X, off):
        self.X, self.off = X, off

    def ids(self, shape):
        return torch.empty(shape, dtype=torch.int64)

    def scores(self, shape, fill=None):
        t = torch.empty(shape, dtype=torch.float64)
        return t if fill is None else t.fill_(fill)

    def _rows(self, sh):
        a, b = sh.id_base, sh.id_base + sh.n_sets
        r0 = self.off[a]
        return self.X[self.off[a]:self.off[b]], self.off[a:b + 1] - r0

    def first_pass(self, sh, q, qo, compute, depth, out_ids, out_scores):
        Xs, os_ = self._rows(sh)
        S = oracle.score_all(q.numpy(), qo.numpy(), Xs, os_)
        for b in range(S.shape[0]):
            ii, ss = oracle.topk(S[b], depth)
            out_ids[b] = -1
            out_scores[b] = -np.inf
            out_ids[b, :len(ii)] = torch.from_numpy(ii + sh.id_base)
            out_scores[b, :len(ss)] = torch.from_numpy(ss)

    def merge(self, scores, ids, k):
        n_lists, rows, k_in = scores.shape
        oi, os_ = self.ids((rows, k)).fill_(-1), self.scores((rows, k), -np.inf)
        for r in range(rows):
            s = scores[:, r, :].reshape(-1).numpy()
            i = ids[:, r, :].reshape(-1).numpy()
            keep = i >= 0
            ii, ss = oracle.topk(s[keep], k, i[keep])
            oi[r, :len(ii)] = torch.from_numpy(ii)
            os_[r, :len(ss)] = torch.from_numpy(ss)
        return oi, os_

    def rerank_owned(self, sh, q, qo, pool_ids, pool_scores):
        Xs, os_ = self._rows(sh)
        B, depth = pool_ids.shape
        local = pool_ids.numpy() - sh.id_base
        own = (pool_ids.numpy() >= 0) & (local >= 0) & (local < sh.n_sets)
        ids = np.where(own, local, -1).reshape(-1)
        co = np.arange(B + 1, dtype=np.int64) * depth
        sc = oracle.score_ids(q.numpy(), qo.numpy(), Xs, os_, co, ids).reshape(B, depth)
        pool_scores[torch.from_numpy(own)] = torch.from_numpy(sc[own])

    def score_owned(self, sh, q, qo, cand_off, cand_ids, compute, scores):
        Xs, os_ = self._rows(sh)
        ids = cand_ids.numpy()
        local = ids - sh.id_base
        own = (ids >= 0) & (local >= 0) & (local < sh.n_sets)
        sc = oracle.score_ids(q.numpy(), qo.numpy(), Xs, os_, cand_off.numpy(), np.where(own, local, -1))
        scores[torch.from_numpy(own)] = torch.from_numpy(sc[own])

    def topk(self, shard, scores, ids, k):
        rows = scores.shape[0]
        oi, os_ = self.ids((rows, k)).fill_(-1), self.scores((rows, k), -np.inf)
        for r in range(rows):
            keep = ids[r].numpy() >= 0
            ii, ss = oracle.topk(scores[r].numpy()[keep], k, ids[r].numpy()[keep])
            oi[r, :len(ii)] = torch.from_numpy(ii)
            os_[r, :len(ss)] = torch.from_numpy(ss)
        return oi, os_


def _data():
    w = synth.exact_fp32(n_sets=90, n_queries=4)
    return w.docs.vecs.numpy(), w.docs.offsets, w.queries.vecs, torch.from_numpy(w.queries.offsets)


def _lists():
    """Candidate lists of global ids over the 90-set store: 4 queries, uneven
    lengths, an empty list, -1 entries."""
    rng = np.random.default_rng(17)
    lens = np.array([7, 0, 19, 12])
    co = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    ci = rng.integers(-1, 90, size=int(co[-1])).astype(np.int64)
    return co, ci


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


class _GatherLog:
    """DistComm with a record of what the gathers returned (the layout check)."""

    def __init__(self, comm):
        self.comm = comm
        self.gathered = []

    @property
    def world(self):
        return self.comm.world

    def all_gather(self, out, local):
        self.comm.all_gather(out, local)
        self.gathered.append((out.clone(), local.clone()))

    def all_reduce_max(self, t):
        self.comm.all_reduce_max(t)


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2603_20336_b300 import shard
        X, off, q, qo = _data()
        bounds = shard.shard_ranges(off, world)
        mine = shard.Shard(None, None, int(bounds[rank]), int(bounds[rank + 1] - bounds[rank]))
        comm = _GatherLog(shard.DistComm(dist))
        ids, sc = shard.sharded_search(OracleEngine(X, off), [mine], world, q, qo, "f32", R, K, comm=comm)
        # layout: slot s of every gather holds rank s's own list
        layout_ok = True
        for full, local in comm.gathered:
            got = [None] * world
            dist.all_gather_object(got, local.numpy())
            layout_ok &= all(np.array_equal(full[s].numpy(), got[s]) for s in range(world))
        co, ci = _lists()
        routed = shard.sharded_score_ids(OracleEngine(X, off), [mine], world, q, qo, torch.from_numpy(co),
                                         torch.from_numpy(ci), "f32", comm=comm)
        out.put((rank, bounds, ids.numpy(), sc.numpy(), layout_ok, routed.numpy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_protocol_on_gloo_ranks_equals_single_store_search(world):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([out.get(timeout=300) for _ in procs], key=lambda x: x[0])
    co, ci = _lists()
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    X, off, q, qo = _data()
    S = oracle.score_all(q.numpy(), qo.numpy(), X, off)
    pool = np.stack([oracle.topk(S[b], R)[0] for b in range(S.shape[0])])
    want_ids, want_sc = oracle.rerank(q.numpy(), qo.numpy(), X, off, pool, K)
    want_routed = oracle.score_ids(q.numpy(), qo.numpy(), X, off, co, ci)
    for rank, bounds, ids, sc, layout_ok, routed in res:
        assert layout_ok
        assert np.array_equal(bounds, res[0][1])
        np.testing.assert_array_equal(ids, want_ids)      # every rank returns the answer
        np.testing.assert_array_equal(sc, want_sc)
        np.testing.assert_array_equal(routed, want_routed)  # candidate lists routed to their owners


def test_routed_candidate_lists_in_one_process():
    """Candidate lists of global ids routed to their owner shards: each shard
    scores what it owns and the max over shards equals the single-store scores."""
    from paper_2603_20336_b300 import shard
    X, off, q, qo = _data()
    co, ci = _lists()
    want = oracle.score_ids(q.numpy(), qo.numpy(), X, off, co, ci)
    for n in (1, 2, 3):
        bounds = shard.shard_ranges(off, n)
        shards = [shard.Shard(None, None, int(bounds[s]), int(bounds[s + 1] - bounds[s])) for s in range(n)]
        got = shard.sharded_score_ids(OracleEngine(X, off), shards, n, q, qo, torch.from_numpy(co),
                                      torch.from_numpy(ci), "f32")
        np.testing.assert_array_equal(got.numpy(), want)


def test_sharded_protocol_in_one_process_equals_single_store_search():
    """The same protocol without a communicator: all shards in one process, the
    lists written in place shard-major."""
    from paper_2603_20336_b300 import shard
    X, off, q, qo = _data()
    for n in (1, 2, 4):
        bounds = shard.shard_ranges(off, n)
        shards = [shard.Shard(None, None, int(bounds[s]), int(bounds[s + 1] - bounds[s])) for s in range(n)]
        ids, sc = shard.sharded_search(OracleEngine(X, off), shards, n, q, qo, "f32", R, K)
        S = oracle.score_all(q.numpy(), qo.numpy(), X, off)
        pool = np.stack([oracle.topk(S[b], R)[0] for b in range(S.shape[0])])
        want_ids, want_sc = oracle.rerank(q.numpy(), qo.numpy(), X, off, pool, K)
        np.testing.assert_array_equal(ids.numpy(), want_ids)
        np.testing.assert_array_equal(sc.numpy(), want_sc)
