"""Doc-range sharded search (Eq. 2 over a store split by set id).

The store is cut into contiguous set-id ranges balanced by vector count
(gem_shard_ranges); every shard is its own Store.  A search runs the exchange
protocol of include/gem.h: each shard's first pass and top rerank_depth with
global ids, a gather of those lists shard-major and their merge into the whole
store's rerank pool, the exact FP32 rerank of each pool entry on the shard that
owns it, an element-wise max across shards, and the final top k.  The answer is
bit for bit gem_search's on the whole store.

`sharded_search` is the protocol itself.  It takes an engine (the per-shard
operations: `GemEngine` runs them through the library's kernels) and an optional
communicator: without one, every shard lives in this process and the gathered
lists are written in place; with one (`DistComm` over torch.distributed, one shard
per rank), the lists are all-gathered and the pool scores all-reduced by max.
`sharded_score_ids` routes candidate lists of global ids the same way: each
shard scores the entries it owns, and a max across shards combines them.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import Store, Workspace, _check, _dtype_code, _ptr, _stream, lib


def shard_ranges(offsets, n_shards: int) -> np.ndarray:
    """Shard boundaries (int64 [n_shards + 1]): shard s owns sets bounds[s] ..
    bounds[s+1]-1, cut at the set boundary closest to s/n_shards of the vectors.
    Host only."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    bounds = np.zeros(n_shards + 1, dtype=np.int64)
    _check(lib.gem_shard_ranges(off.ctypes.data_as(ctypes.c_void_p), len(off) - 1, n_shards,
                                bounds.ctypes.data_as(ctypes.c_void_p)))
    return bounds


@dataclass
class Shard:
    store: object       # Store of the shard's sets (local ids 0 .. n_sets-1)
    ws: object          # Workspace on that store (max_k >= rerank_depth, max_cands >= B * rerank_depth)
    id_base: int        # global id of the shard's first set
    n_sets: int


def build_shards(vecs: torch.Tensor, offsets, n_shards: int, keep=("f32", "bf16"), **ws_kwargs):
    """Stores and workspaces of all shards of one store (for a single process)."""
    off = np.asarray(offsets, dtype=np.int64)
    bounds = shard_ranges(off, n_shards)
    shards = []
    for s in range(n_shards):
        a, b = int(bounds[s]), int(bounds[s + 1])
        r0, r1 = int(off[a]), int(off[b])
        st = Store(vecs[r0:r1], off[a:b + 1] - r0, keep=keep)
        shards.append(Shard(st, Workspace(st, **ws_kwargs), a, b - a))
    return shards, bounds


class GemEngine:
    """The per-shard operations of the protocol, on the library's kernels."""

    def __init__(self, device):
        self.device = torch.device(device)

    def ids(self, shape):
        return torch.empty(shape, dtype=torch.int64, device=self.device)

    def scores(self, shape, fill=None):
        if fill is None:
            return torch.empty(shape, dtype=torch.float32, device=self.device)
        return torch.full(shape, fill, dtype=torch.float32, device=self.device)

    def first_pass(self, sh: Shard, q, qo, compute, depth, out_ids, out_scores):
        _check(lib.gem_shard_first_pass(sh.store.handle, sh.ws.handle, _ptr(q), _ptr(qo), qo.numel() - 1,
                                        q.shape[0], _dtype_code(compute), depth, sh.id_base, _ptr(out_ids),
                                        _ptr(out_scores), _stream()))

    def merge(self, scores, ids, k):
        n_lists, rows, k_in = scores.shape
        out_i = self.ids((rows, k))
        out_s = self.scores((rows, k))
        _check(lib.gem_merge_topk(_ptr(scores), _ptr(ids), n_lists, rows, k_in, k, _ptr(out_i), _ptr(out_s),
                                  _stream()))
        return out_i, out_s

    def rerank_owned(self, sh: Shard, q, qo, pool_ids, pool_scores):
        rows, depth = pool_ids.shape
        _check(lib.gem_shard_rerank(sh.store.handle, sh.ws.handle, _ptr(q), _ptr(qo), rows, q.shape[0],
                                    _ptr(pool_ids), depth, sh.id_base, _ptr(pool_scores), _stream()))

    def score_owned(self, sh: Shard, q, qo, cand_off, cand_ids, compute, scores):
        _check(lib.gem_shard_score_ids(sh.store.handle, sh.ws.handle, _ptr(q), _ptr(qo), qo.numel() - 1,
                                       q.shape[0], _ptr(cand_off), _ptr(cand_ids), cand_ids.numel(),
                                       _dtype_code(compute), sh.id_base, _ptr(scores), _stream()))

    def topk(self, ws_shard: Shard, scores, ids, k):
        rows, cols = scores.shape
        out_i = self.ids((rows, k))
        out_s = self.scores((rows, k))
        _check(lib.gem_topk(ws_shard.ws.handle, _ptr(scores), None, rows, cols, _ptr(ids), k, _ptr(out_i),
                            _ptr(out_s), _stream()))
        return out_i, out_s


class DistComm:
    """The protocol's two collectives over torch.distributed (one shard per rank)."""

    def __init__(self, dist, group=None):
        self.dist = dist
        self.group = group

    @property
    def world(self) -> int:
        return self.dist.get_world_size(self.group)

    def all_gather(self, out, local):
        """out [world, *local.shape] <- every rank's `local`, rank-major."""
        parts = list(out.unbind(0))
        self.dist.all_gather(parts, local.contiguous(), group=self.group)
        if parts[0].data_ptr() != out[0].data_ptr():   # the backend returned new tensors
            out.copy_(torch.stack(parts))

    def all_reduce_max(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)


def sharded_search(engine, shards, n_shards: int, q, qo, compute, rerank_depth: int, k: int, comm=None):
    """Top k per query over all shards (ids global): the protocol of gem_shard_*.

    shards: every shard (comm None) or this rank's single shard (comm given,
    shard index = rank).  Returns (ids int64 [B, k], scores float32 [B, k]).
    """
    B = qo.numel() - 1
    R = rerank_depth
    all_ids = engine.ids((n_shards, B, R))
    all_sc = engine.scores((n_shards, B, R))
    if comm is None:
        assert len(shards) == n_shards
        for s, sh in enumerate(shards):                  # written in place, shard-major
            engine.first_pass(sh, q, qo, compute, R, all_ids[s], all_sc[s])
    else:
        assert len(shards) == 1 and comm.world == n_shards
        li, ls = engine.ids((B, R)), engine.scores((B, R))
        engine.first_pass(shards[0], q, qo, compute, R, li, ls)
        comm.all_gather(all_ids, li)
        comm.all_gather(all_sc, ls)
    pool_ids, _ = engine.merge(all_sc, all_ids, R)        # the whole store's rerank pool
    pool_sc = engine.scores((B, R), fill=float("-inf"))
    for sh in shards:                                      # each entry scored by its owner
        engine.rerank_owned(sh, q, qo, pool_ids, pool_sc)
    if comm is not None:
        comm.all_reduce_max(pool_sc)
    return engine.topk(shards[0], pool_sc, pool_ids, k)


def sharded_score_ids(engine, shards, n_shards: int, q, qo, cand_off, cand_ids, compute="f32", comm=None):
    """Scores of per-query candidate lists of GLOBAL set ids over all shards (the
    scoring step of a beam expansion, Algorithm 5, routed to the owners): every
    shard writes the entries it owns into a buffer of -inf, and an element-wise
    max across shards combines them.  Equal, bit for bit, to gem_score_ids on the
    whole store.  shards as in sharded_search.  Returns float32 [n_cands]."""
    sc = engine.scores((cand_ids.numel(),), fill=float("-inf"))
    if comm is None:
        assert len(shards) == n_shards
    else:
        assert len(shards) == 1 and comm.world == n_shards
    for sh in shards:
        engine.score_owned(sh, q, qo, cand_off, cand_ids, compute, sc)
    if comm is not None:
        comm.all_reduce_max(sc)
    return sc
