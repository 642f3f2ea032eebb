"""Seeded synthetic inputs shaped like the paper's retrieval workloads.

This module only draws random numbers and builds inputs from them: mixture
centres, set lengths, candidate lists and unit-normalised vectors.  It holds none
of the retrieval method's arithmetic (no similarity, no max, no top-k, no
quantisation), so both the FP64 oracle's tests and the GPU path's tests can take
their inputs from here without sharing any code with each other.

Vector recipe (the same for every workload): centre coordinates ~ N(0, 1),
vector = centre + N(0, noise^2) per coordinate with noise = 0.3, each vector picks
its centre uniformly at random, then it is L2-normalised in FP64 and stored FP32.
Queries are drawn from the same mixture with a different seed stream.

Randomness: set lengths, centre choices and candidate lists come from numpy's
PCG64 generator; the Gaussian noise comes from torch's generator on the device the
vectors are built on (CPU for small workloads, CUDA for corpus-sized ones), so a
given (workload, seed, device type) always yields the same bytes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

D = 128
NOISE = 0.3


@dataclass
class VectorSets:
    """A CSR-packed collection of vector sets: rows vecs[offsets[i]:offsets[i+1]] form set i."""

    vecs: torch.Tensor          # float32 [V, D]
    offsets: np.ndarray         # int64 [N + 1], offsets[0] = 0, strictly increasing

    @property
    def n_sets(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_vecs(self) -> int:
        return int(self.offsets[-1])

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)


def _offsets(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


def centres(n_centres: int, seed: int, d: int = D) -> np.ndarray:
    """Mixture centres, coordinates ~ N(0, 1), float64 [n_centres, d]."""
    rng = np.random.default_rng([seed, 0xC3])
    return rng.standard_normal((n_centres, d))


def draw_vectors(n: int, cents: np.ndarray, seed: int, device="cpu",
                 noise: float = NOISE, chunk: int = 1 << 22) -> torch.Tensor:
    """n unit-norm float32 vectors from the Gaussian mixture with centres `cents`."""
    rng = np.random.default_rng([seed, 0xA5])
    which = rng.integers(0, len(cents), size=n)
    d = cents.shape[1]
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    cent_t = torch.from_numpy(cents).to(dev)
    out = torch.empty((n, d), dtype=torch.float32, device=dev)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        idx = torch.from_numpy(which[s:e]).to(dev)
        x = cent_t.index_select(0, idx)
        x.add_(torch.randn((e - s, d), dtype=torch.float64, device=dev, generator=gen), alpha=noise)
        x.div_(torch.linalg.vector_norm(x, dim=1, keepdim=True))
        out[s:e].copy_(x)
    return out


def lengths_uniform(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Set lengths i.i.d. uniform on the integers lo..hi (inclusive)."""
    rng = np.random.default_rng([seed, 0x1E])
    return rng.integers(lo, hi + 1, size=n).astype(np.int64)


def lengths_lognormal(n: int, mean: float, sigma: float, lo: int, hi: int, seed: int) -> np.ndarray:
    """round(clip(LogNormal(mu, sigma), lo, hi)) with mu chosen so the unclipped mean is `mean`."""
    rng = np.random.default_rng([seed, 0x1F])
    mu = math.log(mean) - sigma * sigma / 2.0
    x = rng.lognormal(mu, sigma, size=n)
    return np.rint(np.clip(x, lo, hi)).astype(np.int64)


def vector_sets(lengths: np.ndarray, cents: np.ndarray, seed: int, device="cpu") -> VectorSets:
    lengths = np.asarray(lengths, dtype=np.int64)
    off = _offsets(lengths)
    return VectorSets(draw_vectors(int(off[-1]), cents, seed, device), off)


def candidate_lists(n_queries: int, n_docs: int, len_lo: int, len_hi: int, shared_frac: float,
                    pool_size: int, seed: int):
    """Per-query candidate id lists with no duplicate inside a list.

    Each list length is uniform in len_lo..len_hi; a fraction `shared_frac` of the
    entries comes from a pool of `pool_size` ids common to all queries, the rest are
    uniform over [0, n_docs).  Returns (cand_offsets int64 [B+1], cand_ids int64).
    """
    rng = np.random.default_rng([seed, 0x5C])
    pool = rng.choice(n_docs, size=min(pool_size, n_docs), replace=False)
    lens = rng.integers(len_lo, len_hi + 1, size=n_queries)
    lists = []
    for L in lens:
        n_sh = min(int(round(shared_frac * L)), len(pool))
        sh = rng.choice(pool, size=n_sh, replace=False)
        need = int(L) - n_sh
        rest = np.zeros(0, np.int64)
        while len(rest) < need:
            cand = np.unique(rng.integers(0, n_docs, size=2 * need + 8))
            cand = cand[~np.isin(cand, sh)]
            rest = np.unique(np.concatenate([rest, cand]))
        rest = rng.permutation(rest)[:need]
        ids = np.concatenate([sh, rest]).astype(np.int64)
        rng.shuffle(ids)
        lists.append(ids)
    off = _offsets(np.asarray([len(x) for x in lists], dtype=np.int64))
    return off, (np.concatenate(lists) if lists else np.zeros(0, np.int64))


def shift_lists(cand_ids: np.ndarray, rnd: int, n_docs: int, step: int = 7919) -> np.ndarray:
    """Candidate ids of a later round: (id + rnd * step) mod n_docs.  The map is a
    bijection, so lengths, the shared pool structure and the absence of duplicates
    inside a list carry over unchanged."""
    return ((cand_ids + rnd * step) % n_docs).astype(np.int64)


def random_graph(n: int, degree: int, seed: int):
    """A seeded random undirected graph over n nodes as CSR (offsets int64 [n+1],
    neighbours int32): every node draws `degree` distinct other nodes, edges are
    made symmetric, and each list is sorted without repeats."""
    rng = np.random.default_rng([seed, 0x6A])
    src = np.repeat(np.arange(n), degree)
    dst = (src + rng.integers(1, n, size=n * degree)) % n
    a = np.concatenate([src, dst])
    b = np.concatenate([dst, src])
    key = np.unique(a.astype(np.int64) * n + b)
    a, b = key // n, key % n
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, a + 1, 1)
    return np.cumsum(off), b.astype(np.int32)


# ---------------------------------------------------------------------------
# Workloads.  Sizes follow the five benchmark configurations; the `small`
# variants keep the same structure at sizes the FP64 oracle finishes in seconds.
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    seed: int
    docs: VectorSets
    queries: VectorSets
    params: dict = field(default_factory=dict)


def exact_fp32(seed: int = 1235, n_sets: int = 2000, n_queries: int = 10, m_q: int = 32,
               device="cpu") -> Workload:
    """Plain exact MaxSim: 2,000 sets of 16..64 vectors, 64-centre mixture, 10 queries x 32."""
    cents = centres(64, seed)
    docs = vector_sets(lengths_uniform(n_sets, 16, 64, seed), cents, seed, device)
    qs = vector_sets(np.full(n_queries, m_q, np.int64), cents, seed + 7919, device)
    return Workload("exact-fp32-2k", seed, docs, qs, {"k": 10})


def text_corpus(seed: int = 1236, n_sets: int = 500_000, n_queries: int = 1000, m_q: int = 32,
                n_centres: int = 4096, device="cpu") -> Workload:
    """Text-corpus shape: lognormal lengths (mean 70, sigma 0.5, clipped 20..180), 4,096 centres."""
    cents = centres(n_centres, seed)
    docs = vector_sets(lengths_lognormal(n_sets, 70.0, 0.5, 20, 180, seed), cents, seed, device)
    qs = vector_sets(np.full(n_queries, m_q, np.int64), cents, seed + 7919, device)
    return Workload("text-500k", seed, docs, qs, {"rerank": 1000, "k": 100})


def multimodal_pages(seed: int = 1237, n_sets: int = 50_000, set_len: int = 1024,
                     n_queries: int = 500, n_centres: int = 1024, device="cpu") -> Workload:
    """Multi-modal page shape: fixed-length sets, 1,024 centres, queries of 16..32 vectors."""
    cents = centres(n_centres, seed)
    docs = vector_sets(np.full(n_sets, set_len, np.int64), cents, seed, device)
    qs = vector_sets(lengths_uniform(n_queries, 16, 32, seed + 7919), cents, seed + 7919, device)
    return Workload("pages-50k", seed, docs, qs, {"rerank": 2000, "k": 100})


def beam_batch(docs: VectorSets, cents: np.ndarray, seed: int = 1238, n_queries: int = 4096,
               len_lo: int = 64, len_hi: int = 512, shared_frac: float = 0.3,
               pool_size: int = 10_000, rnd: int = 0, device="cpu"):
    """Beam-expansion batch: queries of 8..64 vectors, candidate lists of len_lo..len_hi ids."""
    qs = vector_sets(lengths_uniform(n_queries, 8, 64, seed + 7919), cents, seed + 7919, device)
    co, ci = candidate_lists(n_queries, docs.n_sets, len_lo, len_hi, shared_frac, pool_size,
                             seed * 1000 + rnd)
    return qs, co, ci


def contrastive_batch(seed: int = 1239, n_queries: int = 256, docs_per_query: int = 64,
                      m_q: int = 32, len_lo: int = 32, len_hi: int = 256, n_centres: int = 1024,
                      device="cpu") -> Workload:
    """In-batch contrastive scoring: each query owns `docs_per_query` doc sets, positive first."""
    cents = centres(n_centres, seed)
    docs = vector_sets(lengths_uniform(n_queries * docs_per_query, len_lo, len_hi, seed), cents,
                       seed, device)
    qs = vector_sets(np.full(n_queries, m_q, np.int64), cents, seed + 7919, device)
    return Workload("contrastive-256x64", seed, docs, qs,
                    {"docs_per_query": docs_per_query, "tau": 0.05})
