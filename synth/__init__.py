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
PCG64 generator.  The noise comes either from torch's generator on the device the
vectors are built on (draw_vectors: a given (workload, seed, device type) always
yields the same bytes), or, for the text-corpus workload, from a counter-based
SplitMix64 hash with an Irwin-Hall(12) variate (draw_vectors_portable: the same
bytes on every device).
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


# SplitMix64 constants (Steele, Lea and Flood, "Fast splittable pseudorandom
# number generators", 2014), as signed 64-bit integers
_SM_GAMMA = 0x9E3779B97F4A7C15 - (1 << 64)
_SM_M1 = 0xBF58476D1CE4E5B9 - (1 << 64)
_SM_M2 = 0x94D049BB133111EB - (1 << 64)


def _srl(x: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (x >> s) & ((1 << (64 - s)) - 1)


def _splitmix64(state: torch.Tensor) -> torch.Tensor:
    """SplitMix64 output for each 64-bit state (wrapping int64 arithmetic)."""
    z = state + _SM_GAMMA
    z = (z ^ _srl(z, 30)) * _SM_M1
    z = (z ^ _srl(z, 27)) * _SM_M2
    return z ^ _srl(z, 31)


def draw_vectors_portable(n: int, cents: np.ndarray, seed: int, device="cpu", noise: float = NOISE,
                          chunk: int = 1 << 18) -> torch.Tensor:
    """n unit-norm float32 vectors of the mixture, bit-identical on every device.

    Each vector picks a centre uniformly (numpy PCG64).  The noise of coordinate
    k of vector v is an Irwin-Hall variate: the sum of twelve 16-bit uniforms
    taken from three SplitMix64 outputs of the counter 3 (128 v + k) + i, at the
    bins' midpoints, minus 6 -- mean 0, variance 1, the textbook sum-of-twelve
    approximation of N(0, 1), tails cut at +-6.  Everything after the integer
    hash is exact or one correctly rounded FP64 operation in a fixed order (the
    squared norm is summed by a fixed pairwise tree), so CPU and GPU give the
    same bytes."""
    rng = np.random.default_rng([seed, 0xA5])
    which = rng.integers(0, len(cents), size=n)
    d = cents.shape[1]
    assert d & (d - 1) == 0, "the pairwise norm tree needs a power-of-two dimension"
    dev = torch.device(device)
    cent_t = torch.from_numpy(cents).to(dev)
    key = (int(seed) * 0x2545F4914F6CDD1D) % (1 << 64)
    key = key - (1 << 64) if key >= (1 << 63) else key
    out = torch.empty((n, d), dtype=torch.float32, device=dev)
    k3 = torch.arange(d * 3, dtype=torch.int64, device=dev)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        ctr = torch.arange(s, e, dtype=torch.int64, device=dev)[:, None] * (3 * d) + k3[None, :]
        h = _splitmix64(ctr + key).view(e - s, d, 3)
        acc = torch.zeros((e - s, d), dtype=torch.int64, device=dev)
        for sh in (0, 16, 32, 48):
            acc += _srl(h, sh).bitwise_and(0xFFFF).sum(dim=2)
        z = (acc.to(torch.float64) + 6.0) / 65536.0 - 6.0
        x = cent_t.index_select(0, torch.from_numpy(which[s:e]).to(dev)) + noise * z
        sq = x * x
        w = d
        while w > 1:                       # fixed pairwise tree over the coordinates
            w //= 2
            sq = sq[:, :w] + sq[:, w:2 * w]
        out[s:e].copy_(x / torch.sqrt(sq))
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


def vector_sets(lengths: np.ndarray, cents: np.ndarray, seed: int, device="cpu", portable: bool = False) -> VectorSets:
    lengths = np.asarray(lengths, dtype=np.int64)
    off = _offsets(lengths)
    draw = draw_vectors_portable if portable else draw_vectors
    return VectorSets(draw(int(off[-1]), cents, seed, device), off)


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
                n_centres: int = 4096, device="cpu", portable: bool = True) -> Workload:
    """Text-corpus shape: lognormal lengths (mean 70, sigma 0.5, clipped 20..180), 4,096 centres.
    portable (default): the device-independent noise of draw_vectors_portable, so
    the FP64 ground truth of the full workload can be computed on any host."""
    cents = centres(n_centres, seed)
    docs = vector_sets(lengths_lognormal(n_sets, 70.0, 0.5, 20, 180, seed), cents, seed, device, portable)
    qs = vector_sets(np.full(n_queries, m_q, np.int64), cents, seed + 7919, device, portable)
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


def fingerprint(docs: VectorSets, queries: VectorSets, n_sample: int = 1024) -> str:
    """SHA-256 of a workload's identity: the offsets of both collections and a
    spread sample of their rows (FP32 bytes).  Equal fingerprints mean the data a
    stored ground truth was computed on is the data at hand."""
    import hashlib
    h = hashlib.sha256()
    for vs in (docs, queries):
        h.update(np.ascontiguousarray(vs.offsets, dtype=np.int64).tobytes())
        n = vs.n_vecs
        rows = np.unique(np.linspace(0, n - 1, num=min(n, n_sample)).astype(np.int64))
        sample = vs.vecs[torch.from_numpy(rows).to(vs.vecs.device)].to("cpu", torch.float32).contiguous()
        h.update(sample.numpy().tobytes())
    return h.hexdigest()

