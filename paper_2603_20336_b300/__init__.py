"""Python binding of libgem, the B300 (sm_103a) multi-vector MaxSim library.

Argument marshalling only: every step of every call runs in the library's CUDA
kernels.  Tensors are passed by device pointer on torch's current stream; torch
supplies device memory and streams.  There is no CPU fallback: importing this
package without the compiled library raises ImportError, and every scoring
call needs a CUDA device.

    store = Store(vecs, offsets, keep=("f32", "bf16"))     # CSR doc-set store
    ws = Workspace(store, max_queries=1000, max_q_rows=32000)
    scores = score_all(store, ws, q, q_offsets, "bf16")    # [B, n_sets]
    ids, sc = search(store, ws, q, q_offsets, "bf16", rerank_depth=1000, k=100)
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import _abi

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgem.so")

if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libgem.so is not built ({_LIB_PATH}); run python paper_2603_20336_b300/build.py")

lib = ctypes.CDLL(_LIB_PATH)
_abi.declare(lib)

DTYPES = {"f32": 0, "bf16": 1, "fp8": 2, "codes": 3, "fp8_set": 4}
KEEP = {"f32": 1, "bf16": 2, "fp8": 4, "fp8_set": 8}
STATUS = {0: "GEM_OK", 1: "GEM_ERR_INVALID", 2: "GEM_ERR_OOM", 3: "GEM_ERR_CUDA", 4: "GEM_ERR_TIMEOUT",
          5: "GEM_ERR_UNSUPPORTED", 6: "GEM_ERR_STATE", 7: "GEM_ERR_BOUNDS"}


class GemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _check(code: int):
    if code != 0:
        raise GemError(code, lib.gem_last_error_message().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, name):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return t


def _dtype_code(compute):
    return DTYPES[compute] if isinstance(compute, str) else int(compute)


class Store:
    """CSR doc-set store (Sec. 3.1 problem statement: the database D of vector sets)."""

    def __init__(self, vecs: torch.Tensor, offsets, keep=("f32", "bf16"), stream=None):
        mask = 0
        for k in keep:
            mask |= KEEP[k]
        offsets = torch.as_tensor(offsets, dtype=torch.int64)
        n_sets = offsets.numel() - 1
        h = ctypes.c_void_p()
        if vecs.is_cuda:
            vecs = _dev(vecs, torch.float32, "vecs")
            off = offsets.to(vecs.device).contiguous()
            _check(lib.gem_store_create(_ptr(vecs), _ptr(off), n_sets, vecs.shape[1], mask, 0,
                                        _stream(stream), ctypes.byref(h)))
        else:
            v = vecs.contiguous().to(torch.float32)
            off = offsets.contiguous()
            _check(lib.gem_store_create(_ptr(v), _ptr(off), n_sets, v.shape[1], mask, 1,
                                        _stream(stream), ctypes.byref(h)))
        self._adopt(h, keep)

    def _adopt(self, h, keep):
        self.handle = h
        n_s, n_v, n_p = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib.gem_store_info(h, ctypes.byref(n_s), ctypes.byref(n_v), ctypes.byref(n_p), None))
        self.n_sets = n_s.value
        self.n_vecs = n_v.value
        self.n_pad_vecs = n_p.value
        self.keep = tuple(keep)
        k1, k2 = ctypes.c_int32(), ctypes.c_int32()
        _check(lib.gem_store_codebook_sizes(h, ctypes.byref(k1), ctypes.byref(k2)))
        if k1.value:
            self.k1 = k1.value
        if k2.value:
            self.k2 = k2.value

    def save(self, path, stream=None):
        """Write the store to `path` (offsets, FP32 vectors, C_quant, C_index,
        deletions); needs the FP32 copy."""
        _check(lib.gem_store_save(self.handle, str(path).encode(), _stream(stream)))

    @classmethod
    def load(cls, path, keep=("f32", "bf16"), stream=None):
        """A store read from a file written by save(); every derived array is
        rebuilt on the current device."""
        mask = 0
        for k in keep:
            mask |= KEEP[k]
        h = ctypes.c_void_p()
        _check(lib.gem_store_load(str(path).encode(), mask, _stream(stream), ctypes.byref(h)))
        self = cls.__new__(cls)
        self._adopt(h, keep)
        return self

    def export(self, what: str, stream=None) -> torch.Tensor:
        """Copy of an internal array: 'bf16' (uint16 bits, padded layout), 'fp8'
        (uint8 bits, padded), 'fp8_scale' (float32, padded), 'fp8_set' (uint8
        bits of the per-set-scale copy, padded), 'set_scale' (float32 per set),
        'offsets' or 'pad_offsets' (int64)."""
        P = self.n_pad_vecs
        spec = {"bf16": (0, torch.int16, (P, 128)), "fp8": (1, torch.uint8, (P, 128)),
                "fp8_scale": (2, torch.float32, (P,)), "offsets": (3, torch.int64, (self.n_sets + 1,)),
                "pad_offsets": (4, torch.int64, (self.n_sets + 1,)),
                "codes": (5, torch.int32, (self.n_vecs,)),
                "codebook": (6, torch.float32, (getattr(self, "k1", 0), 128)),
                "index_codes": (7, torch.int32, (self.n_vecs,)),
                "f32": (8, torch.float32, (self.n_vecs, 128)),
                "index_centroids": (9, torch.float32, (getattr(self, "k2", 0), 128)),
                "deleted": (10, torch.int32, ((self.n_sets + 31) // 32,)),
                "fp8_set": (11, torch.uint8, (P, 128)),
                "set_scale": (12, torch.float32, (self.n_sets,))}
        code, dt, shape = spec[what]
        out = torch.empty(shape, dtype=dt, device="cuda")
        _check(lib.gem_store_export(self.handle, code, _ptr(out), out.numel() * out.element_size(),
                                    _stream(stream)))
        return out

    def close(self):
        if self.handle:
            lib.gem_store_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Workspace:
    """Preallocated scratch for scoring calls against one store."""

    def __init__(self, store: Store, max_queries: int, max_q_rows: int, max_q_len: int = 64,
                 max_cands: int = 0, max_k: int = 0):
        h = ctypes.c_void_p()
        _check(lib.gem_workspace_create(store.handle, max_queries, max_q_rows, max_q_len, max_cands,
                                        max_k, ctypes.byref(h)))
        self.handle = h
        self.store = store
        self.max_k = max_k

    def status(self, stream=None) -> int:
        """Synchronise and return (then clear) the device status word."""
        return lib.gem_stream_status(self.handle, _stream(stream))

    def close(self):
        if self.handle:
            lib.gem_workspace_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _queries(q, q_offsets):
    q = _dev(q, torch.float32, "q")
    qo = _dev(q_offsets, torch.int64, "q_offsets")
    return q, qo, qo.numel() - 1, q.shape[0]


def score_all(store: Store, ws: Workspace, q, q_offsets, compute="bf16", out=None, stream=None):
    """Exact CH (Eq. 1) of every query set against every stored set: float32 [B, n_sets].
    compute: "bf16", "fp8" (per-vector scales), "fp8_set" (one power-of-two scale per
    set) on the tensor cores, from the store copy of that name; or "f32" (SIMT)."""
    q, qo, B, rows = _queries(q, q_offsets)
    if out is None:
        out = torch.empty((B, store.n_sets), dtype=torch.float32, device=q.device)
    _check(lib.gem_score_all(store.handle, ws.handle, _ptr(q), _ptr(qo), B, rows, _dtype_code(compute),
                             _ptr(out), _stream(stream)))
    return out


def score_ids(store: Store, ws: Workspace, q, q_offsets, cand_offsets, cand_ids, compute="f32",
              out=None, stream=None):
    """Exact CH over per-query candidate id lists (Algorithm 5 candidate scoring),
    aligned with cand_ids.  compute: "f32" (the FP32 chain, Kahan sum over query
    vectors) or "codes" (the qCH estimate in similarity form)."""
    q, qo, B, rows = _queries(q, q_offsets)
    co = _dev(cand_offsets, torch.int64, "cand_offsets")
    ci = _dev(cand_ids, torch.int64, "cand_ids")
    if out is None:
        out = torch.empty(ci.numel(), dtype=torch.float32, device=q.device)
    _check(lib.gem_score_ids(store.handle, ws.handle, _ptr(q), _ptr(qo), B, rows, _ptr(co), _ptr(ci),
                             ci.numel(), _dtype_code(compute), _ptr(out), _stream(stream)))
    return out


def rerank_pool(store: Store, ws: Workspace, q, q_offsets, pool_ids, out=None, stream=None):
    """Exact FP32 CH of a rerank pool (Algorithm 5's final rescoring): pool_ids
    int64 [n_queries, depth] (-1 = empty) -> float32 [n_queries, depth], the same
    scores as score_ids with "f32" over the rows as per-query lists."""
    q, qo, B, rows = _queries(q, q_offsets)
    pid = _dev(pool_ids, torch.int64, "pool_ids")
    if pid.dim() != 2 or pid.shape[0] != B:
        raise ValueError("pool_ids must be [n_queries, depth]")
    if out is None:
        out = torch.empty(pid.shape, dtype=torch.float32, device=q.device)
    _check(lib.gem_rerank_pool(store.handle, ws.handle, _ptr(q), _ptr(qo), B, rows, _ptr(pid), pid.shape[1],
                               _ptr(out), _stream(stream)))
    return out


def topk(ws: Workspace, scores, k: int, ids=None, row_offsets=None, stream=None):
    """Per-row top-k by (score desc, id asc): (ids int64 [rows, k], scores float32 [rows, k])."""
    scores = _dev(scores, torch.float32, "scores")
    if row_offsets is None:
        rows, cols = scores.shape
        ro = None
    else:
        ro = _dev(row_offsets, torch.int64, "row_offsets")
        rows, cols = ro.numel() - 1, 0
    if ids is not None:
        ids = _dev(ids, torch.int64, "ids")
    out_i = torch.empty((rows, k), dtype=torch.int64, device=scores.device)
    out_s = torch.empty((rows, k), dtype=torch.float32, device=scores.device)
    _check(lib.gem_topk(ws.handle, _ptr(scores), _ptr(ro), rows, cols, _ptr(ids), k, _ptr(out_i),
                        _ptr(out_s), _stream(stream)))
    return out_i, out_s


def search(store: Store, ws: Workspace, q, q_offsets, compute="bf16", rerank_depth=1000, k=100,
           stream=None):
    """Exhaustive search (Eq. 2): a first pass in `compute` ("bf16", "fp8", "fp8_set",
    "f32" or "codes"), its top rerank_depth per query rescored exactly in FP32, then
    the top k: (ids int64 [B, k], scores float32 [B, k]).  rerank_depth 0 returns
    the first pass's own top k."""
    q, qo, B, rows = _queries(q, q_offsets)
    out_i = torch.empty((B, k), dtype=torch.int64, device=q.device)
    out_s = torch.empty((B, k), dtype=torch.float32, device=q.device)
    _check(lib.gem_search(store.handle, ws.handle, _ptr(q), _ptr(qo), B, rows, _dtype_code(compute),
                          rerank_depth, k, _ptr(out_i), _ptr(out_s), _stream(stream)))
    return out_i, out_s


def search_host(store: Store, ws: Workspace, q_host, q_offsets_host, compute="bf16", rerank_depth=1000,
                k=100, out_ids=None, out_scores=None, stream=None):
    """search() with host tensors in and out (copies run inside the call)."""
    q = q_host.contiguous()
    qo = torch.as_tensor(q_offsets_host, dtype=torch.int64).contiguous()
    B = qo.numel() - 1
    if out_ids is None:
        out_ids = torch.empty((B, k), dtype=torch.int64, pin_memory=True)
    if out_scores is None:
        out_scores = torch.empty((B, k), dtype=torch.float32, pin_memory=True)
    _check(lib.gem_search_host(store.handle, ws.handle, _ptr(q), _ptr(qo), B, _dtype_code(compute),
                               rerank_depth, k, _ptr(out_ids), _ptr(out_scores), _stream(stream)))
    return out_ids, out_scores


TC_VARIANTS = {"plain": 0, "a_tmem": 1, "two_sets": 2}


def set_schedule(ws: Workspace, m_tiles: int = 2, chunk_rows: int = 1 << 16, variant: str = None):
    """Tensor-core kernel schedule of a workspace (results do not depend on it).
    variant: "plain", "a_tmem" (query rows in tensor memory) or "two_sets" (two
    sets of epilogue warps); the last two need m_tiles = 2."""
    if variant is None:
        variant = "plain"
    _check(lib.gem_workspace_set_schedule(ws.handle, m_tiles, TC_VARIANTS[variant], chunk_rows))


def qemd(store: Store, ws: Workspace, set_a, set_b, out=None, stream=None):
    """qEMD (Sec. 4.2.2, Eq. 14) of every pair (set_a[p], set_b[p]) of stored
    sets of at most 128 vectors: float32 [n_pairs].  Needs the store's codebook."""
    a = _dev(set_a.contiguous(), torch.int64, "set_a")
    b = _dev(set_b.contiguous(), torch.int64, "set_b")
    if a.numel() != b.numel():
        raise ValueError("set_a and set_b differ in length")
    if out is None:
        out = torch.empty(a.numel(), dtype=torch.float32, device=a.device)
    _check(lib.gem_qemd(store.handle, ws.handle, _ptr(a), _ptr(b), a.numel(), _ptr(out), _stream(stream)))
    return out


def selftest_wait_timeout(ws: Workspace, budget_cycles: int = 1 << 20, stream=None):
    """Run the bounded-wait self-test: a wait on a barrier nothing arrives on
    gives up after budget_cycles and records a timeout in ws's status word."""
    _check(lib.gem_selftest_wait_timeout(ws.handle, budget_cycles, _stream(stream)))


QCH_FORMS = {"symmetric": 0, "asymmetric": 1}
SIMS = {"ip": 0, "l2": 1}


def set_similarity(ws: Workspace, sim: str = "ip"):
    """Sim of Definition 1 for the exact scorers of this workspace: "ip" (inner
    product) or "l2" (negated L2 distance; FP32 scoring and rerank only)."""
    _check(lib.gem_workspace_set_similarity(ws.handle, SIMS[sim]))


def set_qch_form(ws: Workspace, form: str = "symmetric"):
    """Form of every qCH estimate through this workspace (estimate_codes,
    score_ids with "codes", beam_search): "symmetric" (both sides quantized, as
    Eq. 16 writes) or "asymmetric" (exact query vectors against the stored
    vectors' centroids)."""
    _check(lib.gem_workspace_set_qch_form(ws.handle, QCH_FORMS[form]))


def kmeans(x, k: int, iters: int = 10, seed: int = 0, stream=None):
    """Spherical k-means of the rows of x (e.g. C_quant -> C_index, the second
    clustering stage): float32 [k, 128] unit centroids."""
    x = _dev(x.contiguous(), torch.float32, "x")
    out = torch.empty((k, 128), dtype=torch.float32, device=x.device)
    _check(lib.gem_kmeans(_ptr(x), x.shape[0], k, iters, seed, _ptr(out), _stream(stream)))
    return out


def cluster_filter(q, q_offsets, centroids, t: int = 4, max_q_len: int = 32, stream=None):
    """C_query of every query set: (mask uint32 [B, ceil(k2/32)], ids int32
    [B, max_q_len * t] ascending, count int32 [B])."""
    q, qo, B, rows = _queries(q, q_offsets)
    c = _dev(centroids.contiguous(), torch.float32, "centroids")
    k2 = c.shape[0]
    mask = torch.empty((B, (k2 + 31) // 32), dtype=torch.int32, device=q.device)
    ids = torch.full((B, max_q_len * t), -1, dtype=torch.int32, device=q.device)
    count = torch.empty(B, dtype=torch.int32, device=q.device)
    _check(lib.gem_cluster_filter(_ptr(q), _ptr(qo), B, max_q_len, _ptr(c), k2, t, _ptr(mask), _ptr(ids),
                                  _ptr(count), _stream(stream)))
    return mask, ids, count


def set_index_centroids(store: Store, centroids, stream=None):
    """Attach C_index to the store: nearest coarse centroid of every stored vector
    and the member sets of every cluster."""
    c = _dev(centroids.contiguous(), torch.float32, "centroids")
    _check(lib.gem_store_set_index_centroids(store.handle, _ptr(c), c.shape[0], _stream(stream)))
    store.k2 = c.shape[0]


def mark_deleted(store: Store, ids, deleted: bool = True, stream=None):
    """Lazy deletion (Sec. 4.6): mark the sets `ids` deleted (or restore them with
    deleted=False).  Deleted sets are still scored and traversed by the beam
    search but never returned by topk, search or beam_search."""
    i = torch.as_tensor(ids).to(dtype=torch.int64, device="cuda").reshape(-1).contiguous()
    _check(lib.gem_store_mark_deleted(store.handle, _ptr(i), i.numel(), int(bool(deleted)), _stream(stream)))


def entry_points(store: Store, cluster_lists, cluster_counts, seed: int = 0, stream=None):
    """One random member set per cluster of each query's C_query (rows as from
    cluster_filter): int64 [B, stride], -1 for unused slots and empty clusters."""
    lists = _dev(cluster_lists.contiguous(), torch.int32, "cluster_lists")
    counts = _dev(cluster_counts.contiguous(), torch.int32, "cluster_counts")
    B, stride = lists.shape
    out = torch.empty((B, stride), dtype=torch.int64, device=lists.device)
    _check(lib.gem_entry_points(store.handle, _ptr(lists), _ptr(counts), B, stride, seed, _ptr(out),
                                _stream(stream)))
    return out


def beam_search(store: Store, ws: Workspace, q, q_offsets, graph_off, graph_nbrs, cluster_mask, entries,
                ef: int = 64, max_rounds: int = 1000, max_degree: int = None, stream=None):
    """Cluster-guided multi-path beam search (Algorithm 5) of every query over the
    graph (CSR over the stored sets): (ids int64 [B, ef], qsim float32 [B, ef],
    rounds)."""
    q, qo, B, rows = _queries(q, q_offsets)
    go = _dev(graph_off, torch.int64, "graph_off")
    gn = _dev(graph_nbrs, torch.int32, "graph_nbrs")
    if max_degree is None:
        max_degree = max(1, int((go[1:] - go[:-1]).max().item())) if go.numel() > 1 else 1
    mask = _dev(cluster_mask.contiguous(), torch.int32, "cluster_mask")
    ent = _dev(entries.contiguous(), torch.int64, "entries")
    out_i = torch.empty((B, ef), dtype=torch.int64, device=q.device)
    out_s = torch.empty((B, ef), dtype=torch.float32, device=q.device)
    rounds = ctypes.c_int32()
    _check(lib.gem_beam_search(store.handle, ws.handle, _ptr(q), _ptr(qo), B, rows, _ptr(go), _ptr(gn), max_degree,
                               _ptr(mask), _ptr(ent), ent.shape[1], ef, max_rounds, _ptr(out_i), _ptr(out_s),
                               ctypes.byref(rounds), _stream(stream)))
    return out_i, out_s, rounds.value


def assign_codes(x, centroids, with_best: bool = False, stream=None):
    """NN(x): index of the centroid with the largest inner product (ties: lowest)."""
    x = _dev(x, torch.float32, "x")
    c = _dev(centroids, torch.float32, "centroids")
    codes = torch.empty(x.shape[0], dtype=torch.int32, device=x.device)
    best = torch.empty(x.shape[0], dtype=torch.float32, device=x.device) if with_best else None
    _check(lib.gem_assign_codes(_ptr(x), x.shape[0], _ptr(c), c.shape[0], _ptr(codes), _ptr(best),
                                _stream(stream)))
    return (codes, best) if with_best else codes


def train_codebook(store: Store, k1: int, iters: int = 10, sample: int = 0, seed: int = 0, stream=None):
    """Stage-1 spherical k-means on (a sample of) the store's vectors: float32 [k1, 128]."""
    out = torch.empty((k1, 128), dtype=torch.float32, device="cuda")
    _check(lib.gem_train_codebook(store.handle, k1, iters, sample, seed, _ptr(out), _stream(stream)))
    return out


def set_codebook(store: Store, centroids, stream=None):
    """Attach C_quant to the store and code every stored vector."""
    c = _dev(centroids, torch.float32, "centroids")
    _check(lib.gem_store_set_codebook(store.handle, _ptr(c), c.shape[0], _stream(stream)))
    store.k1 = c.shape[0]


def estimate_codes(store: Store, ws: Workspace, q, q_offsets, cand_offsets=None, cand_ids=None, out=None,
                   stream=None):
    """qCH estimate (Eq. 16) in similarity form, all sets [B, n_sets] or per candidate id."""
    q, qo, B, rows = _queries(q, q_offsets)
    if cand_offsets is None:
        co = ci = None
        n = 0
        shape = (B, store.n_sets)
    else:
        co = _dev(cand_offsets, torch.int64, "cand_offsets")
        ci = _dev(cand_ids, torch.int64, "cand_ids")
        n = ci.numel()
        shape = (n,)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=q.device)
    _check(lib.gem_estimate_codes(store.handle, ws.handle, _ptr(q), _ptr(qo), B, rows, _ptr(co), _ptr(ci), n,
                                  _ptr(out), _stream(stream)))
    return out


class Batch:
    """Batched candidate scoring of many queries in one persistent, graph-replayed
    launch (the scoring step of a beam-search expansion, Algorithm 5).

    The batch owns torch tensors at fixed addresses (q, q_offsets, cand_offsets,
    cand_ids, scores); run() copies a round's inputs into them and launches.
    """

    def __init__(self, store: Store, mode="f32", max_queries=4096, max_q_rows=4096 * 64, max_q_len=64,
                 max_cands=4096 * 512, seg=32, ctas_per_sm=0):
        dev = torch.device("cuda")
        self.store = store
        self.mode = {"f32": 0, "codes": 3}[mode] if isinstance(mode, str) else int(mode)
        self.q = torch.zeros((max_q_rows, 128), dtype=torch.float32, device=dev)
        self.q_offsets = torch.zeros(max_queries + 1, dtype=torch.int64, device=dev)
        self.cand_offsets = torch.zeros(max_queries + 1, dtype=torch.int64, device=dev)
        self.cand_ids = torch.zeros(max(max_cands, 1), dtype=torch.int64, device=dev)
        self.scores = torch.zeros(max(max_cands, 1), dtype=torch.float32, device=dev)
        h = ctypes.c_void_p()
        _check(lib.gem_batch_create(store.handle, self.mode, max_queries, max_q_rows, max_q_len, max_cands, seg,
                                    ctas_per_sm, _ptr(self.q), _ptr(self.q_offsets), _ptr(self.cand_offsets),
                                    _ptr(self.cand_ids), _ptr(self.scores), ctypes.byref(h)))
        self.handle = h

    def run(self, q, q_offsets, cand_offsets, cand_ids, use_graph=True, stream=None):
        """Score one round; returns a view of the scores (valid until the next run)."""
        B = q_offsets.numel() - 1
        R, n = q.shape[0], cand_ids.numel()
        self.q[:R].copy_(q, non_blocking=True)
        self.q_offsets[:B + 1].copy_(q_offsets, non_blocking=True)
        self.cand_offsets[:B + 1].copy_(cand_offsets, non_blocking=True)
        self.cand_ids[:n].copy_(cand_ids, non_blocking=True)
        _check(lib.gem_batch_run(self.handle, B, R, n, 1 if use_graph else 0, _stream(stream)))
        return self.scores[:n]

    def status(self) -> int:
        return lib.gem_batch_status(self.handle)

    def close(self):
        if self.handle:
            lib.gem_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def maxsim_fwd(q, q_offsets, docs, doc_offsets, pair_offsets, pair_ids, compute="bf16", max_q_len=None,
               ws=None, stream=None):
    """Scores of (query, set) pairs and the argmax rows j*(t, i) (int32 [n_pairs, max_q_len])."""
    q, qo, B, _ = _queries(q, q_offsets)
    docs = _dev(docs, torch.float32, "docs")
    do = _dev(doc_offsets, torch.int64, "doc_offsets")
    po = _dev(pair_offsets, torch.int64, "pair_offsets")
    pid = _dev(pair_ids, torch.int64, "pair_ids")
    if max_q_len is None:
        max_q_len = int((qo[1:] - qo[:-1]).max().item())
    n = pid.numel()
    scores = torch.empty(n, dtype=torch.float32, device=q.device)
    argmax = torch.empty((n, max_q_len), dtype=torch.int32, device=q.device)
    _check(lib.gem_maxsim_fwd(_ptr(q), _ptr(qo), B, q.shape[0], _ptr(docs), _ptr(do), do.numel() - 1, docs.shape[0],
                              _ptr(po), _ptr(pid), n, max_q_len, _dtype_code(compute), _ptr(scores), _ptr(argmax),
                              ws.handle if ws is not None else None, _stream(stream)))
    return scores, argmax


def maxsim_bwd(q, q_offsets, docs, doc_offsets, pair_offsets, pair_ids, argmax, grad_scores, stream=None):
    """(grad_q, grad_docs) of the pair scores for upstream gradients grad_scores."""
    q, qo, B, _ = _queries(q, q_offsets)
    g = _dev(grad_scores.contiguous(), torch.float32, "grad_scores")
    grad_q = torch.empty_like(q)
    grad_d = torch.empty_like(docs)
    _check(lib.gem_maxsim_bwd(_ptr(q), _ptr(qo), B, _ptr(docs), _ptr(doc_offsets), doc_offsets.numel() - 1,
                              docs.shape[0], _ptr(pair_offsets), _ptr(pair_ids), pair_ids.numel(), _ptr(argmax),
                              argmax.shape[1], _ptr(g), _ptr(grad_q), _ptr(grad_d), _stream(stream)))
    return grad_q, grad_d


def measure_peaks(stream=None) -> dict:
    """Measured FP32 FMA peak (TFLOP/s) and L2-resident 128-byte gather bandwidth
    (GB/s) of the current GPU: the roofline denominators of the FP32 scorers and
    the qCH table lookups."""
    f, g = ctypes.c_float(), ctypes.c_float()
    _check(lib.gem_measure_peaks(ctypes.byref(f), ctypes.byref(g), _stream(stream)))
    return {"fp32_tflops": f.value, "l2_gather_gbs": g.value}


class MaxSimFn(torch.autograd.Function):
    """Differentiable pair scores S_t = CH(Q_b, P_d) (Eq. 1) with the library's
    forward (argmax side output) and hand-written backward."""

    @staticmethod
    def forward(ctx, q, docs, q_offsets, doc_offsets, pair_offsets, pair_ids, compute="bf16"):
        scores, argmax = maxsim_fwd(q.detach().contiguous(), q_offsets, docs.detach().contiguous(), doc_offsets,
                                    pair_offsets, pair_ids, compute)
        ctx.save_for_backward(q, docs, q_offsets, doc_offsets, pair_offsets, pair_ids, argmax)
        return scores

    @staticmethod
    def backward(ctx, g):
        q, docs, qo, do, po, pid, argmax = ctx.saved_tensors
        gq, gd = maxsim_bwd(q.detach().contiguous(), qo, docs.detach().contiguous(), do, po, pid, argmax, g)
        return gq, gd, None, None, None, None, None


def autotune_score_all(store: Store, ws: Workspace, q, q_offsets, compute="bf16", scores=None, cache_path=None,
                       stream=None):
    """Pick and apply the fastest tensor-core schedule:
    dict(m_tiles, variant, chunk_rows, ms, from_cache)."""
    q, qo, B, rows = _queries(q, q_offsets)
    if scores is None:
        scores = torch.empty((B, store.n_sets), dtype=torch.float32, device=q.device)
    mt, at, cr, fc = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    ms = ctypes.c_float()
    _check(lib.gem_autotune_score_all(store.handle, ws.handle, _ptr(q), _ptr(qo), B, rows, _dtype_code(compute),
                                      _ptr(scores), cache_path.encode() if cache_path else None, ctypes.byref(mt),
                                      ctypes.byref(at), ctypes.byref(cr), ctypes.byref(ms), ctypes.byref(fc),
                                      _stream(stream)))
    names = {v: k for k, v in TC_VARIANTS.items()}
    return {"m_tiles": mt.value, "variant": names[at.value], "chunk_rows": cr.value, "ms": ms.value,
            "from_cache": bool(fc.value)}


def autotune_batch(store: Store, q, q_offsets, cand_offsets, cand_ids, mode="f32", max_q_len=64, cache_path=None,
                   stream=None):
    """Fastest (seg, ctas_per_sm) of a Batch on one representative round."""
    q = _dev(q.contiguous(), torch.float32, "q")
    qo = _dev(q_offsets, torch.int64, "q_offsets")
    co = _dev(cand_offsets, torch.int64, "cand_offsets")
    ci = _dev(cand_ids, torch.int64, "cand_ids")
    scores = torch.empty(ci.numel(), dtype=torch.float32, device=q.device)
    sg, ct, fc = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    ms = ctypes.c_float()
    m = {"f32": 0, "codes": 3}[mode] if isinstance(mode, str) else int(mode)
    _check(lib.gem_autotune_batch(store.handle, m, qo.numel() - 1, q.shape[0], max_q_len, ci.numel(), _ptr(q),
                                  _ptr(qo), _ptr(co), _ptr(ci), _ptr(scores),
                                  cache_path.encode() if cache_path else None, ctypes.byref(sg), ctypes.byref(ct),
                                  ctypes.byref(ms), ctypes.byref(fc), _stream(stream)))
    return {"seg": sg.value, "ctas_per_sm": ct.value, "ms": ms.value, "from_cache": bool(fc.value)}
