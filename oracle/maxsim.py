"""FP64 reference definitions (test infrastructure only; see the package docstring).

All inputs are converted to float64 before any arithmetic.  Vector sets are given
CSR-packed: rows vecs[offsets[i]:offsets[i+1]] are the vectors of set i.
"""
from __future__ import annotations

import math

import numpy as np

# Rows of documents multiplied against one query at a time.  This only bounds
# memory: every document's score is computed independently of the others.
_DOC_ROWS_PER_STEP = 1 << 21


def _f64(x) -> np.ndarray:
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.asarray(x, dtype=np.float64)


def _i64(x) -> np.ndarray:
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.asarray(x, dtype=np.int64)


# ---------------------------------------------------------------------------
# Chamfer / MaxSim (Sec. 3.1, Definition 1, Eq. 1)
# ---------------------------------------------------------------------------

def chamfer(A, B) -> float:
    """CH(A, B) = sum over a in A of max over b in B of <a, b>.

    Definition 1 (Eq. 1) with Sim taken as the inner product, which is the cosine
    similarity on the unit-norm vectors every workload uses.
    """
    A = _f64(A)
    B = _f64(B)
    sims = A @ B.T                   # sims[i, j] = <a_i, b_j>
    return float(sims.max(axis=1).sum())


def score_all(q, q_offsets, vecs, offsets, with_l1: bool = False):
    """CH(Q_b, P_n) for every query set b and every stored set n: float64 [B, N].

    The multi-vector retrieval problem (Eq. 2) ranks every P in D by CH(Q, P);
    this returns all of those scores.  with_l1=True also returns
    sum_i |max_j <q_i, p_j>| per (b, n), the scale a relative error of the sum is
    measured against.
    """
    q = _f64(q)
    qo = _i64(q_offsets)
    off = _i64(offsets)
    n_sets = len(off) - 1
    out = np.empty((len(qo) - 1, n_sets), dtype=np.float64)
    l1 = np.empty_like(out) if with_l1 else None
    # group documents so that one matmul covers about _DOC_ROWS_PER_STEP rows
    groups = []
    d0 = 0
    while d0 < n_sets:
        d1 = int(np.searchsorted(off, off[d0] + _DOC_ROWS_PER_STEP, side="right")) - 1
        d1 = max(d1, d0 + 1)
        d1 = min(d1, n_sets)
        groups.append((d0, d1))
        d0 = d1
    for d0, d1 in groups:
        r0, r1 = int(off[d0]), int(off[d1])
        X = _f64(vecs[r0:r1])
        starts = off[d0:d1] - r0
        for b in range(len(qo) - 1):
            Q = q[qo[b]:qo[b + 1]]
            sims = Q @ X.T                                   # [m_q, rows]
            per_doc_max = np.maximum.reduceat(sims, starts, axis=1)   # max over each doc's rows
            out[b, d0:d1] = per_doc_max.sum(axis=0)          # sum over the query's vectors
            if with_l1:
                l1[b, d0:d1] = np.abs(per_doc_max).sum(axis=0)
    return (out, l1) if with_l1 else out


def chamfer_l2(A, B) -> float:
    """CH(A, B) of Definition 1 (Eq. 1) with Sim(a, b) = -||a - b||_2.

    Definition 1 names the L2 distance as the other usual choice of Sim; as a
    similarity it enters negated, so the maximum picks each a's nearest b:
    CH = -sum over a of min over b of ||a - b||_2.
    """
    A = _f64(A)
    B = _f64(B)
    diff = A[:, None, :] - B[None, :, :]         # [m_a, m_b, d]
    dist = np.sqrt((diff * diff).sum(axis=2))     # ||a_i - b_j||_2
    return float(-dist.min(axis=1).sum())


def score_all_l2(q, q_offsets, vecs, offsets, with_l1: bool = False):
    """chamfer_l2(Q_b, P_n) for every query set b and stored set n: float64 [B, N].
    with_l1=True also returns sum_i min_j ||q_i - p_j|| (= -score), the scale a
    relative error of the sum is measured against."""
    q = _f64(q)
    qo = _i64(q_offsets)
    off = _i64(offsets)
    out = np.empty((len(qo) - 1, len(off) - 1))
    for n in range(len(off) - 1):
        P = _f64(vecs[off[n]:off[n + 1]])
        for b in range(len(qo) - 1):
            out[b, n] = chamfer_l2(q[qo[b]:qo[b + 1]], P)
    return (out, -out) if with_l1 else out


def score_ids(q, q_offsets, vecs, offsets, cand_offsets, cand_ids) -> np.ndarray:
    """CH(Q_b, P_id) for each id of query b's candidate list (Algorithm 5, candidate scoring).

    Returns float64 aligned with cand_ids.  A negative id stands for "no candidate"
    and scores -inf.
    """
    q = _f64(q)
    qo = _i64(q_offsets)
    off = _i64(offsets)
    co = _i64(cand_offsets)
    ids = _i64(cand_ids)
    out = np.empty(len(ids), dtype=np.float64)
    for b in range(len(qo) - 1):
        Q = q[qo[b]:qo[b + 1]]
        for t in range(co[b], co[b + 1]):
            i = ids[t]
            out[t] = -np.inf if i < 0 else chamfer(Q, vecs[off[i]:off[i + 1]])
    return out


# ---------------------------------------------------------------------------
# top-k (Eq. 2) and the final exact rerank of Algorithm 5
# ---------------------------------------------------------------------------

def topk(scores, k: int, ids=None, exclude=None):
    """k-argmax of one row of scores: sorted by score descending, ties by lower id.
    exclude: ids never returned (sets deleted lazily, Sec. 4.6).

    Returns (ids int64 [min(k, n)], scores float64 [min(k, n)]).
    """
    s = _f64(scores)
    i = np.arange(len(s), dtype=np.int64) if ids is None else _i64(ids)
    if exclude is not None and len(exclude):
        keep = ~np.isin(i, np.asarray(list(exclude), dtype=np.int64))
        s, i = s[keep], i[keep]
    order = np.lexsort((i, -s))      # primary key: -score, secondary: id
    order = order[:k]
    return i[order], s[order]


def rerank(q, q_offsets, vecs, offsets, pool_ids, k: int):
    """Exact-CH rerank of each query's candidate pool, then top-k (Algorithm 5, last step).

    pool_ids: int64 [B, R] (negative entries are empty slots).
    Returns (ids int64 [B, k], scores float64 [B, k]); short rows are padded with
    id -1 and score -inf.
    """
    pool = _i64(pool_ids)
    B, R = pool.shape
    co = np.arange(B + 1, dtype=np.int64) * R
    s = score_ids(q, q_offsets, vecs, offsets, co, pool.reshape(-1)).reshape(B, R)
    out_i = np.full((B, k), -1, dtype=np.int64)
    out_s = np.full((B, k), -np.inf)
    for b in range(B):
        keep = pool[b] >= 0
        ii, ss = topk(s[b][keep], k, pool[b][keep])
        out_i[b, :len(ii)] = ii
        out_s[b, :len(ss)] = ss
    return out_i, out_s


def recall_at_k(found_ids, true_ids) -> float:
    """|found ∩ true| / |true| for one query (recall against the exact top-k)."""
    t = set(int(x) for x in np.asarray(true_ids).ravel() if x >= 0)
    f = set(int(x) for x in np.asarray(found_ids).ravel() if x >= 0)
    return len(t & f) / max(1, len(t))


# ---------------------------------------------------------------------------
# Codes and the quantized Chamfer estimate
# ---------------------------------------------------------------------------

def assign_codes(X, C) -> np.ndarray:
    """NN(x): index of the centroid of C_quant with the largest inner product with x.

    Sec. 4.1.1 assigns each vector to its nearest centroid; with unit-norm vectors
    and unit-norm centroids the nearest centroid under d_X = 1 - <x, c> (Sec. 4.2.1)
    is the one with the largest inner product.  Ties go to the lowest index.
    Returns int64 [n].
    """
    C = _f64(C)
    n = len(X)
    out = np.empty(n, dtype=np.int64)
    step = max(1, (1 << 24) // max(1, len(C)))
    for s in range(0, n, step):
        sims = _f64(X[s:s + step]) @ C.T
        out[s:s + step] = np.argmax(sims, axis=1)      # first maximum = lowest index
    return out


def cluster_filter(q, q_offsets, C_index, t: int):
    """C_query of every query set (Sec. 4.5.1, Eq. 15; Algorithm 5, first two steps).

    The relevance matrix S = C_index Q^T scores every coarse centroid against every
    query vector; each query vector keeps its top-t centroids (largest inner
    product, ties to the lower centroid index) and C_query is the union of those
    over the query's vectors.  Returns one sorted int64 array per query set.
    """
    C = _f64(C_index)
    Q = _f64(q)
    qo = _i64(q_offsets)
    idx = np.arange(len(C))
    out = []
    for b in range(len(qo) - 1):
        S = Q[qo[b]:qo[b + 1]] @ C.T          # [m_q, k2] = (C Q^T)^T
        chosen = set()
        for row in S:
            order = np.lexsort((idx, -row))   # score descending, then index ascending
            chosen.update(int(c) for c in order[:t])
        out.append(np.array(sorted(chosen), dtype=np.int64))
    return out


_MASK64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64_next(state: int):
    """One step of the SplitMix64 generator (Steele, Lea and Flood, 2014): the
    state advances by the golden-ratio increment and the output is the state put
    through the variant-13 finalizer.  Returns (new_state, output)."""
    state = (state + _GOLDEN) & _MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return state, z ^ (z >> 31)


def entry_hash(seed: int, b: int, c: int, s: int) -> int:
    """The counter-based draw behind the multi-entry choice: SplitMix64 outputs
    chained over the fields, H = out(out(out(seed + b) + c) + s) where out(x) is
    the output of one step from state x (all arithmetic mod 2^64)."""
    h = seed & _MASK64
    for v in (b, c, s):
        _, h = splitmix64_next((h + v) & _MASK64)
    return h


def cluster_members(index_codes, offsets, k2: int):
    """members(c) = the stored sets with at least one vector whose nearest C_index
    centroid is c (the set's cluster representation C(P), Sec. 4.1.1, Eq. 4).
    index_codes: int [n_vectors].  Returns k2 sorted int64 arrays."""
    codes = _i64(index_codes)
    off = _i64(offsets)
    set_of = np.repeat(np.arange(len(off) - 1), np.diff(off))
    pairs = np.unique(codes * (len(off) + 1) + set_of)
    cl, st = pairs // (len(off) + 1), pairs % (len(off) + 1)
    return [st[cl == c] for c in range(k2)]


def entry_points(query_clusters, members, seed: int):
    """E of Algorithm 5 (Sec. 4.5.2): one random set from every cluster of C_query.
    The draw for (query b, cluster c) is the member s with the smallest
    entry_hash(seed, b, c, s) (then the lower s): uniform over the members and
    independent of their order.  An empty cluster gives -1.  query_clusters: one
    int array of cluster ids per query.  Returns one int64 array per query."""
    out = []
    for b, cl in enumerate(query_clusters):
        seeds = []
        for c in np.asarray(cl, dtype=np.int64).tolist():
            m = members[c]
            if len(m) == 0:
                seeds.append(-1)
                continue
            seeds.append(min((entry_hash(seed, b, c, int(s)), int(s)) for s in m)[1])
        out.append(np.array(seeds, dtype=np.int64))
    return out


def beam_search(score, graph_off, graph_nbrs, set_clusters, query_clusters, entries, ef: int,
                max_rounds: int = 1 << 30, dead=()):
    """Cluster-guided multi-path beam search of one query (Algorithm 5, Sec. 4.5.3),
    in rounds: in every round each non-empty queue W_e pops its best set P (in
    entry order); if P scores below tau (the worst score in R once R holds ef sets,
    else -inf) W_e is emptied; otherwise every neighbour P' of P (in list order) that
    is not visited and shares a cluster with C_query is marked visited and queued
    for scoring.  After the round's expansions the new sets are scored and inserted,
    in the order they were queued, into their own W_e and into R.

    Scores are similarities (qsim = m_q - qCH: higher is closer).  "Better" means
    higher score, then lower set id; W_e and R keep the ef best.  score(s) gives the
    score of set s; set_clusters[s] is the set of clusters of s (C(P)) and
    query_clusters the clusters of C_query.  entries: the entry sets, in order
    (duplicates and -1 skipped).  dead: sets deleted lazily (Sec. 4.6), still
    traversed through their W_e but never placed in R.  Returns (R as a list of
    (score, id), best first, the number of rounds run).
    """
    import bisect

    def key(sc, sid):        # ascending key = better first
        return (-sc, sid)

    qc = set(int(c) for c in query_clusters)
    visited = set()
    R = []                   # sorted ascending by key
    queues = []
    for e in entries:
        e = int(e)
        if e < 0 or e in visited:
            continue
        visited.add(e)
        sc = score(e)
        queues.append([key(sc, e)])
        if e not in dead:
            bisect.insort(R, key(sc, e))
            del R[ef:]
    rounds = 0
    while any(queues) and rounds < max_rounds:
        rounds += 1
        tau = -R[ef - 1][0] if len(R) >= ef else -math.inf
        new = []             # (queue index, set)
        for qi, W in enumerate(queues):
            if not W:
                continue
            nsc, pid = W.pop(0)
            if -nsc < tau:
                W.clear()
                continue
            for nb in graph_nbrs[graph_off[pid]:graph_off[pid + 1]]:
                nb = int(nb)
                if nb in visited or not (set_clusters[nb] & qc):
                    continue
                visited.add(nb)
                new.append((qi, nb))
        for qi, nb in new:
            k = key(score(nb), nb)
            bisect.insort(queues[qi], k)
            del queues[qi][ef:]
            if nb not in dead:
                bisect.insort(R, k)
                del R[ef:]
    return [(-k[0], k[1]) for k in R], rounds


def qch_distance(q_codes, p_codes, C) -> float:
    """qCH(Q, P) = sum over q of min over p of d_X(NN(q), NN(p)) (Sec. 4.5.3, Eq. 16).

    d_X(x, y) = 1 - <x, y> (cosine form, Sec. 4.2.1); both sides are quantized to
    their codebook entries, as Eq. 16 writes NN(q) and NN(p).
    """
    C = _f64(C)
    a = C[_i64(q_codes)]
    b = C[_i64(p_codes)]
    dist = 1.0 - a @ b.T
    return float(dist.min(axis=1).sum())


def qch_similarity(q_codes, p_codes, C) -> float:
    """The similarity form of qCH: sum over q of max over p of <NN(q), NN(p)>.

    Equals m_q - qCH(Q, P) up to rounding; ranking by it is ranking by qCH.
    """
    C = _f64(C)
    a = C[_i64(q_codes)]
    b = C[_i64(p_codes)]
    return float((a @ b.T).max(axis=1).sum())


def qch_score_all(q_codes, q_offsets, p_codes, offsets, C) -> np.ndarray:
    """qch_similarity(Q_b, P_n) for every query b and stored set n: float64 [B, N]."""
    C = _f64(C)
    qo = _i64(q_offsets)
    off = _i64(offsets)
    pc = _i64(p_codes)
    qc = _i64(q_codes)
    starts = off[:-1]
    out = np.empty((len(qo) - 1, len(off) - 1))
    for b in range(len(qo) - 1):
        a = C[qc[qo[b]:qo[b + 1]]]
        table = a @ C.T                          # <C_{a_i}, C_c> for every centroid c
        sims = table[:, pc]                      # [m_q, rows]: <C_{a_i}, C_{NN(p_j)}>
        out[b] = np.maximum.reduceat(sims, starts, axis=1).sum(axis=0)
    return out


def qch_score_ids(q_codes, q_offsets, p_codes, offsets, cand_offsets, cand_ids, C) -> np.ndarray:
    """qch_similarity over each query's candidate list, aligned with cand_ids."""
    qo = _i64(q_offsets)
    off = _i64(offsets)
    pc = _i64(p_codes)
    qc = _i64(q_codes)
    co = _i64(cand_offsets)
    ids = _i64(cand_ids)
    out = np.empty(len(ids))
    for b in range(len(qo) - 1):
        for t in range(co[b], co[b + 1]):
            i = ids[t]
            out[t] = qch_similarity(qc[qo[b]:qo[b + 1]], pc[off[i]:off[i + 1]], C)
    return out


def qch_asym_similarity(Q, p_codes, C) -> float:
    """Asymmetric qCH in similarity form: sum over q of max over p of <q, NN(p)>.

    Only the stored side is quantized; the query vectors stay exact.  This is
    Eq. 16 with d_X(q, NN(p)) = 1 - <q, NN(p)> in place of d_X(NN(q), NN(p)), a
    variant of the estimate (Sec. 4.5.3 quantizes both sides).
    """
    Q = _f64(Q)
    b = _f64(C)[_i64(p_codes)]
    return float((Q @ b.T).max(axis=1).sum())


def qch_asym_score_all(q, q_offsets, p_codes, offsets, C) -> np.ndarray:
    """qch_asym_similarity(Q_b, P_n) for every query b and stored set n: float64 [B, N]."""
    C = _f64(C)
    q = _f64(q)
    qo = _i64(q_offsets)
    off = _i64(offsets)
    pc = _i64(p_codes)
    out = np.empty((len(qo) - 1, len(off) - 1))
    for b in range(len(qo) - 1):
        table = q[qo[b]:qo[b + 1]] @ C.T         # <q_i, C_c> for every centroid c
        sims = table[:, pc]                      # [m_q, rows]: <q_i, C_{NN(p_j)}>
        out[b] = np.maximum.reduceat(sims, off[:-1], axis=1).sum(axis=0)
    return out


def emd_cost(D, a=None, b=None) -> float:
    """Earth mover's distance for the cost matrix D [m1, m2] (Sec. 4.2.1, Eq. 11-12):
    min over plans T >= 0 with row sums a and column sums b of sum_ij T_ij D_ij.
    a, b default to the uniform marginals 1/m1 and 1/m2 of the paper.  The
    linear program is solved exactly by scipy's HiGHS solver (a library step)."""
    from scipy.optimize import linprog

    D = _f64(D)
    m1, m2 = D.shape
    a = np.full(m1, 1.0 / m1) if a is None else _f64(a)
    b = np.full(m2, 1.0 / m2) if b is None else _f64(b)
    # T flattened row-major: T_ij at i * m2 + j
    rows = np.zeros((m1, m1 * m2))
    cols = np.zeros((m2, m1 * m2))
    for i in range(m1):
        rows[i, i * m2:(i + 1) * m2] = 1.0
    for j in range(m2):
        cols[j, j::m2] = 1.0
    res = linprog(D.reshape(-1), A_eq=np.vstack([rows, cols]), b_eq=np.concatenate([a, b]),
                  bounds=(0, None), method="highs")
    if res.status != 0:
        raise RuntimeError(res.message)
    return float(res.fun)


def emd(P1, P2) -> float:
    """EMD(P1, P2) with d_X(p, p') = 1 - <p, p'> (the cosine form, Sec. 4.2.1)."""
    return emd_cost(1.0 - _f64(P1) @ _f64(P2).T)


def qemd(codes1, codes2, C) -> float:
    """qEMD(P1, P2) (Sec. 4.2.2, Eq. 14): EMD with every vector replaced by its
    nearest centroid of C_quant (Eq. 13), d_X(NN(p_i), NN(p'_j)) = 1 - <C_a_i, C_b_j>."""
    C = _f64(C)
    return emd_cost(1.0 - C[_i64(codes1)] @ C[_i64(codes2)].T)


def k1_for(n_vectors: int) -> int:
    """|C_quant| = 2^floor(log2(16 * sqrt(#vectors))) (Sec. 5.1, parameter settings)."""
    return 1 << int(math.floor(math.log2(16.0 * math.sqrt(n_vectors))))


# ---------------------------------------------------------------------------
# Storage formats of the low-precision path, written from the format definitions
# ---------------------------------------------------------------------------

def _round_to_format(x: np.ndarray, mant_bits: int, min_exp: int) -> np.ndarray:
    """Round float64 values to the nearest number with `mant_bits` fraction bits
    (normal exponent >= min_exp, subnormal spacing 2^(min_exp - mant_bits)),
    ties to even.  No overflow handling."""
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    _, e = np.frexp(ax)                 # ax = f * 2^e, f in [0.5, 1)
    e = e - 1                           # ax in [2^e, 2^(e+1))
    e = np.maximum(e, min_exp)
    quantum = np.ldexp(1.0, e - mant_bits)
    r = np.round(ax / quantum) * quantum     # np.round: half to even; the division is exact
    return np.copysign(r, x)


def bf16_round(x) -> np.ndarray:
    """float32 -> bfloat16 (8 exponent bits, 7 fraction bits), round to nearest even.

    Returned as float32 values.  Finite inputs only; results beyond the largest
    bfloat16 become +-inf.
    """
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    r = _round_to_format(x, 7, -126)
    r = np.where(np.abs(r) > 3.3895313892515355e38, np.copysign(np.inf, x), r)
    return r.astype(np.float32)


FP8_E4M3_MAX = 448.0


def fp8_e4m3_round(x) -> np.ndarray:
    """float -> FP8 E4M3 (4 exponent bits, bias 7, 3 fraction bits, no infinities),
    round to nearest even, saturating to +-448.  Returned as float64 values."""
    x = np.asarray(x, dtype=np.float64)
    r = _round_to_format(x, 3, -6)
    return np.clip(r, -FP8_E4M3_MAX, FP8_E4M3_MAX)


def fp8_e4m3_quantize(X):
    """Per-vector scaled E4M3 storage: s_j = max_k |x_jk| / 448 (FP32 division),
    code_jk = E4M3(x_jk / s_j) with the division in FP32, round to nearest even,
    saturating.  A zero vector gets s_j = 1.  Returns (codes float64 [n, d] holding
    the E4M3 values, scales float32 [n]); the dequantised vector is codes * scale."""
    X = np.asarray(X, dtype=np.float32)
    amax = np.abs(X).max(axis=1)
    scale = (amax / np.float32(FP8_E4M3_MAX)).astype(np.float32)
    scale = np.where(amax == 0, np.float32(1.0), scale).astype(np.float32)
    ratio = (X / scale[:, None]).astype(np.float32)         # IEEE float32 division
    return fp8_e4m3_round(ratio.astype(np.float64)), scale


def fp8_e4m3_quantize_sets(X, offsets):
    """Per-set scaled E4M3 storage: set n gets one scale s_n, the smallest power of
    two not below 2^-126 with max |x| over the set's rows <= 448 s_n (1 for an
    all-zero set); code = E4M3(x / s_n), round to nearest even.  Dividing by a
    power of two is exact, so the only rounding is E4M3's.  Returns (codes float64
    [n, d] holding the E4M3 values, set scales float32 [n_sets]); the dequantised
    row j of set n is codes[j] * s_n.  Because s_n > 0 is common to the set,
    max_j <q, codes_j * s_n> = s_n * max_j <q, codes_j> (Eq. 1's inner max)."""
    X = np.asarray(X, dtype=np.float32).astype(np.float64)
    off = _i64(offsets)
    scales = np.ones(len(off) - 1, dtype=np.float32)
    codes = np.zeros_like(X)
    for n in range(len(off) - 1):
        rows = X[off[n]:off[n + 1]]
        amax = np.abs(rows).max() if rows.size else 0.0
        if amax > 0:
            k = -126
            while amax > FP8_E4M3_MAX * 2.0 ** k:
                k += 1
            scales[n] = 2.0 ** k
        codes[off[n]:off[n + 1]] = fp8_e4m3_round(rows / float(scales[n]))
    return codes, scales


# ---------------------------------------------------------------------------
# Gradient of Eq. 1 and the contrastive loss used to exercise it
# ---------------------------------------------------------------------------

def maxsim_grad(Q, P, decide=None):
    """Gradients of CH(Q, P) = sum_i max_j <q_i, p_j> for a fixed argmax.

    j*(i) = argmax_j <q_i, p_j> (lowest j on ties); dCH/dq_i = p_{j*(i)} and
    dCH/dp_j = sum of q_i over the i with j*(i) = j.  Returns (dQ, dP, jstar).
    decide = (Qd, Pd): take the argmax on these inputs instead (a forward that
    rounds its inputs decides j* on the rounded values); the gradient values
    still come from Q and P.
    """
    Q = _f64(Q)
    P = _f64(P)
    Qd, Pd = (Q, P) if decide is None else (_f64(decide[0]), _f64(decide[1]))
    sims = Qd @ Pd.T
    jstar = np.argmax(sims, axis=1)
    dQ = P[jstar].copy()
    dP = np.zeros_like(P)
    np.add.at(dP, jstar, Q)
    return dQ, dP, jstar


def contrastive_loss(S, tau: float) -> float:
    """L = (1/B) sum_b CE(softmax(S_b / tau), target 0): the positive sits at column 0."""
    S = _f64(S) / tau
    m = S.max(axis=1, keepdims=True)
    lse = m[:, 0] + np.log(np.exp(S - m).sum(axis=1))
    return float(np.mean(lse - S[:, 0]))


def contrastive_dscores(S, tau: float) -> np.ndarray:
    """dL/dS[b, d] = (softmax(S_b / tau)[d] - [d == 0]) / (tau * B)."""
    S = _f64(S)
    B = S.shape[0]
    z = S / tau
    z = z - z.max(axis=1, keepdims=True)
    p = np.exp(z)
    p /= p.sum(axis=1, keepdims=True)
    p[:, 0] -= 1.0
    return p / (tau * B)


# ---------------------------------------------------------------------------
# Stage-1 k-means (Sec. 4.1.1): one Lloyd update given the assignment
# ---------------------------------------------------------------------------

def kmeans_update(X, codes, C_prev) -> np.ndarray:
    """One spherical Lloyd update: each centroid becomes the L2-normalised mean of
    the vectors assigned to it.  Where that mean cannot be normalised -- no vector
    is assigned, or the assigned vectors sum to the zero vector -- the centroid
    keeps its old value (the paper is silent; a zero centroid would have no
    direction for d_X = 1 - <.,.>)."""
    X = _f64(X)
    C_prev = _f64(C_prev)
    codes = _i64(codes)
    k, d = C_prev.shape
    sums = np.zeros((k, d))
    np.add.at(sums, codes, X)
    norms = np.linalg.norm(sums, axis=1)
    C = C_prev.copy()
    ok = norms > 0
    C[ok] = sums[ok] / norms[ok, None]
    return C
