"""Writes tests/golden/text500k_truth.npz: the exact FP64 top-100 of every one
of the 1,000 queries of the text-corpus workload (500,000 sets, lognormal
lengths, 4,096-centre mixture, seed 1236) over all 500,000 sets -- the ground
truth of the recall that bench.py reports.

It calls only the oracle: oracle.score_all (exact CH of Definition 1, Eq. 1, in
FP64) on disjoint ranges of sets in worker processes (each set's score depends on
that set alone), and oracle.topk (the k-argmax of Eq. 2, ties to the lower id)
on each query's full row.  The inputs come from synth.text_corpus with its
device-independent noise, so the file matches the data bench.py draws on the GPU;
the workload's fingerprint (synth.fingerprint) is stored with it and checked
before use.

    python tests/golden/make_text500k_truth.py [--procs 8] [--queries 1000]

Stored: ids int32 [Q, 100] (the exact top-100, best first), scores float64
[Q, 101] (the top-101 exact scores: the 101st tells a tie at the boundary),
fingerprint, seed, n_sets.  About half an hour on 8 host cores.
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

_G = {}


def _work(span):
    """Exact CH of every query against the sets [a, b), written into the shared matrix."""
    a, b = span
    X, off, Q, qo, S = _G["X"], _G["off"], _G["Q"], _G["qo"], _G["S"]
    r0, r1 = int(off[a]), int(off[b])
    S[:, a:b] = oracle.score_all(Q, qo, X[r0:r1], off[a:b + 1] - r0)
    return b - a


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count())
    ap.add_argument("--queries", type=int, default=1000)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "text500k_truth.npz"))
    args = ap.parse_args()
    t0 = time.time()
    import torch
    torch.set_num_threads(os.cpu_count())     # the data draw uses every core; the workers' BLAS one each
    w = synth.text_corpus(seed=1236, n_queries=args.queries, device="cpu")
    fp = synth.fingerprint(w.docs, w.queries)
    print(f"data drawn in {time.time() - t0:.0f} s, fingerprint {fp}", flush=True)
    n = w.docs.n_sets
    _G["X"] = w.docs.vecs.numpy()
    _G["off"] = w.docs.offsets
    _G["Q"] = w.queries.vecs.numpy()
    _G["qo"] = w.queries.offsets
    # the score matrix lives in shared memory the forked workers write into
    import mmap
    nbytes = args.queries * n * 8
    buf = mmap.mmap(-1, nbytes)
    _G["S"] = np.frombuffer(buf, dtype=np.float64).reshape(args.queries, n)
    spans = [(a, min(n, a + 4000)) for a in range(0, n, 4000)]
    done = 0
    with mp.get_context("fork").Pool(args.procs) as pool:
        for c in pool.imap_unordered(_work, spans):
            done += c
            if done % 50000 < 4000:
                print(f"{done}/{n} sets, {time.time() - t0:.0f} s", flush=True)
    S = _G["S"]
    ids = np.empty((args.queries, 100), np.int32)
    sc = np.empty((args.queries, 101), np.float64)
    for q in range(args.queries):
        ii, ss = oracle.topk(S[q], 101)
        ids[q] = ii[:100]
        sc[q] = ss
    np.savez_compressed(args.out, ids=ids, scores=sc, fingerprint=np.array(fp), seed=np.array(1236),
                        n_sets=np.array(n))
    print(f"wrote {args.out} in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
