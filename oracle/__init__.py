"""Plain, slow FP64 CPU oracle for GEM's multi-vector scoring path (arXiv 2603.20336).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
benchmark's CPU-baseline leg may import this package; the product path (the CUDA
library and its Python binding) never does, and this package never imports the
product.  Each function restates one definition of the paper in float64 with
numpy; a library matmul or sort may serve as a step, with no blocking or
reordering beyond a loop over documents.

Contents and the passage each follows:
  chamfer, score_all, score_ids   Sec. 3.1, Definition 1 (Eq. 1), Sim = inner product
  chamfer_l2, score_all_l2        Definition 1 with Sim = -(L2 distance)
  topk                            Sec. 3.1, problem statement (Eq. 2); ties by lower id
  rerank                          Algorithm 5, final step: exact CH over a candidate pool
  assign_codes                    Sec. 4.1.1 / Sec. 4.2.2: NN(x) = nearest centroid of C_quant
  cluster_filter                  Sec. 4.5.1, Eq. 15: C_query = union of each query vector's top-t of C_index
  cluster_members, entry_points   Sec. 4.1.1 Eq. 4 (C(P)) and Sec. 4.5.2 / Algorithm 5: one random set per
                                  cluster of C_query (SplitMix64-based draw, splitmix64_next / entry_hash)
  beam_search                     Algorithm 5 / Sec. 4.5.3: cluster-guided multi-path beam search, in rounds
  qch_distance, qch_similarity    Sec. 4.5.3, Eq. 16, with d_X = 1 - <.,.> (Sec. 4.2.1)
  qch_asym_*                      Eq. 16 with only the stored side quantized (a variant)
  emd_cost, emd, qemd             Sec. 4.2.1-4.2.2 (Eq. 11-14): EMD with uniform marginals, exact LP (HiGHS)
  k1_for                          Sec. 5.1 parameter settings: |C_quant| = 2^floor(log2(16 sqrt(#vectors)))
  bf16_round, fp8_e4m3_quantize, fp8_e4m3_quantize_sets
                                  storage formats of the low-precision path (not in the paper)
  maxsim_grad, contrastive_*      gradient of Eq. 1 (not in the paper)
  kmeans_update                   Sec. 4.1.1, one Lloyd update of the stage-1 k-means

Pinned by tests/test_oracle_pins.py against brute force, closed forms, invariants
and the paper's worked example.  kmeans_update (one Lloyd update given the
assignment) is pinned by hand examples with exact answers, an empty centroid and
a zero-sum centroid included; the k-means iteration as a whole (initial centroids,
number of iterations) is a heuristic and is not oracled.
"""
from .maxsim import (  # noqa: F401
    chamfer, score_all, score_ids, chamfer_l2, score_all_l2, topk, rerank, recall_at_k,
    assign_codes, cluster_filter, cluster_members, entry_points, entry_hash, splitmix64_next, beam_search,
    qch_distance, qch_similarity, qch_score_all, qch_score_ids, qch_asym_similarity, qch_asym_score_all, k1_for,
    emd_cost, emd, qemd,
    bf16_round, fp8_e4m3_round, fp8_e4m3_quantize, fp8_e4m3_quantize_sets,
    maxsim_grad, contrastive_loss, contrastive_dscores, kmeans_update,
)
