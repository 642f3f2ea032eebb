"""ctypes signatures of the C ABI in include/gem.h."""
import ctypes as C

P = C.c_void_p
I32 = C.c_int32
I64 = C.c_int64
U32 = C.c_uint32
SZ = C.c_size_t

SIGNATURES = {
    "gem_version": (C.c_int, []),
    "gem_last_error_message": (C.c_char_p, []),
    "gem_device_check": (C.c_int, [C.c_int]),
    "gem_store_create": (C.c_int, [P, P, I64, I32, U32, C.c_int, P, C.POINTER(P)]),
    "gem_store_destroy": (None, [P]),
    "gem_store_info": (C.c_int, [P, P, P, P, P]),
    "gem_store_export": (C.c_int, [P, I32, P, SZ, P]),
    "gem_store_codebook_sizes": (C.c_int, [P, P, P]),
    "gem_store_save": (C.c_int, [P, C.c_char_p, P]),
    "gem_store_load": (C.c_int, [C.c_char_p, U32, P, C.POINTER(P)]),
    "gem_assign_codes": (C.c_int, [P, I64, P, I32, P, P, P]),
    "gem_train_codebook": (C.c_int, [P, I32, I32, I64, C.c_uint64, P, P]),
    "gem_store_set_codebook": (C.c_int, [P, P, I32, P]),
    "gem_kmeans": (C.c_int, [P, I64, I32, I32, C.c_uint64, P, P]),
    "gem_cluster_filter": (C.c_int, [P, P, I32, I32, P, I32, I32, P, P, P, P]),
    "gem_store_set_index_centroids": (C.c_int, [P, P, I32, P]),
    "gem_store_mark_deleted": (C.c_int, [P, P, I64, I32, P]),
    "gem_workspace_set_qch_form": (C.c_int, [P, I32]),
    "gem_workspace_set_similarity": (C.c_int, [P, I32]),
    "gem_selftest_wait_timeout": (C.c_int, [P, I64, P]),
    "gem_qemd": (C.c_int, [P, P, P, P, I64, P, P]),
    "gem_entry_points": (C.c_int, [P, P, P, I32, I32, C.c_uint64, P, P]),
    "gem_beam_search": (C.c_int, [P, P, P, P, I32, I64, P, P, I32, P, P, I32, I32, I32, P, P, P, P]),
    "gem_estimate_codes": (C.c_int, [P, P, P, P, I32, I64, P, P, I64, P, P]),
    "gem_workspace_create": (C.c_int, [P, I32, I64, I32, I64, I32, C.POINTER(P)]),
    "gem_workspace_destroy": (None, [P]),
    "gem_workspace_set_schedule": (C.c_int, [P, I32, I32, I32]),
    "gem_score_all": (C.c_int, [P, P, P, P, I32, I64, I32, P, P]),
    "gem_score_ids": (C.c_int, [P, P, P, P, I32, I64, P, P, I64, I32, P, P]),
    "gem_rerank_pool": (C.c_int, [P, P, P, P, I32, I64, P, I32, P, P]),
    "gem_topk": (C.c_int, [P, P, P, I32, I64, P, I32, P, P, P]),
    "gem_search": (C.c_int, [P, P, P, P, I32, I64, I32, I32, I32, P, P, P]),
    "gem_search_host": (C.c_int, [P, P, P, P, I32, I32, I32, I32, P, P, P]),
    "gem_stream_status": (C.c_int, [P, P]),
    "gem_maxsim_fwd": (C.c_int, [P, P, I32, I64, P, P, I64, I64, P, P, I64, I32, I32, P, P, P, P]),
    "gem_maxsim_bwd": (C.c_int, [P, P, I32, P, P, I64, I64, P, P, I64, P, I32, P, P, P, P]),
    "gem_batch_create": (C.c_int, [P, I32, I32, I64, I32, I64, I32, I32, P, P, P, P, P, C.POINTER(P)]),
    "gem_batch_run": (C.c_int, [P, I32, I64, I64, I32, P]),
    "gem_batch_status": (C.c_int, [P]),
    "gem_batch_destroy": (None, [P]),
    "gem_kernel_launches": (I64, []),
    "gem_autotune_score_all": (C.c_int, [P, P, P, P, I32, I64, I32, P, C.c_char_p, P, P, P, P, P, P]),
    "gem_autotune_batch": (C.c_int, [P, I32, I32, I64, I32, I64, P, P, P, P, P, C.c_char_p, P, P, P, P, P]),
    "gem_score_ids_noalloc": (C.c_int, [P, P, P, I32, I64, I32, P, P, I64, P, P]),
    "gem_shard_ranges": (C.c_int, [P, I64, I32, P]),
    "gem_shard_first_pass": (C.c_int, [P, P, P, P, I32, I64, I32, I32, I64, P, P, P]),
    "gem_shard_rerank": (C.c_int, [P, P, P, P, I32, I64, P, I32, I64, P, P]),
    "gem_shard_score_ids": (C.c_int, [P, P, P, P, I32, I64, P, P, I64, I32, I64, P, P]),
    "gem_merge_topk": (C.c_int, [P, P, I32, I32, I32, I32, P, P, P]),
    "gem_measure_peaks": (C.c_int, [P, P, P]),
}


def declare(lib):
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
