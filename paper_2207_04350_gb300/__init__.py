"""GB300-native contig generation (Guidi et al., ICPP'22, Alg. 2) on one GPU.

The compute lives in libcg.so (hand-written CUDA for sm_103a behind the C ABI
of include/cg.h); `cg` is its thin Python binding.
"""
from .cg import (BORROW_DEVICE, HOST_READS, MAX_PARTS, MEM_DEVICE, MEM_HOST, NO_VALIDATE, WEIGHT_BASES, WEIGHT_READS, CgError,
                 Context, Graph, Server, cg_batch_ranges, cg_chains, cg_create, cg_destroy, cg_emit_contigs,
                 cg_emit_contigs_2bit, cg_free_graph, cg_get_stats, cg_get_tuning, cg_kernel_times, cg_load_batch, cg_load_graph,
                 cg_mask_branches, cg_offsets_noalloc, cg_partition_contigs, cg_set_fault, cg_set_graphs, cg_set_host_direct, cg_set_timing,
                 cg_set_tuning, cg_status_str, cg_sync, cg_transitive_reduction, chains_host, contigs_2bit_host, contigs_host, packed_bytes_2bit)

__all__ = ["BORROW_DEVICE", "HOST_READS", "MAX_PARTS", "MEM_DEVICE", "MEM_HOST", "NO_VALIDATE", "WEIGHT_BASES", "WEIGHT_READS",
           "CgError", "Context", "Graph", "Server", "cg_batch_ranges", "cg_chains", "cg_create", "cg_destroy",
           "cg_emit_contigs", "cg_emit_contigs_2bit", "cg_free_graph", "cg_get_stats", "cg_get_tuning", "cg_kernel_times", "cg_load_batch",
           "cg_load_graph", "cg_mask_branches", "cg_offsets_noalloc", "cg_partition_contigs", "cg_set_graphs",
           "cg_set_fault", "cg_set_host_direct",
           "cg_set_timing", "cg_set_tuning", "cg_status_str", "cg_sync", "cg_transitive_reduction", "chains_host", "contigs_2bit_host", "contigs_host",
           "packed_bytes_2bit"]
