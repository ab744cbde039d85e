/*
 * cg.h - contig generation on one GPU (GB300, sm_103a): the C ABI.
 *
 * The problem these calls solve is ContigGeneration(S, sequences) -> cset of
 * Guidi et al., "Distributed-Memory Parallel Contig Generation for De Novo
 * Long-Read Genome Assembly", ICPP'22 (Alg. 2): mask the branch reads of a
 * bidirected string graph S, group the remaining reads into linear chains,
 * walk each chain and concatenate the oriented read suffixes into contigs.
 *
 * Input format (cg_graph_desc):
 *   - reads 0..n-1; len[r] >= 1 bases; off[r] = first base of read r in one
 *     2-bit stream `packed` (A=0 C=1 G=2 T=3; base i is in byte i>>2 at bits
 *     2*(i&3)); reads may start at any base offset;
 *   - S as CSR: row_ptr[n+1] (int32 or int64), col[m] (int32), and per entry
 *     (u->v) code[m] = E_u | (E_v << 1), where E = 0 names the 5' end (first
 *     stored base) and E = 1 the 3' end of the stored read touched by the
 *     overlap (the bidirected arrows of Sec. 2), and suf[m] = number of bases
 *     of v, in walk orientation, beyond the overlap (the overhang weight of
 *     Sec. 2). The mirror entry (v->u) carries the swapped code.
 *   A read with orientation o (0 forward, 1 reverse complement) is entered
 *   through end o and left through end 1-o (a valid walk, Sec. 2).
 *
 * Output (canonical, identical to the CPU oracle byte for byte):
 *   - branch reads: degree >= 3 in S (Sec. 4.2), or exactly two overlaps to
 *     reads of degree <= 2 that touch the same end of the read;
 *   - one contig per linear chain of at least `min_chain_reads` reads, listed
 *     by the smallest read id of the chain; each is spelled from its
 *     smaller-id end read (oriented to leave through its one overlap), the
 *     first read whole, every later read by the suffix of the overlap used
 *     (Sec. 4.4); a closed chain starts at its smallest read, forward;
 *   - contig i occupies bases[contig_off[i], contig_off[i+1]) as ASCII A/C/G/T;
 *   - for a partition of the contigs (cg_partition_contigs, Sec. 4.3), one
 *     part alone: its contigs back to back in the same order (cg_emit_part).
 *
 * Ownership and ordering: the caller owns every buffer it passes. Calls on
 * one context are ordered on the context's CUDA stream; a context is not
 * thread-safe. A call whose count pointers are all NULL does not wait for the
 * GPU: errors found by its kernels are reported by the next call that waits
 * (cg_sync or any call given a count pointer). After CG_ETIMEOUT or
 * CG_EKERNEL every call on that context fails until cg_destroy.
 * Limits: n_reads < 2^30, n_entries < 2^31, a read shorter than 2^31 bases.
 */
#ifndef CG_H
#define CG_H
#include <stddef.h>
#include <stdint.h>
#if defined(__GNUC__)
#define CG_API __attribute__((visibility("default")))
#else
#define CG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CG_OK = 0,
  CG_EINVAL = 1,    /* bad argument: null, size, alignment, capacity too small */
  CG_ENOMEM = 2,    /* device memory or the context's HBM budget exhausted */
  CG_ECUDA = 3,     /* a CUDA runtime call failed */
  CG_EGRAPH = 4,    /* the input is not a valid string graph (see cg_load_graph) */
  CG_ETIMEOUT = 5,  /* a device-side wait ran past its iteration limit */
  CG_EBUSY = 6,     /* no room: admission refused (server) */
  CG_EKERNEL = 7    /* a kernel found an inconsistency it cannot continue from */
} cg_status;

enum { CG_MEM_HOST = 0, CG_MEM_DEVICE = 1 };

/* cg_load_graph flags */
enum {
  CG_BORROW_DEVICE = 1u, /* desc pointers are device memory used in place (must outlive the graph) */
  CG_NO_VALIDATE = 2u,   /* skip the input checks (only for graphs known to be valid) */
  CG_HOST_READS = 4u,    /* host inputs whose packed reads are pinned host memory: the reads stay
                            there (used in place, must outlive the graph) and the spelling reads
                            only the bases it spells, over the host link; the other arrays are
                            copied. CG_EINVAL when packed is not pinned host memory. */
  CG_NO_READS = 8u       /* the graph without its reads, for a run split over ranks that each
                            hold a slice of them (cg_exchange_*): packed must be NULL, off still
                            places every read in one virtual 2-bit stream of packed_bytes bytes
                            (any layout; the input checks hold reads to it). The mask, chain and
                            layout steps run as usual; the spelling calls other than
                            cg_emit_share_received refuse bases outputs with CG_EINVAL. */
};

typedef struct cg_ctx cg_ctx;
typedef struct cg_graph cg_graph;

typedef struct {
  int64_t n_reads;         /* n */
  int64_t n_entries;       /* m = row_ptr[n] */
  const void* row_ptr;     /* n+1 entries of row_ptr_bytes each */
  int32_t row_ptr_bytes;   /* 4 or 8 */
  int32_t mem;             /* CG_MEM_HOST or CG_MEM_DEVICE: where all pointers below live */
  const int32_t* col;      /* m */
  const uint8_t* code;     /* m, values 0..3 */
  const int32_t* suf;      /* m */
  const int32_t* len;      /* n */
  const int64_t* off;      /* n, base offsets into packed */
  const uint8_t* packed;   /* packed_bytes */
  int64_t packed_bytes;
  int32_t min_chain_reads; /* chains with fewer reads are not contigs; <= 0 means 2 (Sec. 4.4) */
  int32_t reserved;
  /* The x-drop form of the overlaps (Sec. 4.4), optional. When both are
   * non-NULL they replace suf (which may then be NULL) and each contig is
   * l_r[alpha : pre(e_0)] + l_c1[post(e_0) : pre(e_1)] + ... + l_r'[post : beta].
   * For entry (u->v): pre = index in stored u of u's last base before the
   * overlap in walk direction, in [0, len[u]-1]; post = index in stored v of
   * v's first base of the overlap, in [0, len[v]-1]. A read piece whose end
   * comes before its start in walk direction adds no bases. */
  const int32_t* pre;      /* m */
  const int32_t* post;     /* m */
} cg_graph_desc;

/* Create a context on CUDA device `device`. hbm_budget_bytes caps the device
 * memory the context allocates for graphs and scratch (0 = no cap).
 * cuda_stream: a cudaStream_t to order all work on, or NULL for a private
 * non-blocking stream. */
CG_API cg_status cg_create(cg_ctx** ctx, int device, uint64_t hbm_budget_bytes, void* cuda_stream);
CG_API cg_status cg_destroy(cg_ctx* ctx);

/* Load one string graph (Alg. 2 input S, sequences). Copies host or device
 * inputs into context-owned device memory, or with CG_BORROW_DEVICE uses the
 * caller's device buffers in place (16-byte aligned `packed`). Unless
 * CG_NO_VALIDATE is given, checks on the GPU that: row_ptr starts at 0, never
 * decreases and ends at m; 0 <= col < n and col != row; code <= 3; no pair
 * appears twice in a row; every entry has exactly one mirror entry with the
 * swapped code; 1 <= suf(u->v) <= len[v]-1; len >= 1; each read lies inside
 * the packed stream. A failed check returns CG_EGRAPH and no graph. Waits for
 * the GPU. */
CG_API cg_status cg_load_graph(cg_ctx* ctx, const cg_graph_desc* desc, uint32_t flags, cg_graph** out);
CG_API cg_status cg_free_graph(cg_graph* g);

/* The batched form: k string graphs loaded as one disjoint union (reads,
 * entries and packed bases of graph j follow those of graphs 0..j-1), so
 * that each stage below runs as one launch over every graph. All descs must
 * share mem, row_ptr_bytes and min_chain_reads; inputs are copied
 * (CG_BORROW_DEVICE is refused), except with CG_HOST_READS: host descs whose
 * packed reads are pinned host memory, 4-byte aligned, keep them there, and
 * each spelling call first gathers the words of the pieces it spells from the
 * owning graph's stream over the host link (CG_EINVAL when a graph's reads
 * are not pinned). Host inputs that are all pinned memory are read in place
 * by one copy kernel; other host inputs are copied array by array. Chains
 * never cross graphs, so the union's
 * contigs are those of graph 0, then graph 1, ... in each graph's own order,
 * and read r of graph j is read R_j + r of the union (R_j = reads of graphs
 * before j). Waits for the GPU. */
CG_API cg_status cg_load_batch(cg_ctx* ctx, const cg_graph_desc* descs, int k, uint32_t flags, cg_graph** out);
/* For a batch: first_contig[j] / first_base[j] = index of graph j's first
 * contig / its first base in the union's contig_off / bases; entry k holds
 * the totals. Each optional (k+1 entries in `mem`). Runs the earlier stages
 * if needed; waits for the GPU with host outputs. */
CG_API cg_status cg_batch_ranges(cg_graph* g, int64_t* first_contig, int64_t* first_base, int mem);

/* ------------------------------------------------------------- serving
 * A request loop over the batched form. Each request is one string graph
 * in host memory (its buffers must stay valid until the request is done).
 * Requests are admitted while the sum of their device-memory estimates
 * (2 x packed bytes + 400 B per read + 16 B per CSR entry + 1 MiB) stays
 * within hbm_budget_bytes; a request that alone exceeds it is refused with
 * CG_EBUSY. `workers` threads, each with its own context and stream, take
 * every admitted request waiting at that moment (at most max_batch) as one
 * batch (continuous batching), so batches overlap on the device. Each
 * worker's device output buffers come from a stream-ordered memory pool, so
 * a growing batch never synchronises the device. Results stay in
 * server-owned host memory until cg_server_release. */
typedef struct cg_server cg_server;
typedef struct {
  int32_t max_batch;          /* requests per batch, >= 1 */
  int32_t workers;            /* batches in flight, 1..16 */
  uint64_t hbm_budget_bytes;  /* admission budget, > 0 */
} cg_server_opts;
typedef struct {
  cg_status status;
  int32_t batch_size;         /* requests in the batch this one ran in */
  int64_t n_contigs, total_bases;
  const int64_t* contig_off;  /* n_contigs + 1 */
  const uint8_t* bases;       /* total_bases ASCII */
  int64_t t_submit_ns, t_start_ns, t_done_ns;  /* steady clock */
} cg_server_result;
CG_API cg_status cg_server_start(int device, const cg_server_opts* opts, cg_server** out);
CG_API cg_status cg_server_submit(cg_server* s, const cg_graph_desc* desc, uint64_t* id);
CG_API cg_status cg_server_poll(cg_server* s, uint64_t id, int* done);
/* Waits up to timeout_ms (< 0: no limit); CG_ETIMEOUT if not done by then. */
CG_API cg_status cg_server_wait(cg_server* s, uint64_t id, int64_t timeout_ms, cg_server_result* out);
CG_API cg_status cg_server_release(cg_server* s, uint64_t id);
CG_API cg_status cg_server_stats(cg_server* s, uint64_t* batches, uint64_t* requests, uint64_t* in_flight_bytes);
/* Kernels the server's contexts have launched so far (exact while no batch runs). */
CG_API cg_status cg_server_kernels(cg_server* s, uint64_t* launched);
/* Contexts the workers have replaced so far: a worker whose context returns
 * CG_ECUDA, CG_ETIMEOUT or CG_EKERNEL (after which a context refuses all
 * work) destroys it and creates a fresh one on the same stream before its
 * next batch. The requests of the failed batch report that status; later
 * batches run normally. A batch that fails with CG_EGRAPH or CG_EINVAL (one
 * malformed request makes the whole union fail) is run again one request at
 * a time, so that only the malformed requests report the error. */
CG_API cg_status cg_server_contexts_replaced(cg_server* s, uint64_t* replaced);
/* Finishes every submitted request, then stops the workers. */
CG_API cg_status cg_server_stop(cg_server* s);

/* BranchRemoval (Alg. 2; Sec. 4.2). is_branch: NULL or n bytes (1 = branch),
 * in `mem`. n_branch: NULL or receives the count (waits for the GPU).
 * Asked for neither (and with CUDA graphs on, no per-kernel timing), the call
 * only records that the step is due: its kernels are launched by the next call
 * on the graph, in one CUDA graph with that call's own stages when it spells
 * into device buffers. The same holds for cg_chains asked for nothing. */
CG_API cg_status cg_mask_branches(cg_graph* g, uint8_t* is_branch, int mem, int64_t* n_branch);

/* ConnectedComponent + the walk order of every chain (Alg. 2; Sec. 4.2, 4.4).
 * Runs the mask first. Per read, in `mem`, each optional: chain_id = smallest
 * read id of its chain, rank = position in the contig's walk, orient = 0
 * forward / 1 reverse complement; reads in no contig get -1, -1, 255.
 * n_contigs and n_cycles (closed chains) are optional and make the call wait. */
CG_API cg_status cg_chains(cg_graph* g, int32_t* chain_id, int32_t* rank, uint8_t* orient, int mem,
                    int64_t* n_contigs, int64_t* n_cycles);

/* LocalAssembly (Alg. 2; Sec. 4.4): spells every contig. Runs the earlier
 * steps first. contig_off: NULL or contig_off_cap >= n_contigs+1 entries.
 * bases: NULL or bases_cap >= total bases, 16-byte aligned when in device
 * memory. With both NULL only the sizes are computed (two-call size query).
 * A capacity that is too small gives CG_EINVAL and nothing is written; with
 * device outputs and no count pointers that check happens on the GPU and is
 * reported by the next waiting call. */
CG_API cg_status cg_emit_contigs(cg_graph* g, int64_t* contig_off, int64_t contig_off_cap, uint8_t* bases,
                          int64_t bases_cap, int mem, int64_t* n_contigs, int64_t* total_bases);

/* LocalAssembly (Alg. 2; Sec. 4.4) into a 2-bit stream: the same contigs as
 * cg_emit_contigs, base i of the stream at byte i >> 2, bits 2 (i & 3),
 * A=0 C=1 G=2 T=3 (the convention of the packed reads); contig c is bases
 * [contig_off[c], contig_off[c+1]). packed_out: NULL or packed_cap >=
 * 16 * ceil(total_bases / 64) bytes (whole 16-byte chunks; bits past the last
 * base are 0), 16-byte aligned when in device memory. Sizes, capacities and
 * errors as for cg_emit_contigs. */
CG_API cg_status cg_emit_contigs_2bit(cg_graph* g, int64_t* contig_off, int64_t contig_off_cap, uint8_t* packed_out,
                               int64_t packed_cap, int mem, int64_t* n_contigs, int64_t* total_bases);

/* TransitiveReduction (Alg. 1, S <- TransitiveReduction(R); Sec. 2): the
 * string graph S of an overlap graph R given in the suffix form (rows sorted
 * by column; d->len is read, d->off and d->packed are not). An entry (u->w) is
 * transitive when some read v gives a valid walk u -> v -> w that leaves u and
 * enters w through the same ends as (u->w), passes through v (one end in, the
 * other out), and whose suffixes add up to suf(u->w) within +-fuzz; a pair of
 * reads keeps both entries only when neither is transitive. Output: S's CSR
 * with int64 row_ptr (n+1) and up to cap_entries entries of col, code, suf
 * (rows keep their order), all in `mem`. With all outputs NULL only
 * *n_entries is set (two-call size query); a cap below the count gives
 * CG_EINVAL and writes nothing. Device inputs are read in place during the
 * call, host inputs are copied; the call waits for the GPU. An invalid R
 * (unsorted or repeated columns, bad offsets, codes, suffixes or mirrors)
 * gives CG_EGRAPH. S keeps R's reads, so a descriptor with S's arrays and R's
 * reads goes to cg_load_graph. */
CG_API cg_status cg_transitive_reduction(cg_ctx* ctx, const cg_graph_desc* overlaps, int32_t fuzz, int64_t* row_ptr,
                                  int32_t* col, uint8_t* code, int32_t* suf, int64_t cap_entries, int mem,
                                  int64_t* n_entries);

/* GreedyPartitioning (Alg. 2; Sec. 4.3): splits the contigs among n_parts
 * parts (processes, GPUs) with the longest-processing-time rule. Each contig
 * weighs its number of reads (weight CG_WEIGHT_READS, the size estimate of
 * Sec. 4.3) or its spelled bases (CG_WEIGHT_BASES). Contigs are taken by
 * weight, heaviest first, equal weights in contig order (the order of
 * cg_emit_contigs), and each goes to the part whose weight sum is smallest so
 * far, the lowest part index on ties. Runs the earlier steps first and waits
 * for the GPU. part: part_cap >= n_contigs entries, part[c] = part of contig
 * c; part_weight: n_parts entries, the weight sum of each part; both in `mem`.
 * n_parts in [1, CG_MAX_PARTS]; CG_EINVAL otherwise or when part_cap is too
 * small (nothing is written then). */
#define CG_WEIGHT_READS 0
#define CG_WEIGHT_BASES 1
#define CG_MAX_PARTS 1024
CG_API cg_status cg_partition_contigs(cg_graph* g, int32_t n_parts, int32_t weight, int32_t* part, int64_t part_cap,
                               int64_t* part_weight, int mem, int64_t* n_contigs);

/* Spells the contigs of one part only, as each process does with the contigs
 * assigned to it (Sec. 4.3-4.4): part[c] names the part of contig c (at least
 * n_contigs entries, in `mem`, e.g. from cg_partition_contigs; any int32
 * values), p the part to spell. The output holds the contigs c with
 * part[c] == p back to back in contig order, each exactly as cg_emit_contigs
 * spells it. contig_off (n_contigs + 1 entries) gives every contig's range in
 * that output: [contig_off[c], contig_off[c+1]), empty for the contigs of other
 * parts. *n_contigs is the graph's contig count, *total_bases the part's
 * bases. Buffers, capacities, the two-call size query (NULL bases) and `mem`
 * follow cg_emit_contigs; part may be NULL only when the graph has no contigs.
 * Runs the earlier steps first. Not for a batch loaded with CG_HOST_READS
 * (CG_EINVAL). A later cg_emit_contigs or cg_partition_contigs lays out the
 * whole graph again. */
CG_API cg_status cg_emit_part(cg_graph* g, const int32_t* part, int64_t part_cap, int32_t p, int64_t* contig_off,
                              int64_t contig_off_cap, uint8_t* bases, int64_t bases_cap, int mem, int64_t* n_contigs,
                              int64_t* total_bases);

/* One share of the whole spelling, for a run over several GPUs or processes
 * that each hold the whole graph and its reads and split the LocalAssembly
 * work among themselves (Sec. 4.3-4.4). Where the paper gives each process
 * whole contigs (cg_partition_contigs + cg_emit_part), this call cuts the
 * output stream of cg_emit_contigs itself into n_shares runs of whole layout
 * tiles (the graph's: 4 KiB below 2^31 bases of reads, else 8 KiB; runs as
 * equal as the tiles allow) and spells share `share` only, so every share is
 * the same work whatever the contig sizes, and a contig may span two shares.
 * Output: bases[0 .. n_bases) = stream bytes [first_base, first_base +
 * n_bases); concatenating the shares 0..n_shares-1 gives the stream of
 * cg_emit_contigs. contig_off (optional, n_contigs + 1 entries) gets the
 * whole stream's contig offsets. Every share of one split must come from
 * graphs of the same reads (the same layout tile). bases: NULL (sizes only)
 * or bases_cap >= the share's size,
 * 16-byte aligned in device memory; first_base and n_bases are optional
 * (asking for them waits for the GPU). 0 <= share < n_shares, else
 * CG_EINVAL. Runs the earlier steps first. */
CG_API cg_status cg_emit_share(cg_graph* g, int32_t share, int32_t n_shares, int64_t* contig_off,
                               int64_t contig_off_cap, uint8_t* bases, int64_t bases_cap, int mem,
                               int64_t* first_base, int64_t* n_bases);

/* The read exchange of a run split over ranks that each hold only a slice of
 * the reads: the paper's read exchange (Sec. 4.3), for the split of
 * cg_emit_share. Rank r owns reads [read_first[r], read_first[r+1]) (host
 * array of n_shares + 1 entries, from 0 to n, never decreasing) and holds
 * their bases in a 2-bit stream of its own layout. Every rank loads the whole
 * graph with CG_NO_READS (its `off` placing reads in a virtual stream, the same
 * on every rank). For every share p, the pieces of p's output range whose reads
 * rank r owns travel from r to p, in walk order: each as the 32-bit words that
 * cover its stored bases in the virtual stream (from its lowest base / 16 to
 * its highest base / 16 + 1), so the receiver reads them exactly as it would
 * read the virtual stream. Per rank and step:
 *   1. cg_exchange_sizes: send_bytes[p] (to share p) and recv_bytes[r] (from
 *      rank r), host arrays of n_shares entries. Runs the earlier steps first
 *      and waits for the GPU.
 *   2. cg_exchange_pack: fills send_buf (device, 4-byte aligned, send_cap >=
 *      the sum of send_bytes) with the segments for shares 0, 1, ... in order,
 *      each send_bytes[p] long. my_packed (device, my_packed_bytes) holds this
 *      rank's reads; my_off[i] (device) is the first base of read
 *      read_first[rank] + i in it. Waits for the GPU.
 *   3. an all-to-all (outside the library) that delivers every rank's segment
 *      for this rank, laid end to end by source rank;
 *   4. cg_emit_share_received: with recv_buf (device, 4-byte aligned,
 *      recv_bytes = the sum of recv_bytes of step 1), spells this rank's share
 *      exactly as cg_emit_share(g, rank, n_shares, ...) spells it from the
 *      whole stream: bases[0 .. n_bases) = stream bytes [first_base, first_base
 *      + n_bases); contig_off (optional) gets the whole stream's offsets.
 *      Device outputs; bases 16-byte aligned; waits for the GPU.
 * CG_EINVAL for a graph not loaded with CG_NO_READS, bad bounds or sizes. */
CG_API cg_status cg_exchange_sizes(cg_graph* g, int32_t n_shares, const int64_t* read_first, int32_t rank,
                                   int64_t* send_bytes, int64_t* recv_bytes);
CG_API cg_status cg_exchange_pack(cg_graph* g, int32_t n_shares, const int64_t* read_first, int32_t rank,
                                  const uint8_t* my_packed, int64_t my_packed_bytes, const int64_t* my_off,
                                  uint8_t* send_buf, int64_t send_cap);
CG_API cg_status cg_emit_share_received(cg_graph* g, int32_t n_shares, const int64_t* read_first, int32_t rank,
                                        const uint8_t* recv_buf, int64_t recv_bytes, int64_t* contig_off,
                                        int64_t contig_off_cap, uint8_t* bases, int64_t bases_cap,
                                        int64_t* first_base, int64_t* n_bases);

/* Launch parameters of a context's kernels. None changes any output. */
typedef struct {
  int32_t ruler_log2;         /* list ranking: a read starts a sublist with probability 2^-ruler_log2, 1..12 */
  int32_t tile_bytes;         /* spelling: output a warp spells at a time, a power of two from 4096 to
                                 131072; 0 (the default): each launch chooses 4, 8, 16 or 32 KiB from
                                 its output, the largest that leaves every warp at least 8 of them */
  int32_t emit_blocks_per_sm; /* spelling: resident blocks per SM, 1..16 (at most what fits) */
  int32_t emit_block_threads; /* spelling: threads per block (the CTA size), 128, 256 or 512 */
} cg_tuning;

/* Sets the launch parameters (a field <= 0 keeps its value); CG_EINVAL for
 * values out of range. Applies to the next calls. */
CG_API cg_status cg_set_tuning(cg_ctx* ctx, const cg_tuning* t);
CG_API cg_status cg_get_tuning(cg_ctx* ctx, cg_tuning* out);

/* With graphs on (the default), each stage's kernel launches are captured
 * once into a CUDA graph per graph and set of buffers, sizes and launch
 * parameters, and replayed with one launch afterwards. Off: launched one by
 * one. Outputs are the same either way. */
CG_API cg_status cg_set_graphs(cg_ctx* ctx, int enable);

/* Programmatic dependent launch (on by default): a kernel that directly follows
 * another kernel of the same stage on the stream is launched with the
 * programmatic stream-serialization attribute, so it is launched once the
 * blocks of the kernel before it have exited; each of its blocks waits for
 * that kernel to complete before it touches memory. Off: plain stream order. Kernels
 * separated by a timing event, a copy or a memset are always launched in plain
 * order. Outputs are the same either way. */
CG_API cg_status cg_set_pdl(cg_ctx* ctx, int enable);

/* Host outputs of 64 MB or more are spelled into device memory in chunks of
 * 128 MB, each copied to the host while the next one is spelled. Smaller
 * ones in pinned host memory are written in place by the kernels over the
 * host link (the default, enable = 1); with 0 they are written to device
 * memory and copied. Other host memory is always staged and copied. Outputs
 * are the same either way. */
CG_API cg_status cg_set_host_direct(cg_ctx* ctx, int enable);

/* Host-side fault injection, for tests of the error paths that fault no GPU.
 * spec: "site:n[:ms]" entries separated by commas; the n-th time (from 1) this
 * context reaches `site` it fails as that step would: "alloc" (CG_ENOMEM),
 * "h2d" (an input copy, CG_ECUDA), "timeout" (a bounded device wait,
 * CG_ETIMEOUT), "kernel" (a kernel consistency check, CG_EKERNEL), "bad_graph"
 * (input validation, CG_EGRAPH). NULL or "" clears the plan. The CG_FAULT
 * environment variable gives the plan of every new context and server; a
 * server also knows "admit" (cg_server_submit returns CG_EBUSY) and
 * "queue_stall" (a worker sleeps ms milliseconds before its n-th batch) and
 * "batch_timeout" (the n-th batch's first device wait reports CG_ETIMEOUT, so
 * its worker replaces its context). */
CG_API cg_status cg_set_fault(cg_ctx* ctx, const char* spec);

/* Counters of a context, for measurement. */
typedef struct {
  uint64_t kernels_launched; /* CUDA kernels this context has launched so far */
  float stage_ms[4];         /* last mask, chain, offset and emission stage, in ms of GPU time
                                (CUDA events on the context stream; 0 unless timing is on) */
} cg_stats;

/* Timing: 0 off, 1 CUDA events around each stage, 2 also after every
 * kernel (for cg_kernel_time), 3 events around the spelling stage only
 * (cg_stats.stage_ms[3]; the other stages read 0). Events are recorded on the
 * context stream and the work itself is unchanged, but each event inside a
 * replayed stage costs a few microseconds of GPU time. */
CG_API cg_status cg_set_timing(cg_ctx* ctx, int enable);
/* Fills *out; with timing on it waits for the last stages to finish. */
CG_API cg_status cg_get_stats(cg_ctx* ctx, cg_stats* out);
/* With timing 2: the name (static string) and GPU time in ms of the k-th
 * kernel (k from 0) launched since the last mask stage began; each time runs
 * from the previous kernel's end mark, so it includes the small memsets
 * queued between kernels. Waits for the GPU. CG_EINVAL past the last one. */
CG_API cg_status cg_kernel_time(cg_ctx* ctx, int k, const char** name, float* ms);

/* Exclusive prefix offsets without any device allocation. The paper has no
 * counterpart. This is the library's offset scan -- the one that places
 * contigs and read pieces in the output (contig_off of cg_emit_contigs) --
 * for callers that cannot call cudaMalloc: code that runs while another
 * allocator owns the device memory (a caching allocator that must see every
 * allocation, or a hard HBM budget the caller may not exceed), where a
 * cudaMalloc of the library's own would take memory that allocator counts
 * on, or would synchronise the device under it. Its look-back scratch is one
 * file-scope device array instead of allocated buffers.
 *   lengths: device memory, 4-byte aligned, count values >= 0; offsets:
 *   device memory, 8-byte aligned, count + 1 entries; offsets[i] =
 *   lengths[0] + ... + lengths[i-1] and offsets[count] = the total.
 *   count <= CG_NOALLOC_MAX_COUNT; a larger count, a NULL, misaligned or
 *   non-device pointer gives CG_EINVAL and nothing is queued.
 * Work is queued on cuda_stream (NULL = the legacy default stream) of the
 * current device, and every call then waits for that stream (it copies the
 * status word to the host and synchronises), so that it can return
 * CG_ETIMEOUT if the kernel's bounded wait gave up (else CG_OK / CG_ECUDA).
 * After CG_ETIMEOUT the contents of offsets are undefined.
 * The scratch is one file-scope device array of 8 * (CG_NOALLOC_MAX_COUNT /
 * 2048 + 3) bytes (64 KiB + 24) that every GPU which loads the library holds
 * until the process exits. The first call on a device, with that device
 * current, looks up the array's device address (cudaGetSymbolAddress) and the
 * SM count; make that first call before any stream capture. Every call
 * shares the array and clears the part it uses first, so calls that overlap
 * on the GPU (other streams, other threads) race and must be serialised by
 * the caller. */
#define CG_NOALLOC_MAX_COUNT 16777216
CG_API cg_status cg_offsets_noalloc(const int32_t* lengths, int64_t count, int64_t* offsets, void* cuda_stream);

/* Self-test of the bounded device waits (the paper has none: its steps are
 * separated by MPI collectives). Runs the library's look-back scan -- the
 * one that lays out contigs and read pieces (Sec. 4.4 offsets) -- over
 * `tiles` tiles (2..4096) of zeros on the context's stream, with the ticket
 * of tile 0 never handed out, so the tiles after it wait on a descriptor that
 * no block publishes. Their wait is bounded (2^22 polls with a 200 ns back-off,
 * about one to two seconds); it then gives up, the kernel records the timeout
 * in the context's error word and returns. Nothing faults or hangs. Returns
 * CG_ETIMEOUT, after which the context refuses all work until cg_destroy as
 * after any device timeout; CG_EKERNEL if the wait did not run out. Waits
 * for the GPU. */
CG_API cg_status cg_selftest_wait_timeout(cg_ctx* ctx, int32_t tiles);

/* Waits for all work of the context; returns the first error its kernels found. */
CG_API cg_status cg_sync(cg_ctx* ctx);

CG_API const char* cg_status_str(cg_status s);
/* Copies the context's last error message (NUL-terminated) into buf. */
CG_API cg_status cg_last_error(cg_ctx* ctx, char* buf, size_t buflen);

#ifdef __cplusplus
}
#endif
#endif
