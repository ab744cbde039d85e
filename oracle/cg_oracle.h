/*
 * cg_oracle.h - CPU oracle for contig generation (TEST INFRASTRUCTURE ONLY).
 *
 * A plain, slow, single-threaded C restatement of what contig generation
 * computes in Guidi et al., ICPP'22 (Alg. 2, Sec. 4.2 and 4.4). Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may call it;
 * the product path never does. It shares no code with the CUDA path.
 */
#ifndef CG_ORACLE_H
#define CG_ORACLE_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_EGRAPH = 1, ORC_ENOMEM = 2, ORC_EINTERNAL = 3 };

typedef struct orc_result orc_result;

/* Input checks of a string graph (see cg_oracle.c for the list). */
int orc_validate(int64_t n, int64_t m, const int64_t* row_ptr, const int32_t* col, const uint8_t* code,
                 const int32_t* suf, const int32_t* len, const int64_t* off, int64_t packed_bytes,
                 char* msg, size_t msglen);

/* Whole contig generation on one graph. min_chain_reads < 1 is taken as 1.
 * validate != 0 runs orc_validate first. *status gets ORC_*. */
orc_result* orc_run(int64_t n, int64_t m, const int64_t* row_ptr, const int32_t* col, const uint8_t* code,
                    const int32_t* suf, const int32_t* len, const int64_t* off, const uint8_t* packed,
                    int64_t packed_bytes, int32_t min_chain_reads, int validate, int* status);

/* The same with the x-drop form of the overlaps (Sec. 4.4) when pre and post
 * are both non-NULL (then suf is not read and may be NULL): per entry (u->v),
 * pre = index in stored u of u's last base before the overlap in walk
 * direction, post = index in stored v of v's first base of the overlap. */
int orc_validate2(int64_t n, int64_t m, const int64_t* row_ptr, const int32_t* col, const uint8_t* code,
                  const int32_t* suf, const int32_t* pre, const int32_t* post, const int32_t* len,
                  const int64_t* off, int64_t packed_bytes, char* msg, size_t msglen);
orc_result* orc_run2(int64_t n, int64_t m, const int64_t* row_ptr, const int32_t* col, const uint8_t* code,
                     const int32_t* suf, const int32_t* pre, const int32_t* post, const int32_t* len,
                     const int64_t* off, const uint8_t* packed, int64_t packed_bytes, int32_t min_chain_reads,
                     int validate, int* status);

/* TransitiveReduction (Alg. 1, Sec. 2) of an overlap graph in the suffix
 * form: the string graph's CSR into out_* (n+1 row pointers, up to m
 * entries). Returns the number of entries kept. */
int64_t orc_transitive_reduction(int64_t n, int64_t m, const int64_t* row_ptr, const int32_t* col, const uint8_t* code,
                                 const int32_t* suf, int32_t fuzz, int64_t* out_rp, int32_t* out_col,
                                 uint8_t* out_code, int32_t* out_suf);

int64_t orc_n_branch(const orc_result* r);
int64_t orc_n_contigs(const orc_result* r);
int64_t orc_n_cycles(const orc_result* r);
int64_t orc_total_bases(const orc_result* r);
int64_t orc_n_components(const orc_result* r);   /* components of L on the unmasked reads */
int64_t orc_edge_entries_walked(const orc_result* r);
void orc_get_branch(const orc_result* r, uint8_t* is_branch);
void orc_get_chains(const orc_result* r, int32_t* chain_id, int32_t* rank, uint8_t* orient);
void orc_get_contigs(const orc_result* r, int64_t* contig_off, uint8_t* bases);
/* Component labels (min read id of the component, -1 for branch reads) by
 * union-find (which = 0) or by breadth-first search (which = 1). */
void orc_get_labels(const orc_result* r, int which, int32_t* label);
void orc_free(orc_result* r);

/* Reverse complement of an ASCII DNA string (Sec. 2). */
void orc_revcomp(const char* in, int64_t n, char* out);

/* Longest-processing-time greedy partitioning (Sec. 4.3): sizes sorted
 * descending (ties: lower index first), each put in the least-loaded of P
 * bins (ties: lowest bin). assign[i] = bin of job i; loads[P]. */
int orc_lpt(const int64_t* sizes, int64_t k, int32_t P, int32_t* assign, int64_t* loads);

#ifdef __cplusplus
}
#endif
#endif
