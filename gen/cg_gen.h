/* cg_gen.h - seeded synthetic string-graph generator (test and benchmark input only). */
#ifndef CG_GEN_H
#define CG_GEN_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* One class of repeat families: families are drawn until the class covers
 * `share` of the genome; each family is a random segment of length
 * U[seg_min, seg_max] with U[copies_min, copies_max] copies, each copy
 * carrying its own substitution divergence U[0, div_max]. */
typedef struct {
  double share;
  int32_t seg_min, seg_max, copies_min, copies_max;
  double div_max;
} cg_gen_repclass;

typedef struct {
  uint64_t seed;
  int64_t genome_len;
  int32_t n_classes, _pad0;
  cg_gen_repclass cls[4];
  double coverage;
  int32_t len_kind;  /* 0: uniform [len_a, len_b]; 1: lognormal, mean len_a, sd len_b */
  int32_t len_min;   /* lognormal draws below this are redrawn */
  double len_a, len_b;
  int32_t min_overlap; /* shortest overlap kept as an edge (bases) */
  int32_t k_rep;       /* repeat-induced edges per read end, at most */
  double rep_div_accept; /* a repeat edge needs div(X) + div(Y) <= this */
  int32_t threads, shuffle_ids;
  int32_t off_align;   /* read start alignment in the packed stream, bases: 1, 4 or 32 */
  int32_t full_overlaps; /* 1: every pair of reads overlapping >= min_overlap (the overlap
                            graph before transitive reduction); 0: consecutive pairs only */
} cg_gen_cfg;

typedef struct {
  int64_t genome_len, n_sampled, n_reads, n_kept, n_entries, packed_bytes, total_read_bases;
  int64_t n_true_pairs, n_rep_pairs, n_copies, n_families, repeat_bases;
} cg_gen_info;

typedef struct cg_gen cg_gen;

cg_gen* cg_gen_plan(const cg_gen_cfg* cfg);
const char* cg_gen_error(const cg_gen* g); /* "" when the plan succeeded */
void cg_gen_get_info(const cg_gen* g, cg_gen_info* out);
/* Copies the graph into caller buffers; any pointer may be NULL. row_ptr is
 * written as int32 (rp_bytes = 4) or int64 (rp_bytes = 8). gstart/strand give
 * each read's true genome start and whether it is stored reverse-complemented;
 * contained marks reads lying inside another read (edgeless vertices). */
int cg_gen_fill(const cg_gen* g, void* row_ptr, int rp_bytes, int32_t* col, uint8_t* code, int32_t* suf,
                int32_t* len, int64_t* off, uint8_t* packed, uint8_t* is_true, int64_t* gstart, uint8_t* strand,
                uint8_t* contained);
/* ASCII copy of genome[start, start+count). */
int cg_gen_genome(const cg_gen* g, int64_t start, int64_t count, uint8_t* ascii);
void cg_gen_free(cg_gen* g);

#ifdef __cplusplus
}
#endif
#endif
