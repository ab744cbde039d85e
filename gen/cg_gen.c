/*
 * cg_gen.c - seeded synthetic string-graph generator.
 *
 * Test and benchmark input only: this file builds bidirected string graphs
 * shaped like the long-read workloads of Guidi et al., "Distributed-Memory
 * Parallel Contig Generation for De Novo Long-Read Genome Assembly" (ICPP'22),
 * Sec. 2 (string graph, overhang/suffix weights, bidirected arrows) and
 * Table 2 (dataset shapes). It holds none of the contig-generation method
 * (no branch masking, no components, no walks, no spelling): it only lays out
 * a genome, samples reads from it, marks contained reads (kept as edgeless
 * vertices, as a pruned matrix row keeps its index), and records the
 * overlaps that a perfect overlapper plus transitive reduction would keep,
 * plus repeat-induced overlaps that create branches.
 *
 * Everything is a pure function of (config, seed): every random draw comes
 * from a counter-based splitmix64 hash of (seed, stream tag, index), so the
 * output does not depend on the thread count.
 *
 * Encoding of the produced graph (shared input format):
 *   bases  A=0 C=1 G=2 T=3, complement = 3-b; base i of the packed stream is
 *          in byte i>>2 at bits 2*(i&3).
 *   entry (u->v) code = E_u | (E_v << 1); E=0 is the 5' (first stored base)
 *          end of a read, E=1 its 3' end; the mirror (v->u) swaps the bits.
 *   suf(u->v) = number of bases of v, in walk orientation, beyond the overlap.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "cg_gen.h"

/* ------------------------------------------------------------------ rng */
#define GOLDEN 0x9E3779B97F4A7C15ull
static inline uint64_t smix(uint64_t z) {
  z += GOLDEN;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static inline uint64_t hash2(uint64_t a, uint64_t b) { return smix(a ^ smix(b ^ 0x5851F42D4C957F2Dull)); }
static inline uint64_t hash3(uint64_t a, uint64_t b, uint64_t c) { return smix(hash2(a, b) ^ smix(c + 0x632BE59BD9B4E019ull)); }
typedef struct { uint64_t s; } rng_t;
static inline rng_t rng_make(uint64_t seed, uint64_t tag, uint64_t idx) { rng_t r = {hash3(seed, tag, idx)}; return r; }
static inline uint64_t rng_next(rng_t* r) { r->s += GOLDEN; return smix(r->s); }
static inline double rng_u01(rng_t* r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }
static inline int64_t rng_range(rng_t* r, int64_t lo, int64_t hi) { /* inclusive */
  if (hi <= lo) return lo;
  return lo + (int64_t)(rng_next(r) % (uint64_t)(hi - lo + 1));
}

enum { T_FAMLEN = 1, T_FAMSEQ, T_COPYDIV, T_SHUF, T_GAPW, T_GENOME, T_MUT, T_READ, T_PERM, T_REP };

/* ------------------------------------------------------- parallel for */
typedef void (*range_fn)(void* ctx, int64_t lo, int64_t hi);
typedef struct { range_fn fn; void* ctx; int64_t lo, hi; } job_t;
static void* job_run(void* p) { job_t* j = (job_t*)p; if (j->lo < j->hi) j->fn(j->ctx, j->lo, j->hi); return NULL; }
static void pfor(int threads, int64_t n, range_fn fn, void* ctx) {
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  if (n < 4096 || threads == 1) { if (n > 0) fn(ctx, 0, n); return; }
  pthread_t th[256]; job_t jb[256];
  int64_t chunk = (n + threads - 1) / threads;
  int started = 0;
  for (int t = 0; t < threads; ++t) {
    jb[t].fn = fn; jb[t].ctx = ctx; jb[t].lo = t * chunk; jb[t].hi = (t + 1) * chunk < n ? (t + 1) * chunk : n;
    if (pthread_create(&th[t], NULL, job_run, &jb[t]) == 0) started = t + 1; else { job_run(&jb[t]); }
  }
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------ structs */
typedef struct { int64_t start; int32_t len, fam; double div; } copy_t;
typedef struct { int32_t len, cls, n_copies, first; /* index into fam_copies */ int64_t seq_off; } fam_t;

struct cg_gen {
  cg_gen_cfg cfg;
  int64_t G;
  uint64_t* g64;          /* packed genome, 32 bases per word, 2 pad words */
  int64_t n_copy; copy_t* copy;   /* genome order (sorted by start) */
  int32_t n_fam; fam_t* fam;
  int32_t* fam_copies;    /* copy indices grouped by family */
  uint8_t* famseq;        /* one byte per base, all families concatenated */
  int64_t famseq_len;
  /* all sampled reads, sorted by (start asc, end desc); contained reads stay
   * in the read set as edgeless vertices (the matrix rows of a pruned read) */
  int64_t n_sampled, n;
  int64_t *rs, *re; uint8_t *strand, *contained;
  int32_t *id_of, *gidx_of;
  /* non-contained reads, genome order: ks/ke/kst, kp = index into the sorted arrays */
  int64_t n_kept;
  int64_t *ks, *ke, *kp; uint8_t* kst;
  /* graph in read-id space */
  int64_t m;
  int64_t* row_ptr; int32_t* col; uint8_t* code; int32_t* suf; uint8_t* is_true;
  int64_t* off; int32_t* len;
  int64_t packed_bytes, total_read_bases;
  int64_t n_true_pairs, n_rep_pairs;
  char err[160];
};

/* --------------------------------------------------------- genome fill */
static inline int gap_base(uint64_t seed, int64_t p) { return (int)((hash2(seed ^ T_GENOME, (uint64_t)(p >> 5)) >> (2 * (p & 31))) & 3); }

static int copy_base(const cg_gen* g, int64_t ci, int64_t j) {
  const copy_t* c = &g->copy[ci];
  int b = g->famseq[g->fam[c->fam].seq_off + j];
  if (c->div > 0.0) {
    uint64_t u = hash3(g->cfg.seed ^ T_MUT, (uint64_t)ci, (uint64_t)j);
    double x = (double)(u >> 11) * (1.0 / 9007199254740992.0);
    if (x < c->div) b = (b + 1 + (int)((u & 0xFFFF) % 3)) & 3;
  }
  return b;
}

/* first copy with start+len > p (copies are disjoint and sorted) */
static int64_t copy_at_or_after(const cg_gen* g, int64_t p) {
  int64_t lo = 0, hi = g->n_copy;
  while (lo < hi) { int64_t mid = (lo + hi) >> 1; if (g->copy[mid].start + g->copy[mid].len <= p) lo = mid + 1; else hi = mid; }
  return lo;
}

static void fill_genome_range(void* ctx, int64_t w0, int64_t w1) {
  cg_gen* g = (cg_gen*)ctx;
  uint64_t seed = g->cfg.seed;
  int64_t ci = copy_at_or_after(g, w0 * 32);
  for (int64_t w = w0; w < w1; ++w) {
    int64_t p0 = w * 32, p1 = p0 + 32;
    while (ci < g->n_copy && g->copy[ci].start + g->copy[ci].len <= p0) ++ci;
    if (p0 >= g->G) { g->g64[w] = 0; continue; }
    if (ci >= g->n_copy || g->copy[ci].start >= p1) {
      g->g64[w] = hash2(seed ^ T_GENOME, (uint64_t)w);      /* all gap */
      if (p1 > g->G) { int keep = (int)(g->G - p0); g->g64[w] &= (keep >= 32) ? ~0ull : ((1ull << (2 * keep)) - 1); }
      continue;
    }
    uint64_t word = 0;
    int64_t cj = ci;
    for (int64_t p = p0; p < p1 && p < g->G; ++p) {
      while (cj < g->n_copy && g->copy[cj].start + g->copy[cj].len <= p) ++cj;
      int b;
      if (cj < g->n_copy && g->copy[cj].start <= p) b = copy_base(g, cj, p - g->copy[cj].start);
      else b = gap_base(seed, p);
      word |= (uint64_t)b << (2 * (p - p0));
    }
    g->g64[w] = word;
  }
}

static inline uint64_t get64(const uint64_t* g64, int64_t pos) { /* 32 bases from pos >= 0 */
  int64_t w = pos >> 5; int sh = (int)(2 * (pos & 31));
  uint64_t lo = g64[w] >> sh;
  if (sh) lo |= g64[w + 1] << (64 - sh);
  return lo;
}
static inline uint64_t rev2(uint64_t x) { /* reverse order of 2-bit groups */
  x = ((x >> 2) & 0x3333333333333333ull) | ((x & 0x3333333333333333ull) << 2);
  x = ((x >> 4) & 0x0F0F0F0F0F0F0F0Full) | ((x & 0x0F0F0F0F0F0F0F0Full) << 4);
  return __builtin_bswap64(x);
}
static inline int gbase(const uint64_t* g64, int64_t p) { return (int)((g64[p >> 5] >> (2 * (p & 31))) & 3); }

/* ---------------------------------------------------------- radix sort */
static void radix_sort_u64(uint64_t* key, uint32_t* val, int64_t n) {
  uint64_t* k2 = (uint64_t*)malloc((size_t)n * 8); uint32_t* v2 = (uint32_t*)malloc((size_t)n * 4);
  size_t* cnt = (size_t*)malloc(65536 * sizeof(size_t));
  for (int pass = 0; pass < 4; ++pass) {
    int sh = 16 * pass;
    memset(cnt, 0, 65536 * sizeof(size_t));
    for (int64_t i = 0; i < n; ++i) cnt[(key[i] >> sh) & 0xFFFF]++;
    size_t s = 0; for (int d = 0; d < 65536; ++d) { size_t c = cnt[d]; cnt[d] = s; s += c; }
    for (int64_t i = 0; i < n; ++i) { size_t d = cnt[(key[i] >> sh) & 0xFFFF]++; k2[d] = key[i]; v2[d] = val[i]; }
    memcpy(key, k2, (size_t)n * 8); memcpy(val, v2, (size_t)n * 4);
  }
  free(k2); free(v2); free(cnt);
}

/* ------------------------------------------------------------ sampling */
typedef struct { cg_gen* g; int64_t* s; int64_t* e; uint8_t* st; double mu, sigma; } sample_ctx;
static void sample_range(void* p, int64_t lo, int64_t hi) {
  sample_ctx* c = (sample_ctx*)p; const cg_gen_cfg* f = &c->g->cfg; int64_t G = c->g->G;
  for (int64_t i = lo; i < hi; ++i) {
    rng_t r = rng_make(f->seed, T_READ, (uint64_t)i);
    int64_t L;
    if (f->len_kind == 0) {
      L = rng_range(&r, (int64_t)f->len_a, (int64_t)f->len_b);
    } else {
      L = f->len_min;
      for (int t = 0; t < 64; ++t) {
        double u1 = rng_u01(&r), u2 = rng_u01(&r);
        if (u1 < 1e-300) u1 = 1e-300;
        double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
        int64_t x = (int64_t)llround(exp(c->mu + c->sigma * z));
        if (x >= f->len_min) { L = x; break; }
      }
    }
    if (L < 1) L = 1;
    if (L > G) L = G;
    int64_t s = rng_range(&r, 0, G - L);
    c->s[i] = s; c->e[i] = s + L; c->st[i] = (uint8_t)(rng_next(&r) & 1);
  }
}

/* ------------------------------------------------------- repeat edges */
typedef struct { int32_t a, b; int32_t suf_ab, suf_ba; uint8_t code_ab, code_ba, is_true, pad; } pair_t;

static inline int e_right(uint8_t strand) { return strand == 0 ? 1 : 0; } /* stored end at genome-right */
static inline int e_left(uint8_t strand) { return strand == 0 ? 0 : 1; }  /* stored end at genome-left */

static int64_t first_kept_at_or_after(const cg_gen* g, int64_t pos) {
  int64_t lo = 0, hi = g->n_kept;
  while (lo < hi) { int64_t mid = (lo + hi) >> 1; if (g->ks[mid] < pos) lo = mid + 1; else hi = mid; }
  return lo;
}
static int64_t copy_containing(const cg_gen* g, int64_t p) {
  int64_t ci = copy_at_or_after(g, p);
  if (ci < g->n_copy && g->copy[ci].start <= p) return ci;
  return -1;
}

typedef struct { cg_gen* g; pair_t* out; int32_t* cnt; } rep_ctx;
static void rep_range(void* p, int64_t lo, int64_t hi) {
  rep_ctx* c = (rep_ctx*)p; cg_gen* g = c->g; const cg_gen_cfg* f = &g->cfg;
  int K = f->k_rep, mo = f->min_overlap;
  for (int64_t a = lo; a < hi; ++a) {
    c->cnt[a] = 0;
    int64_t ea = g->ke[a], la = g->ke[a] - g->ks[a];
    int64_t xi = copy_containing(g, ea - 1);
    if (xi < 0) continue;
    const copy_t* X = &g->copy[xi];
    int64_t ra = ea - X->start;
    if (ra < mo || ea - mo < X->start) continue;
    const fam_t* F = &g->fam[X->fam];
    if (F->n_copies < 2) continue;
    rng_t r = rng_make(f->seed, T_REP, (uint64_t)a);
    for (int t = 0; t < 16 && c->cnt[a] < K; ++t) {
      int32_t yi = g->fam_copies[F->first + (int32_t)(rng_next(&r) % (uint64_t)F->n_copies)];
      if (yi == xi) continue;
      const copy_t* Y = &g->copy[yi];
      if (X->div + Y->div > f->rep_div_accept) continue;
      int64_t lo_s = Y->start, hi_s = Y->start + ra - mo;
      int64_t cand = -1, ncand = 0;
      for (int64_t b = first_kept_at_or_after(g, lo_s), scanned = 0; b < g->n_kept && g->ks[b] <= hi_s && scanned < 64; ++b, ++scanned) {
        if (b == a) continue;
        int64_t ov = ra - (g->ks[b] - Y->start);
        if (g->ke[b] <= Y->start + ra) continue;
        if (ov >= la || ov < mo) continue;
        int dup = 0;
        for (int q = 0; q < c->cnt[a]; ++q) if (c->out[a * K + q].b == (int32_t)b) dup = 1;
        if (dup) continue;
        ++ncand;
        if ((int64_t)(rng_next(&r) % (uint64_t)ncand) == 0) cand = b;
      }
      if (cand < 0) continue;
      int64_t ov = ra - (g->ks[cand] - Y->start);
      pair_t* e = &c->out[a * K + c->cnt[a]];
      e->a = (int32_t)a; e->b = (int32_t)cand; e->is_true = 0; e->pad = 0;
      e->code_ab = (uint8_t)(e_right(g->kst[a]) | (e_left(g->kst[cand]) << 1));
      e->code_ba = (uint8_t)(e_left(g->kst[cand]) | (e_right(g->kst[a]) << 1));
      e->suf_ab = (int32_t)(g->ke[cand] - (Y->start + ra));
      e->suf_ba = (int32_t)(la - ov);
      c->cnt[a]++;
    }
  }
}

static int pair_cmp(const void* x, const void* y) {
  const pair_t* p = (const pair_t*)x; const pair_t* q = (const pair_t*)y;
  int32_t plo = p->a < p->b ? p->a : p->b, phi = p->a < p->b ? p->b : p->a;
  int32_t qlo = q->a < q->b ? q->a : q->b, qhi = q->a < q->b ? q->b : q->a;
  if (plo != qlo) return plo < qlo ? -1 : 1;
  if (phi != qhi) return phi < qhi ? -1 : 1;
  if (p->is_true != q->is_true) return p->is_true > q->is_true ? -1 : 1;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  return 0;
}

/* --------------------------------------------------------- packed fill */
typedef struct { const cg_gen* g; uint8_t* packed; } pack_ctx;
static void pack_range(void* p, int64_t lo, int64_t hi) {
  pack_ctx* c = (pack_ctx*)p; const cg_gen* g = c->g;
  for (int64_t id = lo; id < hi; ++id) {
    int64_t k = g->gidx_of[id];
    int64_t s = g->rs[k], e = g->re[k], L = e - s, o = g->off[id];
    uint8_t* dst = c->packed + (o >> 2);
    if ((o & 31) == 0) {
      uint64_t* d64 = (uint64_t*)dst;  /* offsets are 32-base aligned here */
      int64_t nw = (L + 31) / 32;
      for (int64_t j = 0; j < nw; ++j) {
        uint64_t w;
        if (g->strand[k] == 0) {
          w = get64(g->g64, s + 32 * j);
        } else {
          int64_t pstart = e - 32 - 32 * j;
          if (pstart >= 0) w = ~rev2(get64(g->g64, pstart));
          else { w = 0; for (int t = 0; t < 32 && 32 * j + t < L; ++t) w |= (uint64_t)(3 - gbase(g->g64, e - 1 - 32 * j - t)) << (2 * t); }
        }
        int64_t rem = L - 32 * j;
        if (rem < 32) w &= (1ull << (2 * rem)) - 1;
        memcpy(d64 + j, &w, 8);
      }
    } else { /* generic offsets: base by base */
      for (int64_t t = 0; t < L; ++t) {
        int b = g->strand[k] == 0 ? gbase(g->g64, s + t) : 3 - gbase(g->g64, e - 1 - t);
        int64_t q = o + t;
        c->packed[q >> 2] = (uint8_t)((c->packed[q >> 2] & ~(3u << (2 * (q & 3)))) | ((unsigned)b << (2 * (q & 3))));
      }
    }
  }
}

/* ---------------------------------------------------------------- plan */
static void fail(cg_gen* g, const char* msg) { strncpy(g->err, msg, sizeof(g->err) - 1); }

cg_gen* cg_gen_plan(const cg_gen_cfg* cfg) {
  cg_gen* g = (cg_gen*)calloc(1, sizeof(cg_gen));
  if (!g) return NULL;
  g->cfg = *cfg;
  const cg_gen_cfg* f = &g->cfg;
  int T = f->threads > 0 ? f->threads : 1;
  g->G = f->genome_len;
  if (g->G < 64 || g->G > 4000000000ll) { fail(g, "genome_len out of range"); return g; }
  if (f->off_align != 1 && f->off_align != 4 && f->off_align != 32) { fail(g, "off_align must be 1, 4 or 32"); return g; }

  /* 1. repeat families per class, copies with divergence */
  int32_t fam_cap = 1024; g->fam = (fam_t*)calloc((size_t)fam_cap, sizeof(fam_t));
  int64_t copy_cap = 1024, n_copy = 0; copy_t* copies = (copy_t*)malloc((size_t)copy_cap * sizeof(copy_t));
  int64_t R = 0; g->famseq_len = 0;
  for (int ci = 0; ci < f->n_classes && ci < 4; ++ci) {
    const cg_gen_repclass* k = &f->cls[ci];
    int64_t target = (int64_t)llround(k->share * (double)g->G), got = 0;
    while (got < target) {
      rng_t r = rng_make(f->seed, T_FAMLEN, (uint64_t)g->n_fam);
      int32_t L = (int32_t)rng_range(&r, k->seg_min, k->seg_max);
      int64_t nc = rng_range(&r, k->copies_min, k->copies_max);
      int64_t need = (target - got + L - 1) / L;
      if (nc > need) nc = need;
      if (nc < 1) nc = 1;
      if (g->n_fam == fam_cap) { fam_cap *= 2; g->fam = (fam_t*)realloc(g->fam, (size_t)fam_cap * sizeof(fam_t)); }
      fam_t* F = &g->fam[g->n_fam];
      F->len = L; F->cls = ci; F->n_copies = (int32_t)nc; F->seq_off = g->famseq_len;
      g->famseq_len += L;
      for (int64_t q = 0; q < nc; ++q) {
        if (n_copy == copy_cap) { copy_cap *= 2; copies = (copy_t*)realloc(copies, (size_t)copy_cap * sizeof(copy_t)); }
        rng_t rd = rng_make(f->seed, T_COPYDIV, (uint64_t)n_copy);
        copies[n_copy].len = L; copies[n_copy].fam = g->n_fam; copies[n_copy].div = rng_u01(&rd) * k->div_max;
        copies[n_copy].start = 0; ++n_copy;
      }
      got += (int64_t)L * nc; R += (int64_t)L * nc;
      g->n_fam++;
    }
  }
  if (R > g->G) { fail(g, "repeat content exceeds genome"); free(copies); return g; }
  g->famseq = (uint8_t*)malloc((size_t)(g->famseq_len > 0 ? g->famseq_len : 1));
  for (int32_t fi = 0; fi < g->n_fam; ++fi)
    for (int32_t j = 0; j < g->fam[fi].len; ++j)
      g->famseq[g->fam[fi].seq_off + j] = (uint8_t)(hash3(f->seed ^ T_FAMSEQ, (uint64_t)fi, (uint64_t)j) & 3);

  /* 2. shuffle copies, lay out gap copy gap copy ... gap */
  {
    rng_t r = rng_make(f->seed, T_SHUF, 0);
    for (int64_t i = n_copy - 1; i > 0; --i) { int64_t j = (int64_t)(rng_next(&r) % (uint64_t)(i + 1)); copy_t t = copies[i]; copies[i] = copies[j]; copies[j] = t; }
    int64_t U = g->G - R;
    double* cw = (double*)malloc((size_t)(n_copy + 1) * sizeof(double));
    double W = 0;
    for (int64_t i = 0; i <= n_copy; ++i) { rng_t rw = rng_make(f->seed, T_GAPW, (uint64_t)i); double u = rng_u01(&rw); if (u < 1e-12) u = 1e-12; W += -log(u); cw[i] = W; }
    int64_t pos = 0, prev_cut = 0;
    for (int64_t i = 0; i < n_copy; ++i) {
      int64_t cut = (int64_t)floor((double)U * (cw[i] / W));
      if (cut < prev_cut) cut = prev_cut;
      if (cut > U) cut = U;
      pos += cut - prev_cut; prev_cut = cut;
      copies[i].start = pos; pos += copies[i].len;
    }
    free(cw);
  }
  g->copy = copies; g->n_copy = n_copy;
  /* family -> copies */
  g->fam_copies = (int32_t*)malloc((size_t)(n_copy > 0 ? n_copy : 1) * sizeof(int32_t));
  {
    int32_t acc = 0;
    for (int32_t fi = 0; fi < g->n_fam; ++fi) { g->fam[fi].first = acc; acc += g->fam[fi].n_copies; g->fam[fi].n_copies = 0; }
    for (int64_t i = 0; i < n_copy; ++i) { fam_t* F = &g->fam[copies[i].fam]; g->fam_copies[F->first + F->n_copies++] = (int32_t)i; }
  }

  /* 3. genome bases */
  int64_t nw = (g->G + 31) / 32;
  g->g64 = (uint64_t*)calloc((size_t)(nw + 2), 8);
  pfor(T, nw, fill_genome_range, g);

  /* 4. sample reads, sort by (start asc, end desc), drop contained */
  double mean = f->len_kind == 0 ? 0.5 * (f->len_a + f->len_b) : f->len_a;
  int64_t N0 = (int64_t)llround(f->coverage * (double)g->G / mean);
  if (N0 < 1) N0 = 1;
  if (N0 > 2000000000ll) { fail(g, "too many reads"); return g; }
  g->n_sampled = N0;
  int64_t* s = (int64_t*)malloc((size_t)N0 * 8); int64_t* e = (int64_t*)malloc((size_t)N0 * 8); uint8_t* st = (uint8_t*)malloc((size_t)N0);
  sample_ctx sc = {g, s, e, st, 0, 0};
  if (f->len_kind == 1) { double cv = f->len_b / f->len_a; sc.sigma = sqrt(log(1.0 + cv * cv)); sc.mu = log(f->len_a) - 0.5 * sc.sigma * sc.sigma; }
  pfor(T, N0, sample_range, &sc);
  uint64_t* key = (uint64_t*)malloc((size_t)N0 * 8); uint32_t* idx = (uint32_t*)malloc((size_t)N0 * 4);
  for (int64_t i = 0; i < N0; ++i) { key[i] = ((uint64_t)s[i] << 32) | (uint64_t)(0xFFFFFFFFull - (uint64_t)e[i]); idx[i] = (uint32_t)i; }
  radix_sort_u64(key, idx, N0);
  g->rs = (int64_t*)malloc((size_t)N0 * 8); g->re = (int64_t*)malloc((size_t)N0 * 8);
  g->strand = (uint8_t*)malloc((size_t)N0); g->contained = (uint8_t*)malloc((size_t)N0);
  g->ks = (int64_t*)malloc((size_t)N0 * 8); g->ke = (int64_t*)malloc((size_t)N0 * 8);
  g->kp = (int64_t*)malloc((size_t)N0 * 8); g->kst = (uint8_t*)malloc((size_t)N0);
  int64_t K = 0, maxe = -1;
  for (int64_t t = 0; t < N0; ++t) {
    int64_t i = idx[t];
    g->rs[t] = s[i]; g->re[t] = e[i]; g->strand[t] = st[i];
    g->contained[t] = (uint8_t)(e[i] <= maxe);   /* [s,e) inside an earlier read */
    if (e[i] > maxe) { g->ks[K] = s[i]; g->ke[K] = e[i]; g->kst[K] = st[i]; g->kp[K] = t; ++K; maxe = e[i]; }
  }
  free(s); free(e); free(st); free(key); free(idx);
  g->n = N0; g->n_kept = K;

  /* 5. read ids: seeded permutation of the sorted order */
  g->id_of = (int32_t*)malloc((size_t)N0 * 4); g->gidx_of = (int32_t*)malloc((size_t)N0 * 4);
  for (int64_t k = 0; k < N0; ++k) g->id_of[k] = (int32_t)k;
  if (f->shuffle_ids) {
    rng_t r = rng_make(f->seed, T_PERM, 0);
    for (int64_t i = N0 - 1; i > 0; --i) { int64_t j = (int64_t)(rng_next(&r) % (uint64_t)(i + 1)); int32_t t = g->id_of[i]; g->id_of[i] = g->id_of[j]; g->id_of[j] = t; }
  }
  for (int64_t k = 0; k < N0; ++k) g->gidx_of[g->id_of[k]] = (int32_t)k;

  /* 6. offsets and lengths in id order */
  g->off = (int64_t*)malloc((size_t)N0 * 8); g->len = (int32_t*)malloc((size_t)N0 * 4);
  {
    int64_t acc = 0, A = f->off_align;
    for (int64_t id = 0; id < N0; ++id) {
      int64_t k = g->gidx_of[id], L = g->re[k] - g->rs[k];
      g->off[id] = acc; g->len[id] = (int32_t)L; g->total_read_bases += L;
      acc += (L + A - 1) / A * A;
    }
    g->packed_bytes = (acc + 3) / 4;
  }

  /* 7. edges among non-contained reads: consecutive overlaps >= min_overlap
   * (the transitive reduction of an exact interval overlap graph), or with
   * full_overlaps every overlapping pair (the graph before that reduction),
   * then repeat-induced ones; pair endpoints are kept-read indices here.
   * Kept reads are sorted by start and none contains another, so their ends
   * increase too and the reads overlapping k by >= min_overlap are k+1 .. */
  int64_t span_total = 0;
  for (int64_t k = 0; k + 1 < K; ++k) {
    int64_t j = k + 1;
    if (f->full_overlaps)
      while (j < K && g->ke[k] - g->ks[j] >= f->min_overlap) ++j;
    else if (g->ke[k] - g->ks[j] >= f->min_overlap)
      ++j;
    span_total += j - (k + 1);
  }
  int64_t cap = span_total + (int64_t)K * (f->k_rep > 0 ? f->k_rep : 0) + 1;
  pair_t* pr = (pair_t*)malloc((size_t)cap * sizeof(pair_t));
  int64_t np = 0;
  for (int64_t k = 0; k + 1 < K; ++k) {
    for (int64_t j = k + 1; j < K && (f->full_overlaps || j == k + 1); ++j) {
      int64_t ov = g->ke[k] - g->ks[j];
      if (ov < f->min_overlap) break;
      pair_t* q = &pr[np++];
      q->a = (int32_t)k; q->b = (int32_t)j; q->is_true = 1; q->pad = 0;
      q->code_ab = (uint8_t)(e_right(g->kst[k]) | (e_left(g->kst[j]) << 1));
      q->code_ba = (uint8_t)(e_left(g->kst[j]) | (e_right(g->kst[k]) << 1));
      q->suf_ab = (int32_t)(g->ke[j] - g->ke[k]);
      q->suf_ba = (int32_t)(g->ks[j] - g->ks[k]);
    }
  }
  if (f->k_rep > 0 && g->n_copy > 0) {
    pair_t* rp = (pair_t*)malloc((size_t)K * f->k_rep * sizeof(pair_t));
    int32_t* rc = (int32_t*)malloc((size_t)K * 4);
    rep_ctx rcx = {g, rp, rc};
    pfor(T, K, rep_range, &rcx);
    for (int64_t a = 0; a < K; ++a) for (int q = 0; q < rc[a]; ++q) pr[np++] = rp[a * f->k_rep + q];
    free(rp); free(rc);
  }
  qsort(pr, (size_t)np, sizeof(pair_t), pair_cmp);
  int64_t nu = 0;
  for (int64_t i = 0; i < np; ++i) {
    if (nu > 0) {
      pair_t* p = &pr[nu - 1];
      int32_t plo = p->a < p->b ? p->a : p->b, phi = p->a < p->b ? p->b : p->a;
      int32_t qlo = pr[i].a < pr[i].b ? pr[i].a : pr[i].b, qhi = pr[i].a < pr[i].b ? pr[i].b : pr[i].a;
      if (plo == qlo && phi == qhi) continue;
    }
    pr[nu++] = pr[i];
  }
  g->n_rep_pairs = 0;
  for (int64_t i = 0; i < nu; ++i) g->n_rep_pairs += pr[i].is_true ? 0 : 1;
  g->n_true_pairs = nu - g->n_rep_pairs;
  for (int64_t i = 0; i < nu; ++i) { /* kept index -> read id */
    pr[i].a = g->id_of[g->kp[pr[i].a]]; pr[i].b = g->id_of[g->kp[pr[i].b]];
  }

  /* 8. CSR in read-id space, rows sorted by column */
  g->m = 2 * nu;
  K = N0;
  g->row_ptr = (int64_t*)calloc((size_t)K + 1, 8);
  g->col = (int32_t*)malloc((size_t)(g->m > 0 ? g->m : 1) * 4);
  g->code = (uint8_t*)malloc((size_t)(g->m > 0 ? g->m : 1));
  g->suf = (int32_t*)malloc((size_t)(g->m > 0 ? g->m : 1) * 4);
  g->is_true = (uint8_t*)malloc((size_t)(g->m > 0 ? g->m : 1));
  for (int64_t i = 0; i < nu; ++i) { g->row_ptr[pr[i].a + 1]++; g->row_ptr[pr[i].b + 1]++; }
  for (int64_t v = 0; v < K; ++v) g->row_ptr[v + 1] += g->row_ptr[v];
  int64_t* fillp = (int64_t*)malloc((size_t)K * 8);
  memcpy(fillp, g->row_ptr, (size_t)K * 8);
  for (int64_t i = 0; i < nu; ++i) {
    int32_t ua = pr[i].a, ub = pr[i].b;
    int64_t x = fillp[ua]++;
    g->col[x] = ub; g->code[x] = pr[i].code_ab; g->suf[x] = pr[i].suf_ab; g->is_true[x] = pr[i].is_true;
    int64_t y = fillp[ub]++;
    g->col[y] = ua; g->code[y] = pr[i].code_ba; g->suf[y] = pr[i].suf_ba; g->is_true[y] = pr[i].is_true;
  }
  free(fillp); free(pr);
  for (int64_t v = 0; v < K; ++v) { /* insertion sort each (short) row by column */
    for (int64_t x = g->row_ptr[v] + 1; x < g->row_ptr[v + 1]; ++x) {
      int32_t c = g->col[x]; uint8_t cd = g->code[x]; int32_t sf = g->suf[x]; uint8_t it = g->is_true[x];
      int64_t y = x - 1;
      while (y >= g->row_ptr[v] && g->col[y] > c) { g->col[y + 1] = g->col[y]; g->code[y + 1] = g->code[y]; g->suf[y + 1] = g->suf[y]; g->is_true[y + 1] = g->is_true[y]; --y; }
      g->col[y + 1] = c; g->code[y + 1] = cd; g->suf[y + 1] = sf; g->is_true[y + 1] = it;
    }
  }
  return g;
}

const char* cg_gen_error(const cg_gen* g) { return g ? g->err : "null"; }

void cg_gen_get_info(const cg_gen* g, cg_gen_info* o) {
  memset(o, 0, sizeof(*o));
  if (!g) return;
  o->genome_len = g->G; o->n_sampled = g->n_sampled; o->n_reads = g->n; o->n_kept = g->n_kept; o->n_entries = g->m;
  o->packed_bytes = g->packed_bytes; o->total_read_bases = g->total_read_bases;
  o->n_true_pairs = g->n_true_pairs; o->n_rep_pairs = g->n_rep_pairs;
  o->n_copies = g->n_copy; o->n_families = g->n_fam;
  int64_t rb = 0; for (int64_t i = 0; i < g->n_copy; ++i) rb += g->copy[i].len;
  o->repeat_bases = rb;
}

int cg_gen_fill(const cg_gen* g, void* row_ptr, int rp_bytes, int32_t* col, uint8_t* code, int32_t* suf,
                int32_t* len, int64_t* off, uint8_t* packed, uint8_t* is_true, int64_t* gstart, uint8_t* strand,
                uint8_t* contained) {
  if (!g || g->err[0]) return -1;
  int64_t K = g->n, m = g->m;
  if (row_ptr) {
    if (rp_bytes == 8) memcpy(row_ptr, g->row_ptr, (size_t)(K + 1) * 8);
    else if (rp_bytes == 4) { if (m > 2147483647ll) return -2; for (int64_t i = 0; i <= K; ++i) ((int32_t*)row_ptr)[i] = (int32_t)g->row_ptr[i]; }
    else return -3;
  }
  if (col) memcpy(col, g->col, (size_t)m * 4);
  if (code) memcpy(code, g->code, (size_t)m);
  if (suf) memcpy(suf, g->suf, (size_t)m * 4);
  if (is_true) memcpy(is_true, g->is_true, (size_t)m);
  if (len) memcpy(len, g->len, (size_t)K * 4);
  if (off) memcpy(off, g->off, (size_t)K * 8);
  if (gstart || strand || contained) for (int64_t id = 0; id < K; ++id) { int64_t k = g->gidx_of[id]; if (gstart) gstart[id] = g->rs[k]; if (strand) strand[id] = g->strand[k]; if (contained) contained[id] = g->contained[k]; }
  if (packed) {
    if (g->cfg.off_align != 32) memset(packed, 0, (size_t)g->packed_bytes);
    pack_ctx pc = {g, packed};
    pfor(g->cfg.threads > 0 ? g->cfg.threads : 1, K, pack_range, &pc);
  }
  return 0;
}

int cg_gen_genome(const cg_gen* g, int64_t start, int64_t count, uint8_t* ascii) {
  static const char A[4] = {'A', 'C', 'G', 'T'};
  if (!g || start < 0 || count < 0 || start + count > g->G) return -1;
  for (int64_t i = 0; i < count; ++i) ascii[i] = (uint8_t)A[gbase(g->g64, start + i)];
  return 0;
}

void cg_gen_free(cg_gen* g) {
  if (!g) return;
  free(g->g64); free(g->copy); free(g->fam); free(g->fam_copies); free(g->famseq);
  free(g->rs); free(g->re); free(g->strand); free(g->contained); free(g->id_of); free(g->gidx_of);
  free(g->ks); free(g->ke); free(g->kp); free(g->kst);
  free(g->row_ptr); free(g->col); free(g->code); free(g->suf); free(g->is_true); free(g->off); free(g->len);
  free(g);
}
