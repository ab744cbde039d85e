/*
 * cg_oracle.c - CPU oracle for contig generation (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, the smoke check and the benchmark's cpu_baseline leg use this
 * file. It is written for a reader to check against the paper by eye:
 * plain loops, no blocking or reordering, one function per step of
 * ContigGeneration (Alg. 2 of Guidi et al., ICPP'22):
 *
 *   BranchRemoval      -> mask_branches()     Sec. 4.2 (degree >= 3), plus the
 *                                             same-end rule for bidirected reads
 *   ConnectedComponent -> components_uf()     Sec. 4.2 (union-find stands in for
 *                         components_bfs()    LACC; BFS is the cross-check)
 *   LocalAssembly      -> walk_component()    Sec. 4.4 (walk from a root vertex)
 *                         pieces()            Sec. 4.4 (each read's part: the suffix
 *                                             form, or l[post : pre] in the x-drop form)
 *                         spell()             Sec. 4.4 (concatenate read parts)
 *
 * and the step before it in Alg. 1: TransitiveReduction -> orc_transitive_reduction()
 * (Sec. 2), plus the input checks of a string graph -> orc_validate2().
 *
 * The partitioning and induced-subgraph steps of Alg. 2 only move data
 * between processes; on one address space they change no result, so the
 * oracle has no counterpart for them except orc_lpt(), the LPT rule itself.
 *
 * Conventions (the graph input format):
 *   bases A=0 C=1 G=2 T=3 in a 2-bit stream (base i: byte i>>2, bits 2*(i&3));
 *   complement of b is 3-b (Sec. 2: A pairs with T, C with G).
 *   entry (u->v): code bit 0 = E_u, bit 1 = E_v, the end of each read the
 *   overlap touches (0 = 5' end of the stored read, 1 = 3' end); suf(u->v) =
 *   bases of v beyond the overlap in walk orientation (Sec. 2, "overhang").
 *   A read with orientation o (0 forward, 1 reverse complement) is left through
 *   end 1-o and entered through end o (a valid walk, Sec. 2).
 *
 * Readings where the paper is silent:
 *   - branch = degree >= 3 (Sec. 4.2) OR exactly two surviving edges on the
 *     same end of the read (no valid walk passes through such a read);
 *     one masking pass, no iteration;
 *   - a component's walk starts at its smaller-id root; a root with one edge
 *     is oriented so that it leaves through that edge; a lone read is forward;
 *   - a component with no root is a cycle: it starts at its smallest read,
 *     forward, leaving through its 3' end, and stops before re-entering it;
 *   - contigs are listed by the smallest read id of their component; chains
 *     with fewer than min_chain_reads reads are not contigs (the paper's own
 *     definition, Sec. 4.4, is min_chain_reads = 2).
 */
#include "cg_oracle.h"

#include <stdio.h>
#include <stdlib.h>
#include <string.h>

struct orc_result {
  int64_t n;
  uint8_t* is_branch;
  int32_t *chain_id, *rank;
  uint8_t* orient;
  int32_t *label_uf, *label_bfs;
  int64_t n_branch, n_contigs, n_cycles, n_components, edges_walked;
  int64_t* contig_off;   /* n_contigs + 1 */
  uint8_t* bases;        /* total_bases ASCII */
  int64_t total_bases;
};

static const char ASCII[4] = {'A', 'C', 'G', 'T'};

static int stored_base(const uint8_t* packed, int64_t off, int64_t k) {
  int64_t q = off + k;
  return (packed[q >> 2] >> (2 * (q & 3))) & 3;
}

/* -------------------------------------------------------------- validate */
/* A string graph as the paper defines it (Sec. 2): every overlap appears in
 * both directions (S is symmetric, Sec. 4.2) with the two end codes swapped,
 * no read overlaps itself, one entry per ordered pair, and a suffix is a
 * proper, non-empty part of the read it extends (no contained reads). */
int orc_validate2(int64_t n, int64_t m, const int64_t* rp, const int32_t* col, const uint8_t* code,
                  const int32_t* suf, const int32_t* pre, const int32_t* post, const int32_t* len,
                  const int64_t* off, int64_t packed_bytes, char* msg, size_t msglen) {
  const int xdrop = pre != NULL && post != NULL;
#define BAD(...) do { if (msg && msglen) snprintf(msg, msglen, __VA_ARGS__); return ORC_EGRAPH; } while (0)
  if (n < 0 || m < 0) BAD("negative size");
  if (rp[0] != 0) BAD("row_ptr[0] != 0");
  for (int64_t v = 0; v < n; ++v) if (rp[v + 1] < rp[v]) BAD("row_ptr decreases at %lld", (long long)v);
  if (rp[n] != m) BAD("row_ptr[n] != n_entries");
  for (int64_t v = 0; v < n; ++v) {
    if (len[v] < 1) BAD("read %lld has length < 1", (long long)v);
    if (off[v] < 0 || off[v] + len[v] > packed_bytes * 4) BAD("read %lld outside the packed stream", (long long)v);
  }
  for (int64_t u = 0; u < n; ++u) {
    for (int64_t x = rp[u]; x < rp[u + 1]; ++x) {
      int64_t v = col[x];
      if (v < 0 || v >= n) BAD("entry %lld: column out of range", (long long)x);
      if (v == u) BAD("entry %lld: self overlap", (long long)x);
      if (code[x] > 3) BAD("entry %lld: code > 3", (long long)x);
      if (xdrop) {                 /* indices into the stored reads u and v (Sec. 4.4) */
        if (pre[x] < 0 || pre[x] > len[u] - 1) BAD("entry %lld: pre outside [0, len-1]", (long long)x);
        if (post[x] < 0 || post[x] > len[v] - 1) BAD("entry %lld: post outside [0, len-1]", (long long)x);
      } else if (suf[x] < 1 || suf[x] > len[v] - 1) {
        BAD("entry %lld: suffix outside [1, len-1]", (long long)x);
      }
      for (int64_t y = rp[u]; y < x; ++y) if (col[y] == v) BAD("entry %lld: duplicate pair", (long long)x);
      int found = 0;
      for (int64_t y = rp[v]; y < rp[v + 1]; ++y) {
        if (col[y] != u) continue;
        ++found;
        uint8_t swapped = (uint8_t)(((code[x] & 1) << 1) | ((code[x] >> 1) & 1));
        if (code[y] != swapped) BAD("entry %lld: mirror code is not the swapped code", (long long)x);
      }
      if (found != 1) BAD("entry %lld: no single mirror entry", (long long)x);
    }
  }
  return ORC_OK;
#undef BAD
}

int orc_validate(int64_t n, int64_t m, const int64_t* rp, const int32_t* col, const uint8_t* code,
                 const int32_t* suf, const int32_t* len, const int64_t* off, int64_t packed_bytes,
                 char* msg, size_t msglen) {
  return orc_validate2(n, m, rp, col, code, suf, NULL, NULL, len, off, packed_bytes, msg, msglen);
}

/* --------------------------------------------------------- BranchRemoval */
/* Sec. 4.2: d = row sums of the 0/1 pattern of S; b = {v : d[v] >= 3}.
 * Same-end rule: a read whose only two edges to non-b reads touch the same
 * end cannot be passed through by a valid walk, so it is a branch too. */
static int64_t mask_branches(int64_t n, const int64_t* rp, const int32_t* col, const uint8_t* code,
                             uint8_t* is_branch) {
  uint8_t* b1 = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  for (int64_t v = 0; v < n; ++v) {
    int64_t d = rp[v + 1] - rp[v];
    b1[v] = (uint8_t)(d >= 3);
  }
  int64_t nb = 0;
  for (int64_t v = 0; v < n; ++v) {
    uint8_t br = b1[v];
    if (!br) {
      int cnt = 0, ends[2] = {-1, -1};
      for (int64_t x = rp[v]; x < rp[v + 1]; ++x) {
        if (b1[col[x]]) continue;
        if (cnt < 2) ends[cnt] = code[x] & 1;
        ++cnt;
      }
      if (cnt == 2 && ends[0] == ends[1]) br = 1;
    }
    is_branch[v] = br;
    nb += br;
  }
  free(b1);
  return nb;
}

/* ---------------------------------------------------- ConnectedComponent */
static int64_t uf_find(int64_t* parent, int64_t v) {
  while (parent[v] != v) { parent[v] = parent[parent[v]]; v = parent[v]; }
  return v;
}

/* label[v] = smallest read id in v's component of L (edges with both ends
 * unmasked), -1 for branch reads. Union-find with path halving. */
static void components_uf(int64_t n, const int64_t* rp, const int32_t* col, const uint8_t* is_branch,
                          int32_t* label) {
  int64_t* parent = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  for (int64_t v = 0; v < n; ++v) parent[v] = v;
  for (int64_t u = 0; u < n; ++u) {
    if (is_branch[u]) continue;
    for (int64_t x = rp[u]; x < rp[u + 1]; ++x) {
      int64_t v = col[x];
      if (is_branch[v]) continue;
      int64_t a = uf_find(parent, u), b = uf_find(parent, v);
      if (a == b) continue;
      if (a < b) parent[b] = a; else parent[a] = b;   /* the root is the smaller id */
    }
  }
  for (int64_t v = 0; v < n; ++v) label[v] = is_branch[v] ? -1 : (int32_t)uf_find(parent, v);
  free(parent);
}

/* The same labels by breadth-first search from each unvisited read in id
 * order (the first read reached is the component's smallest id). */
static void components_bfs(int64_t n, const int64_t* rp, const int32_t* col, const uint8_t* is_branch,
                           int32_t* label) {
  int64_t* queue = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  for (int64_t v = 0; v < n; ++v) label[v] = -2;
  for (int64_t s = 0; s < n; ++s) {
    if (is_branch[s]) { label[s] = -1; continue; }
    if (label[s] != -2) continue;
    int64_t head = 0, tail = 0;
    queue[tail++] = s; label[s] = (int32_t)s;
    while (head < tail) {
      int64_t u = queue[head++];
      for (int64_t x = rp[u]; x < rp[u + 1]; ++x) {
        int64_t v = col[x];
        if (is_branch[v] || label[v] != -2) continue;
        label[v] = (int32_t)s; queue[tail++] = v;
      }
    }
  }
  free(queue);
}

/* ---------------------------------------------------------- LocalAssembly */
/* The L-edge of read v leaving through end e, or -1 (index into the CSR). */
static int64_t edge_at_end(const int64_t* rp, const int32_t* col, const uint8_t* code, const uint8_t* is_branch,
                           int64_t v, int e) {
  for (int64_t x = rp[v]; x < rp[v + 1]; ++x)
    if (!is_branch[col[x]] && (code[x] & 1) == e) return x;
  return -1;
}

static int deg_L(const int64_t* rp, const int32_t* col, const uint8_t* is_branch, int64_t v) {
  int d = 0;
  for (int64_t x = rp[v]; x < rp[v + 1]; ++x) d += !is_branch[col[x]];
  return d;
}

/* One read of a walk: its orientation, the entries through which the walk
 * enters and leaves it (-1: none), and its piece: `contrib` bases of the
 * stored read starting at index `first`, upward when o = 0, downward (and
 * complemented) when o = 1. */
typedef struct { int32_t read; uint8_t o; int64_t x_in, x_out, first, contrib; } step_t;

/* Walk one component (Sec. 4.4): start at root r with orientation o_r, keep
 * leaving the current read through end 1-o and entering the next read w
 * through the edge's far end E_w (so o_w = E_w); stop at a read with no
 * further edge, or when the next read is r again (a cycle). The first read
 * contributes all its bases, each later read the suffix of the edge used. */
static int64_t walk_component(const int64_t* rp, const int32_t* col, const uint8_t* code, const int32_t* suf,
                              const int32_t* len, const uint8_t* is_branch, int64_t r, int o_r, int64_t q,
                              step_t* out, int64_t* edges_touched) {
  int64_t k = 0, cur = r;
  int o = o_r;
  out[k].read = (int32_t)r; out[k].o = (uint8_t)o; out[k].contrib = len[r];
  out[k].x_in = -1; out[k].x_out = -1; ++k;
  for (;;) {
    int64_t x = edge_at_end(rp, col, code, is_branch, cur, 1 - o);
    if (x < 0) break;
    int64_t w = col[x];
    if (w == r) { *edges_touched += 2; break; }   /* the closing edge of a cycle */
    if (k >= q) return -1;                      /* more reads than the component holds */
    *edges_touched += 2;                        /* the entry used and its mirror */
    o = (code[x] >> 1) & 1;
    out[k - 1].x_out = x;
    out[k].read = (int32_t)w; out[k].o = (uint8_t)o; out[k].contrib = suf ? suf[x] : 0;
    out[k].x_in = x; out[k].x_out = -1; ++k;
    cur = w;
  }
  return k;
}

/* The piece of each read of a walk (Sec. 4.4), in stored coordinates.
 * Suffix form: the first read is whole, each later read gives the last
 * suf(e) bases of its oriented sequence (the bases beyond the overlap).
 * x-drop form: the contig is l_r[alpha : pre(e_0)] + l_c1[post(e_0) : pre(e_1)]
 * + ... + l_r'[post(e_last) : beta]: a read runs from post of the entry it is
 * entered through (alpha, its first base in walk direction, for the first
 * read) to pre of the entry it is left through (beta, its last base in walk
 * direction, for the last read). A piece whose end comes before its start in
 * walk direction is empty (the paper does not say). */
static void pieces(step_t* w, int64_t k, const int32_t* pre, const int32_t* post, const int32_t* len) {
  for (int64_t i = 0; i < k; ++i) {
    step_t* s = &w[i];
    const int64_t L = len[s->read];
    const int o = s->o;
    if (pre && post) {
      const int64_t first = s->x_in < 0 ? (o == 0 ? 0 : L - 1) : post[s->x_in];
      const int64_t last = s->x_out < 0 ? (o == 0 ? L - 1 : 0) : pre[s->x_out];
      const int64_t c = o == 0 ? last - first + 1 : first - last + 1;
      s->first = first;
      s->contrib = c > 0 ? c : 0;
    } else {
      /* contrib is already len (first read) or suf(e_in); the last contrib
       * oriented bases start at stored index L - contrib (o = 0) or contrib - 1 */
      s->first = o == 0 ? L - s->contrib : s->contrib - 1;
    }
  }
}

/* Bases of one step (Sec. 4.4: l[i:j] for i<j is forward, l[j:i] its reverse
 * complement): contrib bases from stored index `first`, upward for o = 0,
 * downward and complemented for o = 1. */
static void spell(const uint8_t* packed, int64_t off, int o, int64_t first, int64_t contrib, uint8_t* out) {
  for (int64_t t = 0; t < contrib; ++t) {
    int b = (o == 0) ? stored_base(packed, off, first + t) : 3 - stored_base(packed, off, first - t);
    out[t] = (uint8_t)ASCII[b];
  }
}

orc_result* orc_run2(int64_t n, int64_t m, const int64_t* rp, const int32_t* col, const uint8_t* code,
                     const int32_t* suf, const int32_t* pre, const int32_t* post, const int32_t* len,
                     const int64_t* off, const uint8_t* packed, int64_t packed_bytes, int32_t min_chain_reads,
                     int validate, int* status) {
  *status = ORC_OK;
  if (!(pre && post)) pre = post = NULL;
  if (validate) {
    int s = orc_validate2(n, m, rp, col, code, suf, pre, post, len, off, packed_bytes, NULL, 0);
    if (s != ORC_OK) { *status = s; return NULL; }
  }
  if (min_chain_reads < 1) min_chain_reads = 1;
  orc_result* r = (orc_result*)calloc(1, sizeof(orc_result));
  size_t nn = (size_t)(n > 0 ? n : 1);
  r->n = n;
  r->is_branch = (uint8_t*)calloc(nn, 1);
  r->chain_id = (int32_t*)malloc(nn * 4); r->rank = (int32_t*)malloc(nn * 4); r->orient = (uint8_t*)malloc(nn);
  r->label_uf = (int32_t*)malloc(nn * 4); r->label_bfs = (int32_t*)malloc(nn * 4);

  /* 1. BranchRemoval (Alg. 2, first step) */
  r->n_branch = mask_branches(n, rp, col, code, r->is_branch);

  /* 2. ConnectedComponent on L */
  components_uf(n, rp, col, r->is_branch, r->label_uf);
  components_bfs(n, rp, col, r->is_branch, r->label_bfs);

  /* group members by label (counting sort by label, members in id order) */
  int64_t* cnt = (int64_t*)calloc(nn + 1, sizeof(int64_t));
  for (int64_t v = 0; v < n; ++v) if (r->label_uf[v] >= 0) cnt[r->label_uf[v] + 1]++;
  for (int64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
  int64_t* members = (int64_t*)malloc(nn * sizeof(int64_t));
  int64_t* fillp = (int64_t*)malloc(nn * sizeof(int64_t));
  memcpy(fillp, cnt, nn * sizeof(int64_t));
  for (int64_t v = 0; v < n; ++v) if (r->label_uf[v] >= 0) members[fillp[r->label_uf[v]]++] = v;
  free(fillp);

  for (int64_t v = 0; v < n; ++v) { r->chain_id[v] = -1; r->rank[v] = -1; r->orient[v] = 255; }

  /* 3. LocalAssembly: components in order of their smallest read id */
  step_t* walk = (step_t*)malloc(nn * sizeof(step_t));
  int64_t* wstart = (int64_t*)malloc((nn + 1) * sizeof(int64_t));
  int64_t* cstart = (int64_t*)malloc((nn + 1) * sizeof(int64_t));
  int64_t nw = 0, nc = 0, total = 0;
  for (int64_t c = 0; c < n; ++c) {
    int64_t q = cnt[c + 1] - cnt[c];
    if (q == 0) continue;                          /* c is not a component's smallest id */
    r->n_components++;
    int64_t root = -1;
    int o_root = 0;
    for (int64_t i = cnt[c]; i < cnt[c + 1]; ++i) {  /* members in increasing id */
      int64_t v = members[i];
      int d = deg_L(rp, col, r->is_branch, v);
      if (d <= 1) {
        root = v;
        if (d == 1) {
          int64_t x = edge_at_end(rp, col, code, r->is_branch, v, 0);
          int e = (x >= 0) ? 0 : 1;
          o_root = 1 - e;                          /* leave through the one edge */
        } else {
          o_root = 0;
        }
        break;
      }
    }
    int cycle = 0;
    if (root < 0) { root = c; o_root = 0; cycle = 1; }   /* no root: a cycle */
    int64_t k = walk_component(rp, col, code, suf, len, r->is_branch, root, o_root, q, walk + nw, &r->edges_walked);
    if (k != q) {                                        /* the walk must visit the whole component */
      *status = ORC_EINTERNAL;
      break;
    }
    r->n_cycles += cycle;
    if (q < min_chain_reads) continue;
    pieces(walk + nw, k, pre, post, len);
    wstart[nc] = nw; cstart[nc] = total;
    for (int64_t i = 0; i < k; ++i) {
      step_t* s = &walk[nw + i];
      r->chain_id[s->read] = (int32_t)c; r->rank[s->read] = (int32_t)i; r->orient[s->read] = s->o;
      total += s->contrib;
    }
    nw += k; ++nc;
  }
  wstart[nc] = nw; cstart[nc] = total;
  r->n_contigs = nc; r->total_bases = total;
  r->contig_off = (int64_t*)malloc((size_t)(nc + 1) * sizeof(int64_t));
  memcpy(r->contig_off, cstart, (size_t)(nc + 1) * sizeof(int64_t));
  r->bases = (uint8_t*)malloc((size_t)(total > 0 ? total : 1));
  if (*status == ORC_OK) {
    int64_t pos = 0;
    for (int64_t i = 0; i < nw; ++i) {
      step_t* s = &walk[i];
      spell(packed, off[s->read], s->o, s->first, s->contrib, r->bases + pos);
      pos += s->contrib;
    }
  }
  free(cnt); free(members); free(walk); free(wstart); free(cstart);
  if (*status != ORC_OK) { orc_free(r); return NULL; }
  return r;
}

orc_result* orc_run(int64_t n, int64_t m, const int64_t* rp, const int32_t* col, const uint8_t* code,
                    const int32_t* suf, const int32_t* len, const int64_t* off, const uint8_t* packed,
                    int64_t packed_bytes, int32_t min_chain_reads, int validate, int* status) {
  return orc_run2(n, m, rp, col, code, suf, NULL, NULL, len, off, packed, packed_bytes, min_chain_reads, validate,
                  status);
}

int64_t orc_n_branch(const orc_result* r) { return r->n_branch; }
int64_t orc_n_contigs(const orc_result* r) { return r->n_contigs; }
int64_t orc_n_cycles(const orc_result* r) { return r->n_cycles; }
int64_t orc_total_bases(const orc_result* r) { return r->total_bases; }
int64_t orc_n_components(const orc_result* r) { return r->n_components; }
int64_t orc_edge_entries_walked(const orc_result* r) { return r->edges_walked; }
void orc_get_branch(const orc_result* r, uint8_t* b) { memcpy(b, r->is_branch, (size_t)r->n); }
void orc_get_chains(const orc_result* r, int32_t* cid, int32_t* rank, uint8_t* orient) {
  if (cid) memcpy(cid, r->chain_id, (size_t)r->n * 4);
  if (rank) memcpy(rank, r->rank, (size_t)r->n * 4);
  if (orient) memcpy(orient, r->orient, (size_t)r->n);
}
void orc_get_contigs(const orc_result* r, int64_t* contig_off, uint8_t* bases) {
  if (contig_off) memcpy(contig_off, r->contig_off, (size_t)(r->n_contigs + 1) * 8);
  if (bases) memcpy(bases, r->bases, (size_t)r->total_bases);
}
void orc_get_labels(const orc_result* r, int which, int32_t* label) {
  memcpy(label, which ? r->label_bfs : r->label_uf, (size_t)r->n * 4);
}
void orc_free(orc_result* r) {
  if (!r) return;
  free(r->is_branch); free(r->chain_id); free(r->rank); free(r->orient);
  free(r->label_uf); free(r->label_bfs); free(r->contig_off); free(r->bases);
  free(r);
}

void orc_revcomp(const char* in, int64_t n, char* out) {
  for (int64_t i = 0; i < n; ++i) {
    char c = in[n - 1 - i], d = 'N';
    switch (c) { case 'A': d = 'T'; break; case 'T': d = 'A'; break; case 'C': d = 'G'; break; case 'G': d = 'C'; break; }
    out[i] = d;
  }
}

/* Sec. 4.3: sort the sizes in decreasing order, then put each one in the
 * bin whose current sum is smallest. */
/* ------------------------------------------------- TransitiveReduction */
/* Alg. 1 (S <- TransitiveReduction(R)), Sec. 2: an overlap whose information
 * a parallel path already carries is redundant. Entry x = (u->w) is
 * transitive when some read v (not u, not w) gives a valid walk u -> v -> w
 * that leaves u through the same end as x, passes through v (entered through
 * one end, left through the other) and enters w through the same end as x,
 * and whose suffixes add up to x's: |suf(u->v) + suf(v->w) - suf(u->w)| <=
 * fuzz. A pair of reads keeps its two entries only when neither is
 * transitive. Rows keep their order; returns the number of entries kept. */
int64_t orc_transitive_reduction(int64_t n, int64_t m, const int64_t* rp, const int32_t* col, const uint8_t* code,
                                 const int32_t* suf, int32_t fuzz, int64_t* out_rp, int32_t* out_col,
                                 uint8_t* out_code, int32_t* out_suf) {
  uint8_t* trans = (uint8_t*)calloc((size_t)(m > 0 ? m : 1), 1);
  for (int64_t u = 0; u < n; ++u) {
    for (int64_t x = rp[u]; x < rp[u + 1]; ++x) {
      const int64_t w = col[x];
      const int eu = code[x] & 1, ew = (code[x] >> 1) & 1;
      for (int64_t y = rp[u]; y < rp[u + 1] && !trans[x]; ++y) {
        const int64_t v = col[y];
        if (v == w || (code[y] & 1) != eu) continue;          /* leave u through x's end */
        const int ev_in = (code[y] >> 1) & 1;
        for (int64_t z = rp[v]; z < rp[v + 1]; ++z) {
          if (col[z] != w) continue;
          if ((code[z] & 1) != 1 - ev_in) continue;            /* leave v through its other end */
          if (((code[z] >> 1) & 1) != ew) continue;            /* enter w through x's end */
          const int64_t d = (int64_t)suf[y] + suf[z] - suf[x];
          if (d <= fuzz && d >= -fuzz) { trans[x] = 1; break; }
        }
      }
    }
  }
  int64_t k = 0;
  out_rp[0] = 0;
  for (int64_t u = 0; u < n; ++u) {
    for (int64_t x = rp[u]; x < rp[u + 1]; ++x) {
      const int64_t w = col[x];
      int mirror_trans = 0;
      for (int64_t y = rp[w]; y < rp[w + 1]; ++y)
        if (col[y] == u) mirror_trans = trans[y];
      if (trans[x] || mirror_trans) continue;
      out_col[k] = col[x]; out_code[k] = code[x]; out_suf[k] = suf[x];
      ++k;
    }
    out_rp[u + 1] = k;
  }
  free(trans);
  return k;
}

int orc_lpt(const int64_t* sizes, int64_t k, int32_t P, int32_t* assign, int64_t* loads) {
  if (P < 1 || k < 0) return ORC_EGRAPH;
  int64_t* order = (int64_t*)malloc((size_t)(k > 0 ? k : 1) * sizeof(int64_t));
  for (int64_t i = 0; i < k; ++i) order[i] = i;
  for (int64_t i = 1; i < k; ++i) {                  /* stable insertion sort, decreasing size */
    int64_t j = i, t = order[i];
    while (j > 0 && sizes[order[j - 1]] < sizes[t]) { order[j] = order[j - 1]; --j; }
    order[j] = t;
  }
  for (int32_t b = 0; b < P; ++b) loads[b] = 0;
  for (int64_t i = 0; i < k; ++i) {
    int32_t best = 0;
    for (int32_t b = 1; b < P; ++b) if (loads[b] < loads[best]) best = b;
    assign[order[i]] = best;
    loads[best] += sizes[order[i]];
  }
  free(order);
  return ORC_OK;
}
