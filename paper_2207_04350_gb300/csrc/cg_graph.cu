// cg_graph.cu - graph stage of contig generation on sm_103a:
//   input checks, BranchRemoval (Alg. 2, Sec. 4.2), the oriented successor
//   table of the unbranched matrix L, and chain discovery by list ranking
//   (the GPU counterpart of ConnectedComponent + the walk order of
//   LocalAssembly, Sec. 4.2 and 4.4).
//
// Chains as linked lists. Every unmasked read v becomes two oriented reads
// x = 2v + o (o = 0 forward, 1 reverse complement). Oriented read (v,o) leaves
// v through end 1-o; if L has the overlap (v->w) on that end, its successor
// is (w, E_w), the orientation in which w is entered. Each chain thus appears
// as two directed lists, one the reverse of the other, and a closed chain as
// two directed cycles. (v,o) has a predecessor exactly when (v,1-o) has a
// successor.
//
// List ranking (Helman-JaJa style sublists): every list head and every read
// whose hash falls in a 2^-k sample starts a sublist; one thread walks each
// sublist to the next sublist start, then pointer jumping over the (few)
// sublists gives each one its distance to the list tail, the tail itself and
// the smallest read id up to the tail. A read then knows, from its two
// oriented copies, the chain's length, both end reads, its position from
// either end, and the chain's smallest read id. Closed chains (no tail) are
// detected after the jumping and ranked separately from their smallest read.
#include <cuda_runtime.h>

#include "cg_internal.cuh"

namespace cg {

namespace {

constexpr long long kSpinLimit = 1ll << 22;   // barrier polls before giving up (~1 s with backoff)

__device__ __forceinline__ int sampled(int v, int ruler_log2) {
  unsigned h = (unsigned)v * 0x9E3779B1u;
  h ^= h >> 15;
  h *= 0x85EBCA77u;
  h ^= h >> 13;
  return (h & ((1u << ruler_log2) - 1u)) == 0u;
}

// Software grid barrier for kernels launched cooperatively (all blocks
// co-resident). Bounded: a block that waits too long records DERR_TIMEOUT and
// every block returns false from then on.
__device__ bool grid_sync(Counters* c, DevError* e) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* gen = &c->bar_gen;
    unsigned g0 = *gen;
    __threadfence();
    unsigned arrived = atomicAdd(&c->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      c->bar_count = 0;
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      long long spins = 0;
      while (*gen == g0) {
        if (++spins > kSpinLimit || *(volatile int*)&e->err == DERR_TIMEOUT) {
          set_error(e, DERR_TIMEOUT, K_JUMP, spins);
          ok = 0;
          break;
        }
        __nanosleep(spins < 64 ? 32 : 256);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// -------------------------------------------------------------- validation
__global__ void k_validate_reads(DevGraph g, DevError* c) {
  for (long long v = grid_tid(); v < g.n; v += grid_threads()) {
    int64_t a = rowp(g, v), b = rowp(g, v + 1);
    if (b < a) set_error(c, DERR_GRAPH, K_VALIDATE1, v);
    int32_t L = g.len[v];
    int64_t o = g.off[v];
    if (L < 1 || o < 0 || o + L > g.packed_bytes * 4) set_error(c, DERR_GRAPH, K_VALIDATE1, v);
  }
  if (grid_tid() == 0) {
    if (rowp(g, 0) != 0 || rowp(g, g.n) != g.m) set_error(c, DERR_GRAPH, K_VALIDATE1, -1);
  }
}

__global__ void k_validate_entries(DevGraph g, DevError* c) {
  // Row bounds are clamped to [0, m] so that a malformed row_ptr (reported by
  // k_validate_reads, which runs just before without a wait) reads nothing
  // outside the arrays.
  for (long long u = grid_tid(); u < g.n; u += grid_threads()) {
    int64_t a = max((int64_t)0, min(rowp(g, u), g.m)), b = max(a, min(rowp(g, u + 1), g.m));
    for (int64_t x = a; x < b; ++x) {
      int32_t v = g.col[x];
      uint8_t cd = g.code[x];
      if (v < 0 || v >= g.n || v == u || cd > 3) { set_error(c, DERR_GRAPH, K_VALIDATE2, x); continue; }
      int32_t s = g.suf[x];
      if (s < 1 || s > g.len[v] - 1) set_error(c, DERR_GRAPH, K_VALIDATE2, x);
      for (int64_t y = a; y < x; ++y)
        if (g.col[y] == v) set_error(c, DERR_GRAPH, K_VALIDATE2, x);
      int64_t va = max((int64_t)0, min(rowp(g, v), g.m)), vb = max(va, min(rowp(g, v + 1), g.m));
      int found = 0;
      uint8_t want = (uint8_t)(((cd & 1) << 1) | (cd >> 1));
      for (int64_t y = va; y < vb; ++y) {
        if (g.col[y] != u) continue;
        ++found;
        if (g.code[y] != want) set_error(c, DERR_GRAPH, K_VALIDATE2, x);
      }
      if (found != 1) set_error(c, DERR_GRAPH, K_VALIDATE2, x);
    }
  }
}

// ----------------------------------------------------------- BranchRemoval
// d[v] = row length of S (Sec. 4.2); d >= 3 is a branch. A read of degree
// <= 2 whose overlaps to reads of degree <= 2 are exactly two, both on the
// same end, cannot be passed by a valid walk and is a branch too. Reads with
// no overlap are lone reads: a one-read contig when min_chain <= 1.
constexpr int kMaskItems = 4;

__global__ void __launch_bounds__(kBlock) k_mask(DevGraph g, Scratch s) {
  Counters* c = s.ctr;
  unsigned long long nb = 0;
  const long long step = (long long)gridDim.x * kBlock * kMaskItems;
  for (long long base = (long long)blockIdx.x * kBlock * kMaskItems; base < g.n; base += step) {  // block-uniform
    unsigned candm = 0, lonem = 0;
    for (int k = 0; k < kMaskItems; ++k) {
      long long v = base + (long long)k * kBlock + threadIdx.x;
      if (v >= g.n) continue;
      int64_t a = rowp(g, v), b = rowp(g, v + 1);
      int64_t d = b - a;
      uint8_t br = 0;
      if (d >= 3) {
        br = 1;
      } else if (d > 0) {
        int cnt = 0, e0 = -1, e1 = -1;
        for (int64_t x = a; x < b; ++x) {
          int32_t w = g.col[x];
          int64_t dw = rowp(g, w + 1) - rowp(g, w);
          if (dw >= 3) continue;
          int e = g.code[x] & 1;
          if (cnt == 0) e0 = e; else e1 = e;
          ++cnt;
        }
        br = (cnt == 2 && e0 == e1) ? 1 : 0;
      }
      s.branch[v] = br;
      nb += br;
      if (br) {
        s.headq[v] = 0;
      } else if (d == 0) {
        bool lone = g.min_chain <= 1;
        s.headq[v] = lone ? 1 : 0;
        if (lone) {
          s.cid[v] = (int32_t)v; s.rank[v] = 0; s.orient[v] = 0; s.contrib[v] = g.len[v];
          lonem |= 1u << k;
        }
      } else {
        candm |= 1u << k;
      }
    }
    unsigned cs = block_reserve(&c->n_cand, __popc(candm));
    unsigned ls = block_reserve(&c->n_lone, __popc(lonem));
    for (int k = 0; k < kMaskItems; ++k) {
      int32_t v = (int32_t)(base + (long long)k * kBlock + threadIdx.x);
      if ((candm >> k) & 1u) s.cand[cs++] = v;
      if ((lonem >> k) & 1u) s.emit[ls++] = v;
    }
  }
  for (int o = 16; o > 0; o >>= 1) nb += __shfl_down_sync(0xffffffffu, nb, o);
  if ((threadIdx.x & 31) == 0 && nb) atomicAdd(&c->n_branch, nb);
}

// Successor table of L for the unmasked reads that have overlaps:
// succ[v] = (successor of (v,0), successor of (v,1)); the overlap (v->w)
// on end E_v is the way out of (v, 1-E_v) and enters (w, E_w), whose
// incoming suffix is suf(v->w).
__global__ void k_succ(DevGraph g, Scratch s) {
  Counters* c = s.ctr;
  long long n = block_round(*(volatile unsigned*)&c->n_cand);
  for (long long i = grid_tid(); i < n; i += grid_threads()) {
    bool valid = i < c->n_cand;
    bool chain = false, lone = false;
    int32_t v = 0;
    if (valid) {
      v = s.cand[i];
      int64_t a = rowp(g, v), b = rowp(g, v + 1);
      int s0 = -1, s1 = -1;
      for (int64_t x = a; x < b; ++x) {
        int32_t w = g.col[x];
        if (s.branch[w]) continue;
        int cd = g.code[x];
        int ev = cd & 1, ew = cd >> 1;
        int to = 2 * w + ew;
        if (ev == 1) s0 = to; else s1 = to;
        s.sufin[to] = g.suf[x];
      }
      s.succ[v] = make_int2(s0, s1);
      if (s0 < 0 && s1 < 0) {
        lone = g.min_chain <= 1;
        s.headq[v] = lone ? 1 : 0;
        s.cid[v] = lone ? v : -1;
        s.rank[v] = lone ? 0 : -1;
        s.orient[v] = lone ? 0 : 255;
        s.contrib[v] = g.len[v];
        if (lone) atomicAdd(&c->n_heads, 1u);
      } else {
        chain = true;
        // not yet reached by a sublist walk (closed chains without a
        // sampled read are never reached, and are found by this mark)
        s.rid[2 * v] = -1;
        s.rid[2 * v + 1] = -1;
      }
    }
    unsigned slot = block_reserve(&c->n_chain, chain ? 1u : 0u);
    if (chain) s.chain[slot] = v;
    unsigned eslot = block_reserve(&c->n_emit, lone ? 1u : 0u);
    if (lone) s.emit[eslot] = v;
  }
}

// One thread per sublist start: walk to the next start or the list end.
__global__ void k_walk(Scratch s, int ruler_log2, int64_t limit) {
  Counters* c = s.ctr;
  long long nodes = block_round(2ll * *(volatile unsigned*)&c->n_chain);
  for (long long i = grid_tid(); i < nodes; i += grid_threads()) {
    bool valid = i < 2ll * c->n_chain;
    bool ruler = false;
    int32_t v = 0, o = 0, nx = -1;
    if (valid) {
      v = s.chain[i >> 1];
      o = (int)(i & 1);
      int2 sv = s.succ[v];
      int pred = o == 0 ? sv.y : sv.x;  // (v,o) has a predecessor iff (v,1-o) has a successor
      nx = o == 0 ? sv.x : sv.y;
      ruler = pred < 0 || sampled(v, ruler_log2);
    }
    unsigned r = block_reserve(&c->n_rulers, ruler ? 1u : 0u);
    if (!ruler) continue;
    int32_t y = 2 * v + o, z = nx, mn = v, last = y, next_start = -1;
    int32_t cnt = 0;
    for (;;) {
      s.rid[y] = (int32_t)r;
      s.roff[y] = cnt;
      ++cnt;
      mn = min(mn, y >> 1);
      last = y;
      if (z < 0) break;
      if (sampled(z >> 1, ruler_log2)) { next_start = z; break; }
      int2 sz = s.succ[z >> 1];
      y = z;
      z = (z & 1) ? sz.y : sz.x;
      if (cnt > limit) { set_error(s.derr, DERR_KERNEL, K_WALK, y); break; }
    }
    s.r_next_node[r] = next_start;
    s.r_len[r] = cnt;
    s.r_min[r] = mn;
    s.r_last[r] = last;
  }
}

// Pointer jumping over the sublists (grid-synchronised rounds). After it,
// for a sublist on an open list: acc = oriented reads from its start to the
// list tail, mn = smallest read id over that span, tail = last sublist.
// Sublists on directed cycles keep next >= 0.
__global__ void k_jump(Scratch s) {
  Counters* c = s.ctr;
  unsigned R = *(volatile unsigned*)&c->n_rulers;
  for (long long i = grid_tid(); i < R; i += grid_threads()) {
    int32_t nn = s.r_next_node[i];
    s.pj_next[0][i] = nn >= 0 ? s.rid[nn] : -1;
    s.pj_acc[0][i] = s.r_len[i];
    s.pj_min[0][i] = s.r_min[i];
    s.pj_tail[0][i] = (int32_t)i;
  }
  int rounds = 1;
  while ((1u << rounds) < R + 1u && rounds < 31) ++rounds;
  ++rounds;
  int cur = 0;
  if (!grid_sync(c, s.derr)) return;
  for (int r = 0; r < rounds; ++r) {
    int nxt = cur ^ 1;
    unsigned active = 0;
    for (long long i = grid_tid(); i < R; i += grid_threads()) {
      int32_t j = s.pj_next[cur][i];
      if (j >= 0) {
        long long acc = (long long)s.pj_acc[cur][i] + s.pj_acc[cur][j];
        s.pj_acc[nxt][i] = acc > 0x7fffffffll ? 0x7fffffff : (int32_t)acc;   // saturates on cycles
        s.pj_min[nxt][i] = min(s.pj_min[cur][i], s.pj_min[cur][j]);
        s.pj_tail[nxt][i] = s.pj_tail[cur][j];
        int32_t jj = s.pj_next[cur][j];
        s.pj_next[nxt][i] = jj;
        active |= (jj >= 0);
      } else {
        s.pj_acc[nxt][i] = s.pj_acc[cur][i];
        s.pj_min[nxt][i] = s.pj_min[cur][i];
        s.pj_tail[nxt][i] = s.pj_tail[cur][i];
        s.pj_next[nxt][i] = -1;
      }
    }
    active = __syncthreads_or(active);
    if (threadIdx.x == 0 && active) atomicOr(&c->round_flag[r], 1u);   // zeroed by the stage
    cur = nxt;
    if (!grid_sync(c, s.derr)) return;
    if (*(volatile unsigned*)&c->round_flag[r] == 0) break;
  }
  if (grid_tid() == 0) c->final_buf = (unsigned)cur;
}

// Per chain read: combine its two oriented copies. head(list of (v,0)) is
// the reverse of tail(list of (v,1)). The contig starts at the smaller-id
// end read, so (v,0) is the walk orientation when that end heads the list
// of (v,0).
__global__ void k_final(DevGraph g, Scratch s) {
  Counters* c = s.ctr;
  int fb = (int)*(volatile unsigned*)&c->final_buf;
  long long n = block_round(*(volatile unsigned*)&c->n_chain);
  const int32_t* nx = s.pj_next[fb];
  const int32_t* acc = s.pj_acc[fb];
  const int32_t* mnv = s.pj_min[fb];
  const int32_t* tl = s.pj_tail[fb];
  for (long long k = grid_tid(); k < n; k += grid_threads()) {
    bool valid = k < c->n_chain;
    bool cyc = false, emit = false;
    int32_t v = 0;
    if (valid) {
      v = s.chain[k];
      int32_t x0 = 2 * v, x1 = x0 + 1;
      int32_t i0 = s.rid[x0], i1 = s.rid[x1];
      if (i0 < 0 || i1 < 0 || nx[i0] >= 0 || nx[i1] >= 0) {
        cyc = true;
      } else {
        int32_t d0 = acc[i0] - s.roff[x0] - 1;
        int32_t d1 = acc[i1] - s.roff[x1] - 1;
        int32_t t0 = s.r_last[tl[i0]];
        int32_t t1 = s.r_last[tl[i1]];
        int32_t h0 = t1 >> 1, h1 = t0 >> 1;       // first read of the list of (v,0) / (v,1)
        int32_t hr = s.rid[t1 ^ 1];                // the head of (v,0)'s list starts a sublist
        int32_t m = hr >= 0 ? mnv[hr] : -1;
        int32_t q = d0 + d1 + 1;
        int o = h0 < h1 ? 0 : 1;
        int32_t rk = o == 0 ? d1 : d0;
        if (m < 0 || h0 == h1) set_error(s.derr, DERR_KERNEL, K_FINAL, v);
        if (q >= g.min_chain) {
          emit = true;
          s.cid[v] = m;
          s.rank[v] = rk;
          s.orient[v] = (uint8_t)o;
          s.contrib[v] = rk == 0 ? g.len[v] : s.sufin[x0 + o];
          s.headq[v] = (v == m) ? q : 0;
          if (v == m) atomicAdd(&c->n_heads, 1u);
        } else {
          s.cid[v] = -1;
          s.rank[v] = -1;
          s.orient[v] = 255;
          s.headq[v] = 0;
        }
      }
    }
    unsigned slot = block_reserve(&c->n_cycle_reads, cyc ? 1u : 0u);
    if (cyc) s.cyc[slot] = v;
    unsigned eslot = block_reserve(&c->n_emit, emit ? 1u : 0u);
    if (emit) s.emit[eslot] = v;
  }
}

// Closed chains (rare). Over their oriented reads: pointer jumping for the
// smallest oriented id of each directed cycle (the copy holding (m,0) is the
// walk, m the smallest read), then cut the walk before (m,0) and rank by
// pointer jumping again.
__global__ void k_cycles(DevGraph g, Scratch s) {
  Counters* c = s.ctr;
  unsigned C = *(volatile unsigned*)&c->n_cycle_reads;
  if (C == 0) return;
  long long N = 2ll * C;
  for (long long i = grid_tid(); i < N; i += grid_threads()) {
    int32_t v = s.cyc[i >> 1], y = 2 * v + (int)(i & 1);
    int2 sv = s.succ[v];
    int32_t z = (y & 1) ? sv.y : sv.x;
    if (z < 0) set_error(s.derr, DERR_KERNEL, K_CYCLE, y);
    s.c_ptr[0][y] = z;
    s.c_val[0][y] = y;
  }
  int rounds = 1;
  while ((1ll << rounds) < N + 1 && rounds < 31) ++rounds;
  ++rounds;
  int cur = 0;
  if (!grid_sync(c, s.derr)) return;
  for (int r = 0; r < rounds; ++r) {
    int nxt = cur ^ 1;
    for (long long i = grid_tid(); i < N; i += grid_threads()) {
      int32_t y = 2 * s.cyc[i >> 1] + (int)(i & 1);
      int32_t p = s.c_ptr[cur][y];
      if (p < 0) continue;
      s.c_val[nxt][y] = min(s.c_val[cur][y], s.c_val[cur][p]);
      s.c_ptr[nxt][y] = s.c_ptr[cur][p];
    }
    cur = nxt;
    if (!grid_sync(c, s.derr)) return;
  }
  // cut: on the walk copy, the oriented read before the start has no successor
  for (long long i = grid_tid(); i < N; i += grid_threads()) {
    int32_t v = s.cyc[i >> 1], y = 2 * v + (int)(i & 1);
    int32_t head = s.c_val[cur][y];
    s.c_head[y] = head;
    if ((head & 1) == 0) {
      int2 sv = s.succ[v];
      int32_t z = (y & 1) ? sv.y : sv.x;
      int32_t p = (z == head) ? -1 : z;
      s.c_ptr[0][y] = p;
      s.c_val[0][y] = p < 0 ? 0 : 1;
    }
  }
  cur = 0;
  if (!grid_sync(c, s.derr)) return;
  for (int r = 0; r < rounds; ++r) {
    int nxt = cur ^ 1;
    for (long long i = grid_tid(); i < N; i += grid_threads()) {
      int32_t y = 2 * s.cyc[i >> 1] + (int)(i & 1);
      if (s.c_head[y] & 1) continue;
      int32_t p = s.c_ptr[cur][y];
      if (p >= 0) {
        s.c_val[nxt][y] = s.c_val[cur][y] + s.c_val[cur][p];
        s.c_ptr[nxt][y] = s.c_ptr[cur][p];
      } else {
        s.c_val[nxt][y] = s.c_val[cur][y];
        s.c_ptr[nxt][y] = -1;
      }
    }
    cur = nxt;
    if (!grid_sync(c, s.derr)) return;
  }
  long long NN = block_round(N);
  for (long long i = grid_tid(); i < NN; i += grid_threads()) {
    bool emit = false;
    int32_t v = 0;
    if (i < N) {
      v = s.cyc[i >> 1];
      int32_t y = 2 * v + (int)(i & 1);
      int32_t head = s.c_head[y];
      if ((head & 1) == 0) {
        int32_t L = s.c_val[cur][head] + 1;       // distance from the start to the cut, plus one
        int32_t rk = L - 1 - s.c_val[cur][y];
        int32_t m = head >> 1;
        if (L >= g.min_chain) {
          emit = true;
          s.cid[v] = m;
          s.rank[v] = rk;
          s.orient[v] = (uint8_t)(y & 1);
          s.contrib[v] = rk == 0 ? g.len[v] : s.sufin[y];
          s.headq[v] = rk == 0 ? L : 0;
          if (rk == 0) atomicAdd(&c->n_heads, 1u);
        } else {
          s.cid[v] = -1;
          s.rank[v] = -1;
          s.orient[v] = 255;
          s.headq[v] = 0;
        }
        if (rk == 0) atomicAdd(&c->n_cycles, 1u);
      }
    }
    unsigned eslot = block_reserve(&c->n_emit, emit ? 1u : 0u);
    if (emit) s.emit[eslot] = v;
  }
}

__global__ void k_export_reads(DevGraph g, Scratch s, int32_t* cid, int32_t* rank, uint8_t* orient) {
  for (long long v = grid_tid(); v < g.n; v += grid_threads()) {
    int64_t d = rowp(g, v + 1) - rowp(g, v);
    int32_t a = -1, b = -1;
    uint8_t o = 255;
    if (d == 0) {
      if (g.min_chain <= 1) { a = (int32_t)v; b = 0; o = 0; }
    } else if (!s.branch[v]) {
      a = s.cid[v]; b = s.rank[v]; o = s.orient[v];
    }
    if (cid) cid[v] = a;
    if (rank) rank[v] = b;
    if (orient) orient[v] = o;
  }
}

__global__ void k_sum_len(DevGraph g, unsigned long long* out) {
  unsigned long long acc = 0;
  for (long long v = grid_tid(); v < g.n; v += grid_threads()) acc += (unsigned long long)g.len[v];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

cudaError_t coop(const void* fn, int blocks, void** args, const LaunchEnv& env) {
  ++*env.launches;
  return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(kBlock), args, 0, env.stream);
}

}  // namespace

int coop_blocks_for_grid_kernels(int num_sms) {
  int a = 0, b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_jump, kBlock, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cycles, kBlock, 0);
  int per = a < b ? a : b;
  if (per > 4) per = 4;
  if (per < 1) per = 1;
  return per * num_sms;
}

cudaError_t launch_validate(const DevGraph& g, DevError* derr, const LaunchEnv& env) {
  k_validate_reads<<<grid_for(g.n, env), kBlock, 0, env.stream>>>(g, derr);
  ++*env.launches;
  k_validate_entries<<<grid_for(g.n, env), kBlock, 0, env.stream>>>(g, derr);
  ++*env.launches;
  return cudaGetLastError();
}

cudaError_t launch_sum_len(const DevGraph& g, unsigned long long* out, const LaunchEnv& env) {
  k_sum_len<<<grid_for(g.n, env), kBlock, 0, env.stream>>>(g, out);
  ++*env.launches;
  return cudaGetLastError();
}

cudaError_t launch_mask(const DevGraph& g, const Scratch& s, const LaunchEnv& env) {
  cudaMemsetAsync(&s.ctr->n_branch, 0, sizeof(Counters) - offsetof(Counters, n_branch), env.stream);
  k_mask<<<grid_for(g.n, env), kBlock, 0, env.stream>>>(g, s);
  ++*env.launches;
  return cudaGetLastError();
}

cudaError_t launch_chains(const DevGraph& g, const Scratch& s, const Tuning& t, const LaunchEnv& env) {
  // restart the chain-stage counters; the walk list starts after the lone
  // reads the mask stage already placed in it
  cudaMemsetAsync(&s.ctr->n_chain, 0, offsetof(Counters, n_contigs) - offsetof(Counters, n_chain), env.stream);
  cudaMemcpyAsync(&s.ctr->n_emit, &s.ctr->n_lone, sizeof(unsigned), cudaMemcpyDeviceToDevice, env.stream);
  k_succ<<<grid_for(g.n, env), kBlock, 0, env.stream>>>(g, s);
  ++*env.launches;
  k_walk<<<grid_for(2 * g.n, env), kBlock, 0, env.stream>>>(s, t.ruler_log2, 2 * g.n + 1);
  ++*env.launches;
  Scratch sc = s;
  void* args[] = {&sc};
  cudaError_t e = coop((const void*)k_jump, env.coop_blocks, args, env);
  if (e != cudaSuccess) return e;
  DevGraph gg = g;
  k_final<<<grid_for(g.n, env), kBlock, 0, env.stream>>>(gg, s);
  ++*env.launches;
  void* args2[] = {&gg, &sc};
  e = coop((const void*)k_cycles, env.coop_blocks, args2, env);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_export_reads(const DevGraph& g, const Scratch& s, int32_t* cid, int32_t* rank, uint8_t* orient,
                                const LaunchEnv& env) {
  k_export_reads<<<grid_for(g.n, env), kBlock, 0, env.stream>>>(g, s, cid, rank, orient);
  ++*env.launches;
  return cudaGetLastError();
}

}  // namespace cg
