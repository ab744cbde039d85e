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
// sublist to the next sublist start. Each list head then walks its (short)
// list of sublists twice -- once for the length, the tail and the smallest
// read, once to hand every sublist its distance to the tail. Lists with more
// sublists than that walk follows are left to grid-synchronised pointer
// jumping, which only runs when needed; closed chains (no head) go to their
// own kernel. A read then knows, from its two oriented copies, the chain's
// length, both end reads, its position from either end, and the chain's
// smallest read id.
//
// The mask stage lists the candidates (unmasked reads with overlaps, in
// candidate order c, with cidx[v] = c) and the chain stage indexes its records
// by candidate, oriented copies u = 2c + o: they sit together instead of
// spreading over arrays of n reads. Sublist records keep read ids, which the
// canonical order compares.
#include <cuda_runtime.h>

#include "cg_internal.cuh"

namespace cg {

namespace {

constexpr long long kSpinLimit = 1ll << 22;   // barrier polls before giving up (~1 s with backoff)
constexpr int kListWalkMax = 64;              // sublists a list head follows before leaving it to jumping
constexpr int kUnresolved = -2;               // pj next field of a sublist no list walk has finished

__device__ __forceinline__ int sampled(int v, int ruler_log2) {
  unsigned h = (unsigned)v * 0x9E3779B1u;
  h ^= h >> 15;
  h *= 0x85EBCA77u;
  h ^= h >> 13;
  return (h & ((1u << ruler_log2) - 1u)) == 0u;
}

// Read m is the smallest read of a contig of q reads.
__device__ __forceinline__ void mark_head(const Scratch& s, int32_t m, int32_t q) {
  atomicOr(&s.hb[m >> 5], 1u << (m & 31));
  s.headq[m] = q;
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
      if (g.pre) {                         // x-drop form: indices into the stored reads u and v
        const int32_t p = g.pre[x], q = g.post[x];
        if (p < 0 || p > g.len[u] - 1 || q < 0 || q > g.len[v] - 1) set_error(c, DERR_GRAPH, K_VALIDATE2, x);
      } else {
        const int32_t s = g.suf[x];
        if (s < 1 || s > g.len[v] - 1) set_error(c, DERR_GRAPH, K_VALIDATE2, x);
      }
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
// no overlap are lone reads: a one-read contig when min_chain <= 1. Every
// word of the mask-stage bitmap of contig heads is written here (the lone
// reads' bits); the chain stage adds the other heads to a copy of it.
// A warp owns 256 consecutive reads per pass, eight per lane: a lane loads
// its eight row starts with 16-byte loads (a read's degree is the next start
// minus its own; the eighth read's end is the next lane's first start),
// writes its eight branch bytes as one 8-byte store, and queues the reads of
// degree 1 or 2, whose rule needs the neighbours' degrees. The whole warp
// then resolves the queue together, so that a pass waits for three dependent
// loads (row starts; col and code; the neighbours' rows) whatever the mix of
// degrees in it. The candidate and lone-read lists gather in per-warp
// shared-memory buffers and reach the global lists with one reservation per
// block at the end (a warp flushes early only when a pass would overflow its
// buffer): returning atomics on one counter, one per pass, would serialise.
#ifndef CG_MASK_MIN_BLOCKS
#define CG_MASK_MIN_BLOCKS 4                   // resident blocks per SM the registers must allow
#endif
constexpr int kMaskLane = 8;                  // reads per lane per pass
constexpr int kMaskSpan = 32 * kMaskLane;     // reads per warp per pass
constexpr int kMaskWarps = kBlock / 32;
constexpr int kMaskBuf = 256;                 // buffered list entries per warp

template <typename RP>
__device__ __forceinline__ void load_rows(const RP* p, int64_t r[kMaskLane]);
template <>
__device__ __forceinline__ void load_rows<int64_t>(const int64_t* p, int64_t r[kMaskLane]) {
#pragma unroll
  for (int k = 0; k < kMaskLane / 2; ++k) {
    const longlong2 x = __ldg(reinterpret_cast<const longlong2*>(p) + k);
    r[2 * k] = x.x;
    r[2 * k + 1] = x.y;
  }
}
template <>
__device__ __forceinline__ void load_rows<int32_t>(const int32_t* p, int64_t r[kMaskLane]) {
#pragma unroll
  for (int k = 0; k < kMaskLane / 4; ++k) {
    const int4 x = __ldg(reinterpret_cast<const int4*>(p) + k);
    r[4 * k] = x.x; r[4 * k + 1] = x.y; r[4 * k + 2] = x.z; r[4 * k + 3] = x.w;
  }
}

// Exclusive prefix of per-lane counts across the warp; the total in *tot.
__device__ __forceinline__ unsigned warp_exclusive(unsigned x, unsigned* tot, int lane) {
  unsigned inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  *tot = __shfl_sync(0xffffffffu, inc, 31);
  return inc - x;
}

// Appends n buffered entries of one warp to a global list with one atomic.
__device__ __forceinline__ void warp_flush(unsigned* counter, int32_t* list, const int32_t* buf, unsigned n,
                                           int lane) {
  unsigned base = 0;
  if (lane == 0) base = atomicAdd(counter, n);
  base = __shfl_sync(0xffffffffu, base, 0);
  for (unsigned i = lane; i < n; i += 32) list[base + i] = buf[i];
}

// Reserves n entries of a global list for one warp (one atomic); returns the first.
__device__ __forceinline__ unsigned warp_reserve(unsigned* counter, unsigned n, int lane) {
  unsigned base = 0;
  if (lane == 0) base = atomicAdd(counter, n);
  return __shfl_sync(0xffffffffu, base, 0);
}

// Candidates get their index when written out: cand[c] = v and cidx[v] = c.
__device__ __forceinline__ void flush_cands(const Scratch& s, const int32_t* buf, unsigned n, unsigned base,
                                            int lane) {
  for (unsigned i = lane; i < n; i += 32) {
    const int32_t v = buf[i];
    s.cand[base + i] = v;
    s.cidx[v] = (int32_t)(base + i);
  }
}

template <typename RP, bool kAligned>
__global__ void __launch_bounds__(kBlock, CG_MASK_MIN_BLOCKS) k_mask(DevGraph g, Scratch s) {
  pdl_enter();
  __shared__ int64_t q_row[kMaskWarps][kMaskSpan];   // queued reads: row start
  __shared__ uint16_t q_pos[kMaskWarps][kMaskSpan];  //   and position in the pass | (degree == 2) << 8
  __shared__ int32_t b_cand[kMaskWarps][kMaskBuf];   // buffered list entries
  __shared__ int32_t b_lone[kMaskWarps][kMaskBuf];
  __shared__ unsigned blk_n[2], blk_base[2];
  const RP* const rp = reinterpret_cast<const RP*>(g.row_ptr);
  Counters* c = s.ctr;
  if (threadIdx.x < 2) blk_n[threadIdx.x] = 0;       // read after the first barrier below
  unsigned long long nb = 0;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* const bc = b_cand[wib];
  int32_t* const bl = b_lone[wib];
  unsigned nc = 0, nl = 0;                           // buffered entries (warp-uniform)
  const long long stride = (long long)gridDim.x * kMaskWarps * kMaskSpan;
  // The row starts of a pass (and, on lane 31, the start after its last read).
  // They are loaded one pass ahead, so that the next pass's stream of row_ptr
  // is in flight while this pass resolves its queued reads.
  const int p0 = kMaskLane * lane;
  auto load_pass = [&](long long wb, int64_t (&r)[kMaskLane], int64_t& e31) {
    const int cnt = (int)min((long long)kMaskSpan, g.n - wb);
    const bool full = cnt == kMaskSpan;
    if (kAligned && full) {
      load_rows<RP>(rp + wb + p0, r);
    } else {
#pragma unroll
      for (int j = 0; j < kMaskLane; ++j) r[j] = p0 + j <= cnt ? (int64_t)rp[wb + p0 + j] : 0;
    }
    e31 = lane == 31 && full ? (int64_t)rp[wb + kMaskSpan] : 0;
  };
  long long wbase = ((long long)blockIdx.x * kMaskWarps + wib) * kMaskSpan;
  int64_t r[kMaskLane], e31 = 0;
  if (wbase < g.n) load_pass(wbase, r, e31);
  for (; wbase < g.n; wbase += stride) {
    // warp-uniform trip count; row_ptr holds n + 1 entries
    const int cnt = (int)min((long long)kMaskSpan, g.n - wbase);
    const bool full = cnt == kMaskSpan;
    int64_t e = __shfl_down_sync(0xffffffffu, r[0], 1);
    if (lane == 31) e = e31;
    uint32_t br[2] = {0u, 0u};
    unsigned pend = 0, two = 0, lone = 0;
#pragma unroll
    for (int j = 0; j < kMaskLane; ++j) {
      const int64_t d = (j < kMaskLane - 1 ? r[j + 1] : e) - r[j];
      if (p0 + j < cnt) {
        if (d >= 3) { br[j >> 2] |= 1u << (8 * (j & 3)); ++nb; }
        else if (d > 0) { pend |= 1u << j; two |= (d == 2 ? 1u : 0u) << j; }
        else lone |= 1u << j;
      }
    }
    if (g.min_chain > 1) lone = 0;
    int64_t rn[kMaskLane], en31 = 0;                   // the next pass's row starts, in flight from here
    if (wbase + stride < g.n) load_pass(wbase + stride, rn, en31);
    if (full) {
      *reinterpret_cast<uint2*>(s.branch + wbase + p0) = make_uint2(br[0], br[1]);
    } else {
#pragma unroll
      for (int j = 0; j < kMaskLane; ++j)
        if (p0 + j < cnt) s.branch[wbase + p0 + j] = (uint8_t)(br[j >> 2] >> (8 * (j & 3)));
    }
#pragma unroll
    for (int j = 0; j < kMaskLane; ++j)
      if ((br[j >> 2] >> (8 * (j & 3))) & 1u) s.cidx[wbase + p0 + j] = -1;
    unsigned T;                                        // queued reads of this pass
    unsigned k = warp_exclusive(__popc(pend), &T, lane);
#pragma unroll
    for (int j = 0; j < kMaskLane; ++j)
      if ((pend >> j) & 1u) {
        q_row[wib][k] = r[j];
        q_pos[wib][k] = (uint16_t)((p0 + j) | (((two >> j) & 1u) << 8));
        ++k;
      }
    // the pass's eight words of the heads bitmap: lane 4w + l holds bits 8l..8l+7 of word w
    if (g.min_chain <= 1) {                            // uniform
      unsigned x = lone << (8 * (lane & 3));
      x |= __shfl_xor_sync(0xffffffffu, x, 1);
      x |= __shfl_xor_sync(0xffffffffu, x, 2);
      if ((lane & 3) == 0 && kMaskLane * lane < cnt) s.hb_mask[(wbase >> 5) + (lane >> 2)] = x;
      unsigned L;
      unsigned kl = warp_exclusive(__popc(lone), &L, lane);
      if (nl + L > kMaskBuf) {                         // uniform: this pass would overflow the buffer
        warp_flush(&c->n_lone, s.lone, bl, nl, lane);
        nl = 0;
        __syncwarp();
      }
      kl += nl;
#pragma unroll
      for (int j = 0; j < kMaskLane; ++j)
        if ((lone >> j) & 1u) {
          const int32_t v = (int32_t)(wbase + p0 + j);
          bl[kl++] = v;
          s.headq[v] = 1;
        }
      nl += L;
    } else if (lane < kMaskSpan / 32 && 32 * lane < cnt) {
      s.hb_mask[(wbase >> 5) + lane] = 0u;
    }
    if (nc + T > kMaskBuf) {                           // uniform: the queue could overflow the buffer
      flush_cands(s, bc, nc, warp_reserve(&c->n_cand, nc, lane), lane);
      nc = 0;
    }
    __syncwarp();                                      // queue written; branch bytes ordered before the fix-ups
    for (unsigned j0 = 0; j0 < T; j0 += 32) {          // warp-uniform
      const unsigned jj = j0 + lane;
      bool cand = false;
      int32_t v = 0;
      if (jj < T) {
        const unsigned q = q_pos[wib][jj];
        const int64_t x = q_row[wib][jj];
        const bool two2 = (q >> 8) != 0;
        v = (int32_t)(wbase + (q & 255u));
        const int32_t w0 = g.col[x];
        const int32_t w1 = two2 ? g.col[x + 1] : w0;
        const int c0 = g.code[x] & 1, c1 = two2 ? (g.code[x + 1] & 1) : c0;
        const bool k0 = (int64_t)rp[w0 + 1] - (int64_t)rp[w0] < 3;
        const bool k1 = two2 && (int64_t)rp[w1 + 1] - (int64_t)rp[w1] < 3;
        // two overlaps to reads of degree <= 2, both on one end: a branch
        if (k0 && k1 && c0 == c1) {
          s.branch[v] = 1;
          s.cidx[v] = -1;
          ++nb;
        } else {
          cand = true;
        }
      }
      const unsigned cm = __ballot_sync(0xffffffffu, cand);
      if (cand) bc[nc + __popc(cm & ((1u << lane) - 1u))] = v;
      nc += __popc(cm);
    }
    __syncwarp();                                      // queue and buffers reused next pass
#pragma unroll
    for (int j = 0; j < kMaskLane; ++j) r[j] = rn[j];
    e31 = en31;
  }
  // one reservation per block for the entries the warps still hold
  __syncthreads();
  unsigned oc = 0, ol = 0;
  if (lane == 0) {
    oc = nc ? atomicAdd(&blk_n[0], nc) : 0;
    ol = nl ? atomicAdd(&blk_n[1], nl) : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    blk_base[0] = blk_n[0] ? atomicAdd(&c->n_cand, blk_n[0]) : 0;
    blk_base[1] = blk_n[1] ? atomicAdd(&c->n_lone, blk_n[1]) : 0;
  }
  __syncthreads();
  oc = blk_base[0] + __shfl_sync(0xffffffffu, oc, 0);
  ol = blk_base[1] + __shfl_sync(0xffffffffu, ol, 0);
  flush_cands(s, bc, nc, oc, lane);
  for (unsigned i = lane; i < nl; i += 32) s.lone[ol + i] = bl[i];
  for (int o = 16; o > 0; o >>= 1) nb += __shfl_down_sync(0xffffffffu, nb, o);
  if (lane == 0 && nb) atomicAdd(&c->n_branch, nb);
}

template <typename RP, bool kAligned>
void launch_mask_kernel(const DevGraph& g, const Scratch& s, const LaunchEnv& env) {
  static const int resident = resident_blocks(k_mask<RP, kAligned>);   // a persistent grid
  const long long need = (g.n + (long long)kMaskWarps * kMaskSpan - 1) / ((long long)kMaskWarps * kMaskSpan);
  const int grid = (int)std::max(1LL, std::min(need, (long long)env.num_sms * resident));
  k_mask<RP, kAligned><<<grid, kBlock, 0, env.stream>>>(g, s);
}

// Successor table of L over the candidates (unmasked reads with overlaps),
// in candidate order: succ[c] = (successor of (c,0), successor of (c,1), read
// id); the overlap (v->w) on end E_v is the way out of (v, 1-E_v) and enters
// (w, E_w), whose incoming suffix is suf(v->w). Also lists the sublist starts
// (list heads and sampled reads) and, among them, the list heads. A
// candidate has one or two overlaps: both entries' fields and their reads'
// candidate indexes (-1: a branch read) are loaded before any store. The
// start lists gather in per-warp shared-memory buffers and reach the global
// lists with one reservation per block at the end (a warp flushes early only
// when its buffer runs full); a start learns its sublist id (kept in the
// successor record's last field for (c,0)) when it is written out.
constexpr int kSuccWarps = kBlock / 32;
constexpr int kSuccStarts = 256;    // sublist starts per warp: oriented candidate | list head << 31

// Writes n buffered sublist starts of one warp to rlist[rbase..] with their
// rr records, and the list heads among them to hlist[hbase..].
__device__ __forceinline__ void put_starts(const Scratch& s, const uint32_t* buf, unsigned n, unsigned rbase,
                                           unsigned hbase, int lane) {
  const unsigned lt = (1u << lane) - 1u;
  unsigned h = 0;
  for (unsigned i0 = 0; i0 < n; i0 += 32) {          // warp-uniform
    const unsigned i = i0 + lane;
    bool head = false;
    if (i < n) {
      const uint32_t e = buf[i];
      const int32_t u = (int32_t)(e & 0x7fffffffu);
      head = (e >> 31) != 0;
      s.rlist[rbase + i] = u;
      // a sampled read's two copies are consecutive starts, (c,0) first: its
      // record keeps the first id, for the walks that end there
      if ((u & 1) == 0) s.succ[u >> 1].w = (int32_t)(rbase + i);
    }
    const unsigned hm = __ballot_sync(0xffffffffu, head);
    if (head) s.hlist[hbase + h + __popc(hm & lt)] = (int32_t)(rbase + i);
    h += __popc(hm);
  }
}

__global__ void __launch_bounds__(kBlock) k_succ(DevGraph g, Scratch s, int ruler_log2) {
  pdl_enter();
  __shared__ uint32_t b_start[kSuccWarps][kSuccStarts];
  __shared__ unsigned blk_n[2], blk_base[2];
  Counters* c = s.ctr;
  const long long N = *(volatile unsigned*)&c->n_cand;
  if (threadIdx.x < 2) blk_n[threadIdx.x] = 0;       // read after the first barrier below
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t* const bs = b_start[wib];
  unsigned ns = 0, nh = 0;                           // buffered starts (warp-uniform), and the heads among them
  // the chain stage's heads bitmap starts from the mask stage's words (lone reads)
  for (long long w = grid_tid(); w < (g.n + 31) / 32; w += grid_threads()) s.hb[w] = s.hb_mask[w];
  const long long Nw = (N + 31) / 32 * 32;           // whole warps iterate together
  for (long long ci = grid_tid(); ci < Nw; ci += grid_threads()) {
    int s0 = -1, s1 = -1;
    bool r0 = false, r1 = false;
    if (ci < N) {
      const int32_t v = s.cand[ci];
      const int64_t a = rowp(g, v);
      const bool two = rowp(g, v + 1) - a == 2;
      const int32_t w0 = g.col[a], w1 = two ? g.col[a + 1] : 0;
      const int cd0 = g.code[a], cd1 = two ? g.code[a + 1] : 0;
      int32_t q0, q1 = 0, p0 = 0, p1 = 0;
      if (g.pre) {
        q0 = g.post[a]; p0 = g.pre[a];
        if (two) { q1 = g.post[a + 1]; p1 = g.pre[a + 1]; }
      } else {
        q0 = g.suf[a];
        if (two) q1 = g.suf[a + 1];
      }
      // a neighbour's candidate index, -1 for a branch read; an entry without its
      // mirror (a graph loaded unvalidated) may reach a read whose index the mask
      // stage never wrote: an out-of-range value counts as a branch read, so the
      // successor and suffix stores below stay inside their arrays
      int32_t c0 = s.cidx[w0], c1 = two ? s.cidx[w1] : -1;
      if ((uint32_t)c0 >= (uint32_t)N) c0 = -1;
      if ((uint32_t)c1 >= (uint32_t)N) c1 = -1;
      const int32_t u0 = 2 * (int32_t)ci;
      if (c0 >= 0) {                     // (v, 1-ev) leaves through end ev
        const int ev = cd0 & 1, to = 2 * c0 + (cd0 >> 1);
        if (ev == 1) s0 = to; else s1 = to;
        s.sufin[to] = q0;
        if (g.pre) s.preout[u0 + 1 - ev] = p0;
      }
      if (c1 >= 0) {
        const int ev = cd1 & 1, to = 2 * c1 + (cd1 >> 1);
        if (ev == 1) s0 = to; else s1 = to;
        s.sufin[to] = q1;
        if (g.pre) s.preout[u0 + 1 - ev] = p1;
      }
      s.succ[ci] = make_int4(s0, s1, v, 0);
      if (s0 < 0 && s1 < 0) {            // every overlap leads to a branch read: spelled alone, or in no contig
        const bool lone = g.min_chain <= 1;
        s.prd[ci] = make_int4(lone ? v : -1, lone ? 0 : -1, lone ? g.len[v] : 0, lone ? 0 : 255);
        if (g.pre) s.pfirst[ci] = 0;   // its contig head is marked by k_final
      } else {
        reinterpret_cast<int4*>(s.rr)[ci] = make_int4(-1, 0, -1, 0);   // not yet reached by a sublist walk
        const bool smp = sampled(v, ruler_log2) != 0;
        r0 = s1 < 0 || smp;              // (c,0) has no predecessor when (c,1) has no successor
        r1 = s0 < 0 || smp;
      }
    }
    const bool h0 = r0 && s1 < 0, h1 = r1 && s0 < 0;
    const unsigned m0 = __ballot_sync(0xffffffffu, r0), m1 = __ballot_sync(0xffffffffu, r1);
    const unsigned slot = ns + __popc(m0 & lt) + __popc(m1 & lt);
    if (r0) bs[slot] = (uint32_t)(2 * ci) | (h0 ? 0x80000000u : 0u);
    if (r1) bs[slot + (r0 ? 1 : 0)] = (uint32_t)(2 * ci + 1) | (h1 ? 0x80000000u : 0u);
    ns += __popc(m0) + __popc(m1);
    nh += __popc(__ballot_sync(0xffffffffu, h0)) + __popc(__ballot_sync(0xffffffffu, h1));
    __syncwarp();
    if (ns > kSuccStarts - 64) {         // an iteration adds at most 64 starts
      unsigned rb = 0, hb = 0;
      if (lane == 0) { rb = atomicAdd(&c->n_rulers, ns); hb = nh ? atomicAdd(&c->n_hlist, nh) : 0u; }
      put_starts(s, bs, ns, __shfl_sync(0xffffffffu, rb, 0), __shfl_sync(0xffffffffu, hb, 0), lane);
      ns = 0;
      nh = 0;
    }
    __syncwarp();
  }
  // one reservation per block for the starts the warps still hold
  __syncthreads();
  unsigned o[2] = {0, 0};
  if (lane == 0) {
    o[0] = ns ? atomicAdd(&blk_n[0], ns) : 0u;
    o[1] = nh ? atomicAdd(&blk_n[1], nh) : 0u;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    blk_base[0] = blk_n[0] ? atomicAdd(&c->n_rulers, blk_n[0]) : 0u;
    blk_base[1] = blk_n[1] ? atomicAdd(&c->n_hlist, blk_n[1]) : 0u;
  }
  __syncthreads();
  for (int f = 0; f < 2; ++f) o[f] = blk_base[f] + __shfl_sync(0xffffffffu, o[f], 0);
  put_starts(s, bs, ns, o[0], o[1], lane);
}

// One thread per sublist start: walk to the next start or the list end. The
// sublist's record keeps read ids: its smallest read and its last oriented
// read as 2v + o.
__global__ void k_walk(Scratch s, int ruler_log2, int64_t limit) {
  pdl_enter();
  Counters* c = s.ctr;
  const long long R = *(volatile unsigned*)&c->n_rulers;
  for (long long r = grid_tid(); r < R; r += grid_threads()) {
    const int32_t x = s.rlist[r];
    const int4 sv = s.succ[x >> 1];
    int32_t y = x, z = (x & 1) ? sv.y : sv.x, vy = sv.z, mn = sv.z, next = -1;
    int32_t cnt = 0;
    for (;;) {
      s.rr[y] = make_int2((int32_t)r, cnt);
      ++cnt;
      mn = min(mn, vy);
      if (z < 0) break;
      const int4 sz = s.succ[z >> 1];
      if (sampled(sz.z, ruler_log2)) { next = sz.w + (z & 1); break; }   // the sublist z starts
      y = z;
      vy = sz.z;
      z = (z & 1) ? sz.y : sz.x;
      if (cnt > limit) { set_error(s.derr, DERR_KERNEL, K_WALK, y); break; }
    }
    s.rec[r] = make_int4(next, cnt, mn, 2 * vy + (y & 1));
    s.pj[0][r].x = kUnresolved;
  }
}

// One thread per list head, one walk over the list of sublists: each sublist
// gets the reads before it and its list's head (pj[0][r] = (kViaHead, reads
// before r, head, 0)), and the list's head the totals (pj[1][head] = (total
// reads, smallest read, last oriented read, 0)); the finals turn the pair into
// the reads from r to the tail. Longer lists are left to pointer jumping,
// which rewrites every record in the direct form (-1, reads to the tail,
// smallest read, last read) into both buffers, so the finals read that form
// whenever it ran.
constexpr int kViaHead = -3;                  // pj x-field of a sublist the list walk resolved

__global__ void k_listwalk(Scratch s) {
  pdl_enter();
  Counters* c = s.ctr;
  const long long H = *(volatile unsigned*)&c->n_hlist;
  for (long long h = grid_tid(); h < H; h += grid_threads()) {
    const int32_t r0 = s.hlist[h];
    int32_t r = r0, mn = 0x7fffffff, steps = 0, tail = -1;
    long long total = 0;
    bool ok = true;
    for (;;) {
      const int4 rc = s.rec[r];
      s.pj[0][r] = make_int4(kViaHead, (int32_t)min(total, 0x7fffffffll), r0, 0);
      total += rc.y;
      mn = min(mn, rc.z);
      if (rc.x < 0) {
        tail = rc.w;                     // the list's last oriented read
        break;
      }
      if (++steps >= kListWalkMax) { ok = false; break; }
      r = rc.x;
    }
    if (!ok || total > 0x7fffffffll) {
      atomicOr(&c->need_jump, 1u);
      continue;
    }
    s.pj[1][r0] = make_int4((int32_t)total, mn, tail, 0);
  }
}

// Pointer jumping over all sublists (grid-synchronised rounds), only when a
// list walk gave up (very long chains). After it, for a sublist on an open
// list: acc = oriented reads from its start to the list tail, mn = smallest
// read id over that span, tail = the list's last oriented read. Sublists on
// directed cycles keep next >= 0.
__global__ void k_jump(Scratch s) {
  pdl_enter();
  Counters* c = s.ctr;
  if (*(volatile unsigned*)&c->need_jump == 0) return;   // the same for every block: written by the kernel before
  unsigned R = *(volatile unsigned*)&c->n_rulers;
  for (long long i = grid_tid(); i < R; i += grid_threads()) {
    const int4 rc = s.rec[i];
    s.pj[0][i] = make_int4(rc.x, rc.y, rc.z, rc.w);
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
      const int4 a = s.pj[cur][i];
      if (a.x >= 0) {
        const int4 b = s.pj[cur][a.x];
        const long long acc = (long long)a.y + b.y;
        s.pj[nxt][i] = make_int4(b.x, acc > 0x7fffffffll ? 0x7fffffff : (int32_t)acc,   // saturates on cycles
                                 min(a.z, b.z), b.w);
        active |= (b.x >= 0);
      } else {
        s.pj[nxt][i] = make_int4(-1, a.y, a.z, a.w);
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

// x-drop form (Sec. 4.4): read v (candidate ci), walked as oriented
// candidate u at rank rk of a contig of q reads, contributes
// l_v[post(e_in) : pre(e_out)] with alpha (its first base in walk direction)
// for the first read and beta (its last) for the last one; a piece whose end
// comes before its start is empty. Returns the piece's length; its first
// stored base goes to pfirst.
__device__ __forceinline__ int32_t set_piece(const DevGraph& g, const Scratch& s, int32_t v, int32_t ci, int32_t u,
                                             int32_t rk, int32_t q) {
  const int o = u & 1;
  const int32_t L = g.len[v];
  const int32_t first = rk == 0 ? (o == 0 ? 0 : L - 1) : s.sufin[u];
  const int32_t last = rk == q - 1 ? (o == 0 ? L - 1 : 0) : s.preout[u];
  const int32_t cnt = o == 0 ? last - first + 1 : first - last + 1;
  s.pfirst[ci] = first;
  return cnt > 0 ? cnt : 0;
}

// The bases a chain read adds: the first read whole, each later one the
// suffix of the overlap it is entered through (or, in the x-drop form, its
// piece).
__device__ __forceinline__ int32_t piece_len(const DevGraph& g, const Scratch& s, int32_t v, int32_t ci, int32_t u,
                                             int32_t rk, int32_t q) {
  if (g.pre) return set_piece(g, s, v, ci, u, rk, q);
  return rk == 0 ? g.len[v] : s.sufin[u];
}

// Per chain candidate: combine its two oriented copies. head(list of (c,0))
// is the reverse of tail(list of (c,1)). The contig starts at the
// smaller-id end read, so (c,0) is the walk orientation when that end heads
// the list of (c,0). Candidates of closed chains (no list head reached them)
// are listed for the cycle kernel; candidates cut off by branch reads got
// their record from the successor kernel. A thread takes two candidates at a
// time and issues each level of their dependent loads (successor records;
// rank records; list records; length and entering overlap) together, before
// any store.
constexpr int kFinalItems = 2;

__global__ void k_final(DevGraph g, Scratch s) {
  pdl_enter();
  Counters* c = s.ctr;
  const int fb = (int)*(volatile unsigned*)&c->final_buf;
  const long long N = *(volatile unsigned*)&c->n_cand;
  const long long n = (N + 31) & ~31ll;
  const int4* pj = s.pj[fb];
  const long long T = grid_threads();
  for (long long k0 = grid_tid(); k0 < n; k0 += kFinalItems * T) {   // warp-uniform trip count
    bool in[kFinalItems];
    int32_t v[kFinalItems];
    int4 r01[kFinalItems], p0[kFinalItems], p1[kFinalItems];
#pragma unroll
    for (int j = 0; j < kFinalItems; ++j) {
      const int4 sv = k0 + j * T < N ? s.succ[k0 + j * T] : make_int4(-1, -1, 0, 0);
      in[j] = sv.x >= 0 || sv.y >= 0;      // a chain candidate
      v[j] = sv.z;
    }
#pragma unroll
    for (int j = 0; j < kFinalItems; ++j)   // (sublist, position) of (c,0) and (c,1)
      r01[j] = in[j] ? reinterpret_cast<const int4*>(s.rr)[k0 + j * T] : make_int4(-1, 0, -1, 0);
#pragma unroll
    for (int j = 0; j < kFinalItems; ++j) {
      p0[j] = r01[j].x >= 0 ? pj[r01[j].x] : make_int4(0, 0, 0, 0);
      p1[j] = r01[j].z >= 0 ? pj[r01[j].z] : make_int4(0, 0, 0, 0);
    }
    // a sublist resolved by the list walk: its list's totals sit at the head
    // (in the other buffer), and the reads from it to the tail are the total
    // less the reads before it
    int4 t0[kFinalItems], t1[kFinalItems];
#pragma unroll
    for (int j = 0; j < kFinalItems; ++j) {
      t0[j] = p0[j].x == kViaHead ? s.pj[fb ^ 1][p0[j].z] : make_int4(0, 0, 0, 0);
      t1[j] = p1[j].x == kViaHead ? s.pj[fb ^ 1][p1[j].z] : make_int4(0, 0, 0, 0);
    }
#pragma unroll
    for (int j = 0; j < kFinalItems; ++j) {
      if (p0[j].x == kViaHead) p0[j] = make_int4(-1, t0[j].x - p0[j].y, t0[j].y, t0[j].z);
      if (p1[j].x == kViaHead) p1[j] = make_int4(-1, t1[j].x - p1[j].y, t1[j].y, t1[j].z);
    }
    bool cyc[kFinalItems], ok[kFinalItems];
    int32_t m[kFinalItems], q[kFinalItems], rk[kFinalItems], o[kFinalItems], L[kFinalItems], sin[kFinalItems],
        pout[kFinalItems];
#pragma unroll
    for (int j = 0; j < kFinalItems; ++j) {
      cyc[j] = in[j] && (r01[j].x < 0 || r01[j].z < 0 || p0[j].x != -1 || p1[j].x != -1);
      ok[j] = in[j] && !cyc[j];
      const int32_t d0 = p0[j].y - r01[j].y - 1;
      const int32_t d1 = p1[j].y - r01[j].w - 1;
      const int32_t h0 = p1[j].w >> 1, h1 = p0[j].w >> 1;   // first read of the list of (c,0) / (c,1)
      // the smallest read of the chain: (c,0)'s list from c's sublist on and
      // (c,1)'s list (the same reads, reversed) from c's sublist on cover it
      m[j] = min(p0[j].z, p1[j].z);
      q[j] = d0 + d1 + 1;
      o[j] = h0 < h1 ? 0 : 1;
      rk[j] = o[j] == 0 ? d1 : d0;
      if (ok[j] && (m[j] < 0 || h0 == h1)) set_error(s.derr, DERR_KERNEL, K_FINAL, v[j]);
      ok[j] = ok[j] && q[j] >= g.min_chain;
    }
    // the piece's inputs: the read's length and its walk copy's overlaps
#pragma unroll
    for (int j = 0; j < kFinalItems; ++j) {
      const long long u = 2 * (k0 + j * T) + o[j];
      L[j] = ok[j] ? g.len[v[j]] : 0;
      sin[j] = ok[j] && rk[j] > 0 ? s.sufin[u] : 0;
      pout[j] = ok[j] && g.pre && rk[j] < q[j] - 1 ? s.preout[u] : 0;
    }
#pragma unroll
    for (int j = 0; j < kFinalItems; ++j) {
      const long long ci = k0 + j * T;
      if (ok[j]) {
        int32_t len;
        if (g.pre) {   // x-drop form: l_v[post(e_in) : pre(e_out)], alpha / beta at the contig's ends
          const int32_t first = rk[j] == 0 ? (o[j] == 0 ? 0 : L[j] - 1) : sin[j];
          const int32_t last = rk[j] == q[j] - 1 ? (o[j] == 0 ? L[j] - 1 : 0) : pout[j];
          const int32_t cnt = o[j] == 0 ? last - first + 1 : first - last + 1;
          s.pfirst[ci] = first;
          len = cnt > 0 ? cnt : 0;
        } else {       // the first read whole, each later one the suffix it is entered through
          len = rk[j] == 0 ? L[j] : sin[j];
        }
        s.prd[ci] = make_int4(m[j], rk[j], len, o[j]);
        if (v[j] == m[j]) {
          mark_head(s, m[j], q[j]);
          atomicAdd(&c->n_heads, 1u);
        }
      } else if (in[j] && !cyc[j]) {
        s.prd[ci] = make_int4(-1, -1, 0, 255);
      } else if (!in[j] && ci < N && g.min_chain <= 1) {   // cut off by branch reads: its own contig
        mark_head(s, v[j], 1);
        atomicAdd(&c->n_heads, 1u);
      }
      const unsigned slot = warp_append(&c->n_cycle_reads, cyc[j]);
      if (cyc[j]) s.cyc[slot] = (int32_t)ci;
    }
  }
}

// Closed chains (rare). Over their oriented candidates: pointer jumping for
// the smallest oriented read 2v + o of each directed cycle, carried with the
// oriented candidate that holds it (the copy holding (m,0) is the walk, m the
// smallest read), then cut the walk before (m,0) and rank by pointer jumping
// again.
__global__ void k_cycles(DevGraph g, Scratch s) {
  pdl_enter();
  Counters* c = s.ctr;
  unsigned C = *(volatile unsigned*)&c->n_cycle_reads;
  if (C == 0) return;
  long long N = 2ll * C;
  for (long long i = grid_tid(); i < N; i += grid_threads()) {
    const int32_t ci = s.cyc[i >> 1], u = 2 * ci + (int)(i & 1);
    const int4 sv = s.succ[ci];
    const int32_t z = (u & 1) ? sv.y : sv.x;
    if (z < 0) set_error(s.derr, DERR_KERNEL, K_CYCLE, u);
    s.c_ptr[0][u] = z;
    s.c_val[0][u] = ((long long)(2 * sv.z + (u & 1)) << 32) | (unsigned)u;
  }
  int rounds = 1;
  while ((1ll << rounds) < N + 1 && rounds < 31) ++rounds;
  ++rounds;
  int cur = 0;
  if (!grid_sync(c, s.derr)) return;
  for (int r = 0; r < rounds; ++r) {
    int nxt = cur ^ 1;
    for (long long i = grid_tid(); i < N; i += grid_threads()) {
      const int32_t u = 2 * s.cyc[i >> 1] + (int)(i & 1);
      const int32_t p = s.c_ptr[cur][u];
      if (p < 0) continue;
      s.c_val[nxt][u] = min(s.c_val[cur][u], s.c_val[cur][p]);
      s.c_ptr[nxt][u] = s.c_ptr[cur][p];
    }
    cur = nxt;
    if (!grid_sync(c, s.derr)) return;
  }
  // cut: on the walk copy, the oriented candidate before the start has no successor
  for (long long i = grid_tid(); i < N; i += grid_threads()) {
    const int32_t ci = s.cyc[i >> 1], u = 2 * ci + (int)(i & 1);
    const int32_t head = (int32_t)(s.c_val[cur][u] & 0xffffffffll);   // the oriented candidate holding the smallest read
    s.c_head[u] = head;
    if ((head & 1) == 0) {
      const int4 sv = s.succ[ci];
      const int32_t z = (u & 1) ? sv.y : sv.x;
      const int32_t p = (z == head) ? -1 : z;
      s.c_ptr[0][u] = p;
      s.c_val[0][u] = p < 0 ? 0 : 1;
    }
  }
  cur = 0;
  if (!grid_sync(c, s.derr)) return;
  for (int r = 0; r < rounds; ++r) {
    int nxt = cur ^ 1;
    for (long long i = grid_tid(); i < N; i += grid_threads()) {
      const int32_t u = 2 * s.cyc[i >> 1] + (int)(i & 1);
      if (s.c_head[u] & 1) continue;
      const int32_t p = s.c_ptr[cur][u];
      if (p >= 0) {
        s.c_val[nxt][u] = s.c_val[cur][u] + s.c_val[cur][p];
        s.c_ptr[nxt][u] = s.c_ptr[cur][p];
      } else {
        s.c_val[nxt][u] = s.c_val[cur][u];
        s.c_ptr[nxt][u] = -1;
      }
    }
    cur = nxt;
    if (!grid_sync(c, s.derr)) return;
  }
  for (long long i = grid_tid(); i < N; i += grid_threads()) {
    const int32_t ci = s.cyc[i >> 1];
    const int32_t u = 2 * ci + (int)(i & 1);
    const int32_t head = s.c_head[u];
    if (head & 1) continue;
    const int32_t L = (int32_t)s.c_val[cur][head] + 1;      // distance from the start to the cut, plus one
    const int32_t rk = L - 1 - (int32_t)s.c_val[cur][u];
    const int32_t m = s.cand[head >> 1];
    const int32_t v = s.cand[ci];
    if (L >= g.min_chain) {
      s.prd[ci] = make_int4(m, rk, piece_len(g, s, v, ci, u, rk, L), u & 1);
      if (rk == 0) {
        mark_head(s, m, L);
        atomicAdd(&c->n_heads, 1u);
      }
    } else {
      s.prd[ci] = make_int4(-1, -1, 0, 255);
    }
    if (rk == 0) atomicAdd(&c->n_cycles, 1u);
  }
}

// Per-read chain outputs: first every read's default (a lone read, when
// spelled, is its own one-read contig), then every candidate's record.
__global__ void k_export_fill(DevGraph g, int32_t* cid, int32_t* rank, uint8_t* orient) {
  pdl_enter();
  for (long long v = grid_tid(); v < g.n; v += grid_threads()) {
    const bool lone = rowp(g, v + 1) == rowp(g, v) && g.min_chain <= 1;
    if (cid) cid[v] = lone ? (int32_t)v : -1;
    if (rank) rank[v] = lone ? 0 : -1;
    if (orient) orient[v] = lone ? 0 : 255;
  }
}

__global__ void k_export_cands(Scratch s, int32_t* cid, int32_t* rank, uint8_t* orient) {
  pdl_enter();
  const long long N = *(volatile unsigned*)&s.ctr->n_cand;
  for (long long ci = grid_tid(); ci < N; ci += grid_threads()) {
    const int32_t v = s.cand[ci];
    const int4 p = s.prd[ci];
    if (cid) cid[v] = p.x;
    if (rank) rank[v] = p.y;
    if (orient) orient[v] = (uint8_t)p.w;
  }
}

__global__ void k_sum_len(DevGraph g, unsigned long long* out) {
  unsigned long long acc = 0;
  for (long long v = grid_tid(); v < g.n; v += grid_threads()) acc += (unsigned long long)g.len[v];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// Cooperative launch (all blocks co-resident, as the grid barrier needs);
// expressed as a launch attribute so that stream capture can record it.
// A cooperative launch (every block resident at once, for the grid barrier).
// Directly after another kernel of the stage it also carries programmatic
// dependent launch, like launch_k: no kernel signals its dependents early, so
// the grid is launched only once every block of the kernel before it has
// exited (the SMs are free for all of its blocks), and each block waits for
// that kernel's completion before it touches memory.
cudaError_t coop(const void* fn, int blocks, void** args, const LaunchEnv& env, bool chained) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = env.stream;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained && env.pdl && !(env.marks && env.marks->on) ? 2 : 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace

int coop_blocks_for_grid_kernels(int num_sms) {
  int a = 0, b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_jump, kBlock, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cycles, kBlock, 0);
  int per = a < b ? a : b;
  if (per > 2) per = 2;
  if (per < 1) per = 1;
  return per * num_sms;
}

cudaError_t launch_validate(const DevGraph& g, DevError* derr, const LaunchEnv& env) {
  k_validate_reads<<<grid_for(g.n, env), kBlock, 0, env.stream>>>(g, derr);
  mark(env, "k_validate_reads");
  k_validate_entries<<<grid_for(g.n, env), kBlock, 0, env.stream>>>(g, derr);
  mark(env, "k_validate_entries");
  return cudaGetLastError();
}

cudaError_t launch_sum_len(const DevGraph& g, unsigned long long* out, const LaunchEnv& env) {
  k_sum_len<<<grid_for(g.n, env), kBlock, 0, env.stream>>>(g, out);
  mark(env, "k_sum_len");
  return cudaGetLastError();
}

cudaError_t launch_mask(const DevGraph& g, const Scratch& s, const LaunchEnv& env) {
  cudaMemsetAsync(&s.ctr->n_branch, 0, sizeof(Counters) - offsetof(Counters, n_branch), env.stream);
  const bool al = (reinterpret_cast<uintptr_t>(g.row_ptr) & 15) == 0;   // 16-byte row_ptr loads
  if (g.rp64) {
    if (al) launch_mask_kernel<int64_t, true>(g, s, env);
    else launch_mask_kernel<int64_t, false>(g, s, env);
  } else {
    if (al) launch_mask_kernel<int32_t, true>(g, s, env);
    else launch_mask_kernel<int32_t, false>(g, s, env);
  }
  mark(env, "k_mask");
  return cudaGetLastError();
}

cudaError_t launch_chains(const DevGraph& g, const Scratch& s, const Tuning& t, const LaunchEnv& env) {
  // restart the chain-stage counters; the head bitmap restarts from the mask
  // stage's words (lone reads; k_succ copies them) and gains the chain heads
  cudaMemsetAsync(&s.ctr->n_rulers, 0, offsetof(Counters, n_contigs) - offsetof(Counters, n_rulers), env.stream);
  static const int succ_resident = resident_blocks(k_succ);   // persistent grids
  static const int final_resident = resident_blocks(k_final);
  // a persistent grid, but no more blocks than the reads can use (a small
  // graph's launches would otherwise spend their time starting idle blocks)
  auto cap = [&](long long resident_grid, long long items_per_block) {
    const long long need = (g.n + items_per_block - 1) / items_per_block;
    return (int)std::max(1LL, std::min(resident_grid, need));
  };
  k_succ<<<cap((long long)env.num_sms * succ_resident, kBlock), kBlock, 0, env.stream>>>(g, s, t.ruler_log2);
  mark(env, "k_succ");
  cudaError_t e = launch_k(k_walk, grid_for(2 * g.n, env), env, true, s, t.ruler_log2, (int64_t)(2 * g.n + 1));
  if (e != cudaSuccess) return e;
  mark(env, "k_walk");
  e = launch_k(k_listwalk, grid_for(2 * g.n, env), env, true, s);
  if (e != cudaSuccess) return e;
  mark(env, "k_listwalk");
  Scratch sc = s;
  void* args[] = {&sc};
  const int coop_grid = cap(env.coop_blocks, kBlock / 2);   // up to 2 rulers or candidates per read
  e = coop((const void*)k_jump, coop_grid, args, env, true);
  if (e != cudaSuccess) return e;
  mark(env, "k_jump");
  DevGraph gg = g;
  e = launch_k(k_final, cap((long long)env.num_sms * final_resident, (long long)kBlock * kFinalItems), env, true, gg,
               s);
  if (e != cudaSuccess) return e;
  mark(env, "k_final");
  void* args2[] = {&gg, &sc};
  e = coop((const void*)k_cycles, coop_grid, args2, env, true);
  if (e != cudaSuccess) return e;
  mark(env, "k_cycles");
  return cudaGetLastError();
}

cudaError_t launch_export_reads(const DevGraph& g, const Scratch& s, int32_t* cid, int32_t* rank, uint8_t* orient,
                                const LaunchEnv& env) {
  k_export_fill<<<grid_for(g.n, env), kBlock, 0, env.stream>>>(g, cid, rank, orient);
  mark(env, "k_export_fill");
  cudaError_t e = launch_k(k_export_cands, grid_for(g.n, env), env, true, s, cid, rank, orient);
  if (e != cudaSuccess) return e;
  mark(env, "k_export_cands");
  return cudaGetLastError();
}

}  // namespace cg
