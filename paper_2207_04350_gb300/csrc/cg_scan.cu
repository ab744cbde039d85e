// cg_scan.cu - output layout of the contigs (sm_103a): the single-GPU form of
// the contig-size estimate, the redistribution by contig and the offsets of
// the concatenation (Alg. 2, Sec. 4.2-4.4).
//
//   1. scan over the words of the heads bitmap (bit m set when read m is the
//      smallest read of a contig) of their heads and those heads' read
//      counts: the contig index of every head, listing contigs by smallest
//      read id, and every contig's first walk position; the store step lays
//      the read counts out in contig order;
//   2. scatter every spelled read to walk position first(contig) + rank: the
//      on-device compaction that replaces the induced-subgraph exchange;
//   3. scan over walk positions of the bases each read adds: the output
//      offset of every piece, the contig offsets and the map from output
//      tiles to the piece holding each tile's first byte.
//
// For one part of a contig partition (cg_emit_part, Sec. 4.3) step 2 gives
// the reads of other parts' contigs empty pieces, so step 3 lays out that
// part's contigs alone, back to back.
//
// The scans are single-pass decoupled look-back scans: tiles take tickets in
// order, publish their aggregate, then look back over predecessors with one
// warp (32 descriptors at a time) until an inclusive prefix is found. The
// wait on a predecessor is bounded; on timeout the kernel records
// DERR_TIMEOUT and stops.
#include <cuda_runtime.h>

#include <algorithm>

#include "cg_internal.cuh"
#include "cg_lookback.cuh"

namespace cg {

namespace {

// ---- scan 1: contig index and first walk position of every head ----
// The value of bitmap word w packs the contigs headed in it (their count,
// above bit kHeadShift) and their reads (below): both stay under 2^30, so
// one scan gives every head its contig index and its contig's first walk
// position at once.
constexpr int kHeadShift = 31;
constexpr unsigned long long kHeadLow = (1ull << kHeadShift) - 1;

struct HeadWordLoad {
  const unsigned* hb;
  const int32_t* headq;
  // the word's bits and the read count of its first head
  using Item = int2;
  __device__ int2 fetch(long long w) const {
    const unsigned bits = hb[w];
    return make_int2((int)bits, bits ? headq[32 * w + __ffs(bits) - 1] : 0);
  }
  __device__ unsigned long long value(long long w, const int2& it) const {
    unsigned bits = (unsigned)it.x;
    const unsigned long long heads = (unsigned long long)__popc(bits);
    unsigned long long reads = (unsigned)it.y;
    if (bits) bits &= bits - 1;
    while (bits) {                     // a second head in one word: rare
      reads += (unsigned)headq[32 * w + __ffs(bits) - 1];
      bits &= bits - 1;
    }
    return (heads << kHeadShift) | reads;
  }
};
struct HeadWordStore {
  unsigned* wp;
  const int32_t* headq;
  int32_t* qd;
  unsigned long long* cbase;
  int64_t* contig_off;
  int64_t* user_off;           // the caller's contig offsets, written by the piece scan (or nullptr)
  long long user_cap;
  Counters* c;
  __device__ void item(long long w, unsigned long long e, const int2& it) const {
    unsigned k = (unsigned)(e >> kHeadShift);
    wp[w] = k;
    unsigned bits = (unsigned)it.x;
    if (!bits) return;
    unsigned long long r = e & kHeadLow;
    int32_t q = it.y;
    for (;;) {                         // contigs in order of their smallest read
      qd[k] = q;
      cbase[k] = r;
      r += (unsigned)q;
      ++k;
      bits &= bits - 1;
      if (!bits) break;
      q = headq[32 * w + __ffs(bits) - 1];
    }
  }
  __device__ void last(long long, unsigned long long total) const {
    const unsigned C = (unsigned)(total >> kHeadShift);
    c->n_contigs = C;
    cbase[C] = total & kHeadLow;
    c->n_walk = (unsigned)(total & kHeadLow);
    if (C == 0) {                      // no contigs: the piece scan has nothing to scan
      contig_off[0] = 0;
      if (user_off && user_cap >= 1) user_off[0] = 0;
      c->total_bases = 0;
      c->n_tiles = 0;
    }
  }
};

// ---- scan 3: piece offsets over walk positions ----
struct PieceLoad {
  const int32_t* wlen;
  const int32_t* wfirst;
  // the piece's length and the contig it starts, or -1
  using Item = int2;
  __device__ int2 fetch(long long j) const { return make_int2(wlen[j], wfirst[j]); }
  __device__ unsigned long long value(long long, const int2& it) const { return (unsigned long long)(unsigned)it.x; }
};
struct PieceStore {
  int64_t* out_off;
  int64_t* contig_off;
  int32_t* tile_seg;
  long long tiles_cap;
  long long tile_bytes;
  Counters* c;
  DevError* derr;
  // The caller's contig offsets, when the offsets are spelled for a caller
  // buffer in the same replayed stage: written here instead of by a copy kernel
  // afterwards, and only when all n_contigs + 1 fit (else a capacity error).
  int64_t* user_off;
  long long user_cap;
  __device__ bool user_fits() const {
    return user_off && (long long)*(const volatile unsigned*)&c->n_contigs + 1 <= user_cap;
  }
  __device__ void item(long long j, unsigned long long e, const int2& it) const {
    long long o = (long long)e, L = it.x;
    out_off[j] = o;
    if (it.y >= 0) {
      contig_off[it.y] = o;
      if (user_fits()) user_off[it.y] = o;
    }
    // tile_bytes is a power of two: the first tile starting at or after o, and after o + L
    const int sh = __ffsll(tile_bytes) - 1;
    long long t0 = (o + tile_bytes - 1) >> sh, t1 = (o + L + tile_bytes - 1) >> sh;
    for (long long t = t0; t < t1; ++t) {
      if (t < tiles_cap) tile_seg[t] = (int32_t)j;
      else set_error(derr, DERR_KERNEL, K_SCAN_OFFSETS, t);
    }
  }
  __device__ void last(long long count, unsigned long long total) const {
    out_off[count] = (long long)total;
    contig_off[c->n_contigs] = (long long)total;
    if (user_off) {
      if (user_fits()) user_off[c->n_contigs] = (long long)total;
      else set_error(derr, DERR_CAPACITY, K_CONTIG_OFF, (long long)c->n_contigs + 1);
    }
    c->total_bases = (long long)total;
    long long nt = ((long long)total + tile_bytes - 1) / tile_bytes;
    c->n_tiles = (unsigned)nt;
    if (nt <= tiles_cap) tile_seg[nt] = (int32_t)(count - 1);
    else set_error(derr, DERR_KERNEL, K_SCAN_OFFSETS, nt);
  }
};

// Every spelled read goes to walk position first(contig) + rank, with the
// stored-base address of its piece (for one part's layout, an empty piece
// when its contig belongs to another part): forward reads add stored bases
// [len-contrib, len), reverse-complement reads the complement of stored
// bases contrib-1 down to 0. The spelled reads are the lone reads of the mask
// stage (each its own contig, whole and forward) and the candidates with a
// contig in their record (chains long enough, and reads cut off by branch
// reads when those are spelled alone). A thread takes two reads at a time and
// issues each level of their dependent loads together, before any store.
constexpr int kScatterItems = 2;

__global__ void k_scatter(DevGraph g, Scratch s) {
  pdl_enter();
  Counters* c = s.ctr;
  const long long L1 = *(volatile unsigned*)&c->n_lone, NC = *(volatile unsigned*)&c->n_cand;
  const long long W = *(volatile unsigned*)&c->n_walk;
  const long long total = L1 + NC;
  const long long T = grid_threads();
  for (long long k0 = grid_tid(); k0 < total; k0 += kScatterItems * T) {
    long long k[kScatterItems];
    int32_t v[kScatterItems];
    int4 p[kScatterItems];
    bool ok[kScatterItems];
#pragma unroll
    for (int j = 0; j < kScatterItems; ++j) {
      k[j] = k0 + j * T;
      v[j] = k[j] >= total ? 0 : (k[j] < L1 ? s.lone[k[j]] : s.cand[k[j] - L1]);
      // a lone read: its own contig, rank 0, whole and forward (its length is filled in below)
      p[j] = k[j] >= total ? make_int4(-1, 0, 0, 0) : (k[j] < L1 ? make_int4(v[j], 0, -1, 0) : s.prd[k[j] - L1]);
      ok[j] = p[j].x >= 0;                 // not a chain shorter than min_chain
    }
    unsigned word[kScatterItems], wpv[kScatterItems];
    int32_t L[kScatterItems], pf[kScatterItems];
    int64_t base[kScatterItems];
#pragma unroll
    for (int j = 0; j < kScatterItems; ++j) {
      const int32_t m = ok[j] ? p[j].x : 0;
      word[j] = ok[j] ? s.hb[m >> 5] : 0u;
      wpv[j] = ok[j] ? s.wp[m >> 5] : 0u;
      L[j] = ok[j] ? g.len[v[j]] : 0;
      base[j] = ok[j] ? g.off[v[j]] : 0;
      pf[j] = ok[j] && g.pre && k[j] >= L1 ? s.pfirst[k[j] - L1] : 0;
    }
    long long cidx[kScatterItems], pos[kScatterItems];
#pragma unroll
    for (int j = 0; j < kScatterItems; ++j) {
      const int32_t m = p[j].x;
      cidx[j] = (long long)wpv[j] + __popc(word[j] & ((1u << (m & 31)) - 1u));
      pos[j] = ok[j] ? (long long)s.cbase[cidx[j]] + p[j].y : 0;
    }
#pragma unroll
    for (int j = 0; j < kScatterItems; ++j) {
      if (!ok[j]) continue;
      const int32_t m = p[j].x, rk = p[j].y;
      if (!((word[j] >> (m & 31)) & 1u) || pos[j] >= W) { set_error(s.derr, DERR_KERNEL, K_SCATTER, v[j]); continue; }
      const int o = p[j].w;
      const int32_t cb = p[j].z < 0 ? L[j] : p[j].z;
      // stored index of the piece's first base: suffix form, the last cb bases
      // of the oriented read; x-drop form, set by the chain stage (a read spelled
      // alone is whole and forward)
      const int64_t first = !g.pre ? (o == 0 ? L[j] - cb : cb - 1) : pf[j];
      const unsigned long long src = o == 0 ? (unsigned long long)(base[j] + first)
                                            : ((unsigned long long)(base[j] + first) | (1ull << 63));
      s.wsrc[pos[j]] = src;
      s.wlen[pos[j]] = s.part && s.part[cidx[j]] != s.part_p ? 0 : cb;   // another part's contig: empty
      s.wfirst[pos[j]] = rk == 0 ? (int32_t)cidx[j] : -1;
      if (s.wread) s.wread[pos[j]] = v[j];           // a graph without its reads: for the read exchange
    }
  }
}

// An empty graph: no contigs, and the one offset 0.
__global__ void k_contig_off(Scratch s) {
  pdl_enter();
  if (grid_tid() == 0) {
    s.contig_off[0] = 0;
    s.ctr->n_contigs = 0;
    s.ctr->n_walk = 0;
    s.ctr->n_tiles = 0;
    s.ctr->total_bases = 0;
  }
}

__global__ void k_export_contig_off(Scratch s, int64_t* out, long long cap) {
  pdl_enter();
  Counters* c = s.ctr;
  long long C = *(volatile unsigned*)&c->n_contigs;
  if (C + 1 > cap) {
    if (grid_tid() == 0) set_error(s.derr, DERR_CAPACITY, K_CONTIG_OFF, C + 1);
    return;
  }
  for (long long i = grid_tid(); i <= C; i += grid_threads()) out[i] = s.contig_off[i];
}

}  // namespace

cudaError_t launch_offsets(const DevGraph& g, const Scratch& s, const Tuning& t, const LaunchEnv& env,
                           int64_t* user_off, long long user_cap) {
  // No memset: the scans' last steps assign every counter of this stage, and
  // each scan zeroes the other one's descriptors (the heads scan the piece
  // scan's, the piece scan the heads scan's, for the next run); the graph
  // load zeroes both once.
  const long long words = (g.n + 31) / 32;
  const long long tiles_w = (words + kTileItems - 1) / kTileItems;
  const long long tiles_n = (g.n + kTileItems - 1) / kTileItems;
  if (tiles_n > s.scan_tiles_cap || tiles_w > s.scan_tiles_cap) return cudaErrorInvalidValue;
  const long long state_words = s.scan_tiles_cap + 1;
  if (g.n == 0) {
    k_contig_off<<<1, kBlock, 0, env.stream>>>(s);
    mark(env, "k_contig_off");
    return cudaGetLastError();
  }
  HeadWordLoad hl{s.hb, s.headq};
  HeadWordStore hs{s.wp, s.headq, s.qd, s.cbase, s.contig_off, user_off, user_cap, s.ctr};
  cudaError_t e = launch_k(k_scan<HeadWordLoad, HeadWordStore>, scan_grid(tiles_w, env), env, env.pdl_first, hl, hs,
                           words, (const unsigned*)nullptr, s.scan_state[0], s.scan_tiles_cap, s.derr,
                           (int)K_SCAN_HEADS, s.scan_state[2], state_words);
  if (e != cudaSuccess) return e;
  mark(env, "k_scan_heads");
  static const int scatter_resident = resident_blocks(k_scatter);   // a persistent grid
  const long long scatter_need = (g.n + (long long)kBlock * kScatterItems - 1) / ((long long)kBlock * kScatterItems);
  e = launch_k(k_scatter, (int)std::max(1LL, std::min((long long)env.num_sms * scatter_resident, scatter_need)), env,
               true, g, s);
  if (e != cudaSuccess) return e;
  mark(env, "k_scatter");
  PieceLoad pl{s.wlen, s.wfirst};
  PieceStore ps{s.out_off, s.contig_off, s.tile_seg, s.tiles_cap, t.tile_bytes, s.ctr, s.derr, user_off, user_cap};
  e = launch_k(k_scan<PieceLoad, PieceStore>, scan_grid(tiles_n, env), env, true, pl, ps, 0ll,
               (const unsigned*)&s.ctr->n_walk, s.scan_state[2], s.scan_tiles_cap, s.derr, (int)K_SCAN_OFFSETS,
               s.scan_state[0], state_words);
  if (e != cudaSuccess) return e;
  mark(env, "k_scan_pieces");
  return cudaGetLastError();
}

namespace {
struct ZeroLoad {
  __device__ unsigned long long operator()(long long) const { return 0ull; }
};
struct NoStore {
  __device__ void item(long long, unsigned long long) const {}
  __device__ void last(long long, unsigned long long) const {}
};
}  // namespace

cudaError_t launch_selftest_wait(unsigned long long* state, long long tiles, DevError* derr, const LaunchEnv& env) {
  k_scan<<<scan_grid(tiles, env), kBlock, 0, env.stream>>>(ZeroLoad{}, NoStore{}, tiles * kTileItems, nullptr, state,
                                                           tiles, derr, (int)K_SELFTEST_WAIT);
  mark(env, "k_scan_selftest");
  return cudaGetLastError();
}

cudaError_t launch_export_contig_off(const Scratch& s, int64_t* out, int64_t cap, const LaunchEnv& env) {
  cudaError_t e = launch_k(k_export_contig_off, env.num_sms, env, env.pdl_first, s, out, (long long)cap);
  if (e != cudaSuccess) return e;
  mark(env, "k_export_contig_off");
  return cudaGetLastError();
}

}  // namespace cg

// ------------------------------------------------------------------------
// GreedyPartitioning (LPT, Sec. 4.3). Contigs are weighted by their number of
// reads (the size estimate of Sec. 4.3) or by their spelled bases, sorted by
// weight, largest first, equal weights in contig order, and each in turn goes
// to the part whose weight sum is smallest so far, the lowest part on ties.
// The sort is a stable LSD radix sort, 8-bit digits, of kmax - weight; the
// assignment is sequential by definition and runs in one warp.
namespace cg {

namespace {

constexpr int kSortItems = 8;
constexpr long long kSortTile = (long long)kSortItems * kBlock;     // 2048 keys per tile

__device__ __forceinline__ unsigned digit_of(unsigned long long key, int pass) {
  return (unsigned)((key >> (8 * pass)) & 255ull);
}

__global__ void k_sort_keys(const Scratch s, long long C, int weight, unsigned long long kmax, unsigned long long* key,
                            int32_t* val) {
  for (long long i = grid_tid(); i < C; i += grid_threads()) {
    const long long w = weight == 0 ? (long long)s.qd[i] : s.contig_off[i + 1] - s.contig_off[i];
    key[i] = kmax - (unsigned long long)w;
    val[i] = (int32_t)i;
  }
}

// Per tile and digit, the keys of the tile with that digit, stored digit-major
// (hist[d * tiles + t]) so that one exclusive scan gives every scatter base.
__global__ void k_sort_hist(const unsigned long long* key, long long C, int pass, unsigned* hist, long long tiles) {
  __shared__ unsigned cnt[256];
  for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    for (int d = threadIdx.x; d < 256; d += blockDim.x) cnt[d] = 0;
    __syncthreads();
    for (int k = 0; k < kSortItems; ++k) {
      const long long i = t * kSortTile + k * kBlock + threadIdx.x;
      if (i < C) atomicAdd(&cnt[digit_of(key[i], pass)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(long long)d * tiles + t] = cnt[d];
    __syncthreads();
  }
}

struct HistLoad {
  const unsigned* h;
  __device__ unsigned long long operator()(long long i) const { return h[i]; }
};
struct HistStore {
  unsigned long long* base;
  __device__ void item(long long i, unsigned long long e) const { base[i] = e; }
  __device__ void last(long long, unsigned long long) const {}
};

// Stable scatter. A tile's keys are taken in index order, 256 per round; a
// key's place is its digit's base for the tile, plus the keys with that digit
// in earlier rounds, in earlier warps of this round and in earlier lanes.
__global__ void k_sort_scatter(const unsigned long long* key_in, const int32_t* val_in, unsigned long long* key_out,
                               int32_t* val_out, long long C, int pass, const unsigned long long* base,
                               long long tiles) {
  __shared__ unsigned running[256];
  __shared__ unsigned wcnt[kBlock / 32][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    for (int d = threadIdx.x; d < 256; d += blockDim.x) running[d] = 0;
    for (int k = 0; k < kSortItems; ++k) {
      const long long i = t * kSortTile + k * kBlock + threadIdx.x;
      const bool valid = i < C;
      const unsigned long long kk = valid ? key_in[i] : 0ull;
      const unsigned d = valid ? digit_of(kk, pass) : 256u + lane;   // no two invalid lanes match
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const unsigned before_lane = __popc(peers & ((1u << lane) - 1u));
      for (int x = threadIdx.x; x < (kBlock / 32) * 256; x += blockDim.x) (&wcnt[0][0])[x] = 0;
      __syncthreads();
      if (valid && before_lane == 0) wcnt[warp][d] = __popc(peers);
      __syncthreads();
      if (valid) {
        unsigned before_warp = 0;
        for (int w = 0; w < warp; ++w) before_warp += wcnt[w][d];
        const unsigned long long pos = base[(long long)d * tiles + t] + running[d] + before_warp + before_lane;
        key_out[pos] = kk;
        val_out[pos] = val_in[i];
      }
      __syncthreads();
      for (int dd = threadIdx.x; dd < 256; dd += blockDim.x) {
        unsigned sum = 0;
        for (int w = 0; w < kBlock / 32; ++w) sum += wcnt[w][dd];
        running[dd] += sum;
      }
      __syncthreads();
    }
  }
}

// One warp. A part is the key (weight sum << part_bits) | part index, so that
// the smallest key is the least-loaded part, the lowest index on ties, and no
// two keys are equal. Lane l holds the keys of parts l + 32 j, j < KPL, in
// registers. Per contig the warp takes the smallest key overall with the
// redux unit (one 32-bit minimum when every key fits in 32 bits, else the
// high halves, then the low halves at that high half) and the part holding
// it adds the contig's weight; no branch depends on the data.
template <int KPL, bool Narrow>
__global__ void __launch_bounds__(32) k_lpt_assign(const unsigned long long* key, const int32_t* val, long long C,
                                                   unsigned long long kmax, int P, int part_bits, int32_t* part,
                                                   int64_t* psum) {
  const unsigned full = 0xffffffffu;
  const unsigned long long idx_mask = (1ull << part_bits) - 1;
  const int lane = threadIdx.x;
  unsigned long long K[KPL];
#pragma unroll
  for (int j = 0; j < KPL; ++j) K[j] = lane + 32 * j < P ? (unsigned long long)(lane + 32 * j) : ~0ull;
  for (long long i0 = 0; i0 < C; i0 += 32) {
    const long long ii = i0 + lane;
    const int32_t ci = ii < C ? val[ii] : -1;
    const unsigned long long w = ii < C ? (kmax - key[ii]) << part_bits : 0ull;
    unsigned long long mine = 0;
    const int cnt = (int)min(32ll, C - i0);
    for (int q = 0; q < cnt; ++q) {
      const unsigned long long wq = __shfl_sync(full, w, q);
      unsigned long long my = K[0];
#pragma unroll
      for (int j = 1; j < KPL; ++j) my = min(my, K[j]);
      unsigned long long m;
      if (Narrow) {
        m = __reduce_min_sync(full, (unsigned)min(my, 0xffffffffull));
      } else {
        const unsigned hi = (unsigned)(my >> 32);
        const unsigned mhi = __reduce_min_sync(full, hi);
        const unsigned mlo = __reduce_min_sync(full, hi == mhi ? (unsigned)my : 0xffffffffu);
        m = ((unsigned long long)mhi << 32) | mlo;
      }
      mine = lane == q ? m : mine;
#pragma unroll
      for (int j = 0; j < KPL; ++j) K[j] += K[j] == m ? wq : 0ull;
    }
    if (ii < C) part[ci] = (int32_t)(mine & idx_mask);
  }
#pragma unroll
  for (int j = 0; j < KPL; ++j)
    if (lane + 32 * j < P) psum[lane + 32 * j] = (int64_t)(K[j] >> part_bits);
}

template <int KPL>
void lpt_launch(bool narrow, const unsigned long long* key, const int32_t* val, long long C, unsigned long long kmax,
                int P, int part_bits, int32_t* part, int64_t* psum, cudaStream_t st) {
  if (narrow) k_lpt_assign<KPL, true><<<1, 32, 0, st>>>(key, val, C, kmax, P, part_bits, part, psum);
  else k_lpt_assign<KPL, false><<<1, 32, 0, st>>>(key, val, C, kmax, P, part_bits, part, psum);
}

}  // namespace

cudaError_t launch_partition(const Scratch& s, long long C, int weight, long long max_weight, int P,
                             const SortBuffers& b, int32_t* part, int64_t* psum, const LaunchEnv& env) {
  int bits = 8;
  while (bits < 63 && (max_weight >> bits) != 0) bits += 8;
  const unsigned long long kmax = bits >= 64 ? ~0ull : (1ull << bits) - 1;
  if (C > 0) {
    const long long tiles = (C + kSortTile - 1) / kSortTile;
    const long long nh = 256 * tiles;
    const long long scan_tiles = (nh + kTileItems - 1) / kTileItems;
    if (scan_tiles > b.state_cap || tiles > b.tiles_cap) return cudaErrorInvalidValue;
    k_sort_keys<<<grid_for(C, env), kBlock, 0, env.stream>>>(s, C, weight, kmax, b.key[0], b.val[0]);
    mark(env, "k_sort_keys");
    const int grid = (int)std::min<long long>(tiles, (long long)env.num_sms * 4);
    int cur = 0;
    for (int pass = 0; pass < bits / 8; ++pass) {
      k_sort_hist<<<grid, kBlock, 0, env.stream>>>(b.key[cur], C, pass, b.hist, tiles);
      mark(env, "k_sort_hist");
      cudaMemsetAsync(b.state, 0, (size_t)(b.state_cap + 1) * sizeof(unsigned long long), env.stream);
      k_scan<<<scan_grid(scan_tiles, env), kBlock, 0, env.stream>>>(HistLoad{b.hist}, HistStore{b.base}, nh, nullptr,
                                                              b.state, b.state_cap, s.derr, K_SORT);
      mark(env, "k_scan_digits");
      k_sort_scatter<<<grid, kBlock, 0, env.stream>>>(b.key[cur], b.val[cur], b.key[cur ^ 1], b.val[cur ^ 1], C,
                                                      pass, b.base, tiles);
      mark(env, "k_sort_scatter");
      cur ^= 1;
    }
    int part_bits = 0;
    while ((1 << part_bits) < P) ++part_bits;
    if (part_bits + bits > 63) return cudaErrorInvalidValue;
    // narrow: the largest key, max_weight << part_bits | (P - 1), stays below 2^32 - 1
    const bool narrow = (((unsigned long long)max_weight << part_bits) | (unsigned long long)(P - 1)) < 0xffffffffull;
    const unsigned long long* kk = b.key[cur];
    const int32_t* vv = b.val[cur];
    if (P <= 32) lpt_launch<1>(narrow, kk, vv, C, kmax, P, part_bits, part, psum, env.stream);
    else if (P <= 64) lpt_launch<2>(narrow, kk, vv, C, kmax, P, part_bits, part, psum, env.stream);
    else if (P <= 128) lpt_launch<4>(narrow, kk, vv, C, kmax, P, part_bits, part, psum, env.stream);
    else if (P <= 256) lpt_launch<8>(narrow, kk, vv, C, kmax, P, part_bits, part, psum, env.stream);
    else if (P <= 512) lpt_launch<16>(narrow, kk, vv, C, kmax, P, part_bits, part, psum, env.stream);
    else lpt_launch<32>(narrow, kk, vv, C, kmax, P, part_bits, part, psum, env.stream);
    mark(env, "k_lpt_assign");
  } else {
    cudaMemsetAsync(psum, 0, (size_t)P * sizeof(int64_t), env.stream);
  }
  return cudaGetLastError();
}

}  // namespace cg
