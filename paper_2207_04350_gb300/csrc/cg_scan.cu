// cg_scan.cu - output layout of the contigs (sm_103a): the single-GPU form of
// the contig-size estimate, the redistribution by contig and the offsets of
// the concatenation (Alg. 2, Sec. 4.2-4.4).
//
//   1. scan over the words of the heads bitmap (bit m set when read m is the
//      smallest read of a contig) of their popcounts: the contig index of
//      every head, listing contigs by smallest read id; each word's store
//      step lays the heads' read counts out in contig order;
//   2. scan of those read counts: every contig's first walk position;
//   3. scatter every spelled read to walk position first(contig) + rank: the
//      on-device compaction that replaces the induced-subgraph exchange;
//   4. scan over walk positions of the bases each read adds: the output
//      offset of every piece, the contig offsets and the map from output
//      tiles to the piece holding each tile's first byte.
//
// The scans are single-pass decoupled look-back scans: tiles take tickets in
// order, publish their aggregate, then look back over predecessors with one
// warp (32 descriptors at a time) until an inclusive prefix is found. The
// wait on a predecessor is bounded; on timeout the kernel records
// DERR_TIMEOUT and stops.
#include <cuda_runtime.h>

#include "cg_internal.cuh"

namespace cg {

namespace {

constexpr int kItems = 8;                       // items per thread
constexpr int kTileItems = kItems * kBlock;     // 2048 items per tile
constexpr unsigned long long kAgg = 1ull << 62, kPre = 2ull << 62, kValMask = (1ull << 62) - 1;
constexpr long long kLookbackSpins = 1ll << 22;

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
  return *(const volatile unsigned long long*)p;
}

// Warp 0 of the block: publish this tile's aggregate, find its exclusive
// prefix, publish the inclusive prefix. Returns the exclusive prefix.
__device__ unsigned long long lookback(unsigned long long* state, long long tile, unsigned long long agg,
                                       DevError* derr, int where) {
  int lane = threadIdx.x & 31;
  if (tile == 0) {
    if (lane == 0) atomicExch(&state[0], kPre | agg);
    return 0;
  }
  if (lane == 0) atomicExch(&state[tile], kAgg | agg);
  unsigned long long excl = 0;
  long long base = tile - 1;
  long long spins = 0;
  for (;;) {
    long long idx = base - lane;
    unsigned long long w = idx >= 0 ? ld_volatile(&state[idx]) : kPre;   // before tile 0: prefix 0
    unsigned st = (unsigned)(w >> 62);
    if (__any_sync(0xffffffffu, st == 0)) {
      if (++spins > kLookbackSpins) {
        if (lane == 0) set_error(derr, DERR_TIMEOUT, where, tile);
        return excl;
      }
      __nanosleep(spins < 32 ? 20 : 200);
      continue;
    }
    unsigned pm = __ballot_sync(0xffffffffu, st == 2);
    int first = pm ? __ffs(pm) - 1 : 32;
    unsigned long long v = lane <= first ? (w & kValMask) : 0ull;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    excl += __shfl_sync(0xffffffffu, v, 0);
    if (pm) break;
    base -= 32;
  }
  if (lane == 0) atomicExch(&state[tile], kPre | (excl + agg));
  return excl;
}

// Generic single-pass exclusive scan of `count` 64-bit values.
//   Load:  unsigned long long operator()(long long i)
//   Store: void item(long long i, unsigned long long exclusive)
//          void last(long long count, unsigned long long total)
template <class Load, class Store>
__global__ void __launch_bounds__(kBlock) k_scan(Load ld, Store st, long long count_host, const unsigned* count_dev,
                                                 unsigned long long* state, long long ticket_index, DevError* derr,
                                                 int where) {
  __shared__ unsigned long long sm[kTileItems];
  __shared__ unsigned long long warp_tot[kBlock / 32];
  __shared__ long long s_tile;
  __shared__ unsigned long long s_excl;
  long long count = count_dev ? (long long)*(const volatile unsigned*)count_dev : count_host;
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = (long long)atomicAdd(&state[ticket_index], 1ull);
  __syncthreads();
  long long tile = s_tile;
  long long base = tile * kTileItems;
  if (base >= count) return;
  for (int k = 0; k < kItems; ++k) {
    long long i = base + k * kBlock + tid;
    sm[k * kBlock + tid] = i < count ? ld(i) : 0ull;
  }
  __syncthreads();
  unsigned long long v[kItems], sum = 0;
  for (int k = 0; k < kItems; ++k) { v[k] = sm[tid * kItems + k]; sum += v[k]; }
  unsigned long long inc = sum;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  unsigned long long warp_excl = 0, agg = 0;
  for (int w = 0; w < kBlock / 32; ++w) {
    if (w < warp) warp_excl += warp_tot[w];
    agg += warp_tot[w];
  }
  if (warp == 0) {
    unsigned long long e = lookback(state, tile, agg, derr, where);
    if (lane == 0) s_excl = e;
  }
  __syncthreads();
  unsigned long long run = s_excl + warp_excl + inc - sum;
  for (int k = 0; k < kItems; ++k) { sm[tid * kItems + k] = run; run += v[k]; }
  __syncthreads();
  for (int k = 0; k < kItems; ++k) {
    long long i = base + k * kBlock + tid;
    if (i < count) {
      unsigned long long e = sm[k * kBlock + tid];
      st.item(i, e);
      if (i == count - 1) st.last(count, e + ld(i));
    }
  }
}

// ---- scan 1: contig index of every head (bitmap popcounts) ----
struct HeadWordLoad {
  const unsigned* hb;
  __device__ unsigned long long operator()(long long w) const { return (unsigned long long)__popc(hb[w]); }
};
struct HeadWordStore {
  const unsigned* hb;
  unsigned* wp;
  const int32_t* headq;
  int32_t* qd;
  Counters* c;
  __device__ void item(long long w, unsigned long long e) const {
    wp[w] = (unsigned)e;
    unsigned bits = hb[w];
    unsigned k = (unsigned)e;
    while (bits) {
      int b = __ffs(bits) - 1;
      bits &= bits - 1;
      qd[k++] = headq[32 * w + b];     // contigs in order of their smallest read
    }
  }
  __device__ void last(long long, unsigned long long total) const { c->n_contigs = (unsigned)total; }
};

// ---- scan 2: first walk position of every contig ----
struct ContigLoad {
  const int32_t* qd;
  __device__ unsigned long long operator()(long long i) const { return (unsigned long long)(unsigned)qd[i]; }
};
struct ContigStore {
  unsigned long long* cbase;
  Counters* c;
  __device__ void item(long long i, unsigned long long e) const { cbase[i] = e; }
  __device__ void last(long long count, unsigned long long total) const {
    cbase[count] = total;
    c->n_walk = (unsigned)total;
  }
};

// ---- scan 4: piece offsets over walk positions ----
struct PieceLoad {
  const int32_t* wlen;
  __device__ unsigned long long operator()(long long j) const { return (unsigned long long)(unsigned)wlen[j]; }
};
struct PieceStore {
  const int32_t* wlen;
  int64_t* out_off;
  int32_t* tile_seg;
  long long tiles_cap;
  long long tile_bytes;
  Counters* c;
  DevError* derr;
  __device__ void item(long long j, unsigned long long e) const {
    long long o = (long long)e, L = wlen[j];
    out_off[j] = o;
    long long t0 = (o + tile_bytes - 1) / tile_bytes, t1 = (o + L + tile_bytes - 1) / tile_bytes;
    for (long long t = t0; t < t1; ++t) {
      if (t < tiles_cap) tile_seg[t] = (int32_t)j;
      else set_error(derr, DERR_KERNEL, K_SCAN_OFFSETS, t);
    }
  }
  __device__ void last(long long count, unsigned long long total) const {
    out_off[count] = (long long)total;
    c->total_bases = (long long)total;
    long long nt = ((long long)total + tile_bytes - 1) / tile_bytes;
    c->n_tiles = (unsigned)nt;
    if (nt <= tiles_cap) tile_seg[nt] = (int32_t)(count - 1);
    else set_error(derr, DERR_KERNEL, K_SCAN_OFFSETS, nt);
  }
};

// Every spelled read goes to walk position first(contig) + rank, with the
// stored-base address of its piece: forward reads add stored bases
// [len-contrib, len), reverse-complement reads the complement of stored
// bases contrib-1 down to 0. The spelled reads are the lone reads of the
// mask stage, those cut off by branch reads, and the chain reads of chains
// long enough to be contigs.
__global__ void k_scatter(DevGraph g, Scratch s) {
  Counters* c = s.ctr;
  const long long L1 = *(volatile unsigned*)&c->n_lone, L2 = *(volatile unsigned*)&c->n_lone2;
  const long long NC = *(volatile unsigned*)&c->n_chain, W = *(volatile unsigned*)&c->n_walk;
  const long long total = L1 + L2 + NC;
  for (long long k = grid_tid(); k < total; k += grid_threads()) {
    const int32_t v = k < L1 ? s.lone[k] : (k < L1 + L2 ? s.lone2[k - L1] : s.chain[k - L1 - L2]);
    const int32_t m = s.cid[v];
    if (m < 0) continue;                 // a chain shorter than min_chain
    const unsigned word = s.hb[m >> 5];
    const long long cidx = (long long)s.wp[m >> 5] + __popc(word & ((1u << (m & 31)) - 1u));
    const int32_t rk = s.rank[v];
    const long long pos = (long long)s.cbase[cidx] + rk;
    if (!((word >> (m & 31)) & 1u) || pos >= W) { set_error(s.derr, DERR_KERNEL, K_SCATTER, v); continue; }
    const int o = s.orient[v];
    const int32_t L = g.len[v], cb = s.contrib[v];
    const int64_t base = g.off[v];
    const unsigned long long src = o == 0 ? (unsigned long long)(base + L - cb)
                                          : ((unsigned long long)(base + cb - 1) | (1ull << 63));
    s.wsrc[pos] = src;
    s.wlen[pos] = cb;
    if (rk == 0) s.cstart[cidx] = (int32_t)pos;
  }
}

__global__ void k_contig_off(Scratch s) {
  Counters* c = s.ctr;
  long long C = *(volatile unsigned*)&c->n_contigs;
  for (long long i = grid_tid(); i <= C; i += grid_threads())
    s.contig_off[i] = i < C ? s.out_off[s.cstart[i]] : c->total_bases;
}

__global__ void k_export_contig_off(Scratch s, int64_t* out, long long cap) {
  Counters* c = s.ctr;
  long long C = *(volatile unsigned*)&c->n_contigs;
  if (C + 1 > cap) {
    if (grid_tid() == 0) set_error(s.derr, DERR_CAPACITY, K_CONTIG_OFF, C + 1);
    return;
  }
  for (long long i = grid_tid(); i <= C; i += grid_threads()) out[i] = s.contig_off[i];
}

}  // namespace

cudaError_t launch_offsets(const DevGraph& g, const Scratch& s, const Tuning& t, const LaunchEnv& env) {
  cudaMemsetAsync(&s.ctr->n_contigs, 0, sizeof(Counters) - offsetof(Counters, n_contigs), env.stream);
  const long long words = (g.n + 31) / 32;
  const long long tiles_w = (words + kTileItems - 1) / kTileItems;
  const long long tiles_n = (g.n + kTileItems - 1) / kTileItems;
  if (tiles_n > s.scan_tiles_cap || tiles_w > s.scan_tiles_cap) return cudaErrorInvalidValue;
  // the three scans' tile descriptors and tickets are contiguous: one memset
  cudaMemsetAsync(s.scan_state[0], 0, (size_t)3 * (s.scan_tiles_cap + 1) * sizeof(unsigned long long), env.stream);
  if (g.n == 0) {
    k_contig_off<<<1, kBlock, 0, env.stream>>>(s);
    mark(env, "k_contig_off");
    return cudaGetLastError();
  }
  HeadWordLoad hl{s.hb};
  HeadWordStore hs{s.hb, s.wp, s.headq, s.qd, s.ctr};
  k_scan<<<(unsigned)tiles_w, kBlock, 0, env.stream>>>(hl, hs, words, nullptr, s.scan_state[0], s.scan_tiles_cap,
                                                       s.derr, K_SCAN_HEADS);
  mark(env, "k_scan_heads");
  ContigLoad cl{s.qd};
  ContigStore cs{s.cbase, s.ctr};
  k_scan<<<(unsigned)tiles_n, kBlock, 0, env.stream>>>(cl, cs, 0, &s.ctr->n_contigs, s.scan_state[1],
                                                       s.scan_tiles_cap, s.derr, K_SCAN_HEADS);
  mark(env, "k_scan_contigs");
  k_scatter<<<grid_for(g.n, env), kBlock, 0, env.stream>>>(g, s);
  mark(env, "k_scatter");
  PieceLoad pl{s.wlen};
  PieceStore ps{s.wlen, s.out_off, s.tile_seg, s.tiles_cap, t.tile_bytes, s.ctr, s.derr};
  k_scan<<<(unsigned)tiles_n, kBlock, 0, env.stream>>>(pl, ps, 0, &s.ctr->n_walk, s.scan_state[2], s.scan_tiles_cap,
                                                       s.derr, K_SCAN_OFFSETS);
  mark(env, "k_scan_pieces");
  k_contig_off<<<grid_for(g.n + 1, env), kBlock, 0, env.stream>>>(s);
  mark(env, "k_contig_off");
  return cudaGetLastError();
}

cudaError_t launch_export_contig_off(const Scratch& s, int64_t* out, int64_t cap, const LaunchEnv& env) {
  k_export_contig_off<<<env.num_sms, kBlock, 0, env.stream>>>(s, out, cap);
  mark(env, "k_export_contig_off");
  return cudaGetLastError();
}

}  // namespace cg
