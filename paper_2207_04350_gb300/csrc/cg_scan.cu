// cg_scan.cu - output layout of the contigs (sm_103a): the single-GPU form of
// the contig-size estimate, the redistribution by contig and the offsets of
// the concatenation (Alg. 2, Sec. 4.2-4.4).
//
//   1. scan over read ids of (1<<32 | q) at each chain's smallest read: the
//      contig index (high word) and the chain's first walk position (low word)
//      in contig order (contigs are listed by smallest read id);
//   2. scatter every spelled read to walk position first(chain) + rank: the
//      on-device compaction that replaces the induced-subgraph exchange;
//   3. scan over walk positions of the bases each read adds: the output
//      offset of every piece, the contig offsets and the map from output
//      tiles to the piece holding each tile's first byte.
//
// Both scans are single-pass decoupled look-back scans: tiles take tickets
// in order, publish their aggregate, then look back over predecessors with
// one warp (32 descriptors at a time) until an inclusive prefix is found.
// The wait on a predecessor is bounded; on timeout the kernel records
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

// ---- scan 1: chains in contig order ----
struct HeadsLoad {
  const int32_t* headq;
  __device__ unsigned long long operator()(long long i) const {
    int32_t q = headq[i];
    return q > 0 ? ((1ull << 32) | (unsigned)q) : 0ull;
  }
};
struct HeadsStore {
  unsigned long long* rb;
  Counters* c;
  DevError* derr;
  __device__ void item(long long i, unsigned long long e) const { rb[i] = e; }
  __device__ void last(long long count, unsigned long long total) const {
    rb[count] = total;
    c->n_contigs = (unsigned)(total >> 32);
    if ((unsigned)(total & 0xffffffffull) != c->n_emit) set_error(derr, DERR_KERNEL, K_SCAN_HEADS, count);
  }
};

// ---- scan 2: piece offsets over walk positions ----
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

// Every spelled read goes to walk position first(chain) + rank, with the
// stored-base address of its piece: forward reads add stored bases
// [len-contrib, len), reverse-complement reads the complement of stored
// bases contrib-1 down to 0.
__global__ void k_scatter(DevGraph g, Scratch s) {
  Counters* c = s.ctr;
  long long W = *(volatile unsigned*)&c->n_emit;
  for (long long k = grid_tid(); k < W; k += grid_threads()) {
    int32_t v = s.emit[k];
    int32_t ch = s.cid[v];
    unsigned long long pb = s.rb[ch];
    long long first = (long long)(pb & 0xffffffffull), cidx = (long long)(pb >> 32);
    int32_t rk = s.rank[v];
    long long pos = first + rk;
    if (ch < 0 || pos >= W) { set_error(s.derr, DERR_KERNEL, K_SCATTER, v); continue; }
    int o = s.orient[v];
    int32_t L = g.len[v], cb = s.contrib[v];
    int64_t base = g.off[v];
    unsigned long long src = o == 0 ? (unsigned long long)(base + L - cb)
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
  long long tiles_n = (g.n + kTileItems - 1) / kTileItems;
  if (tiles_n > s.scan_tiles_cap) return cudaErrorInvalidValue;
  // scan 1 (count = n, host known)
  cudaMemsetAsync(s.scan_state, 0, (size_t)(s.scan_tiles_cap + 1) * sizeof(unsigned long long), env.stream);
  HeadsLoad hl{s.headq};
  HeadsStore hs{s.rb, s.ctr, s.derr};
  if (g.n > 0)
    k_scan<<<(unsigned)tiles_n, kBlock, 0, env.stream>>>(hl, hs, (long long)g.n, nullptr, s.scan_state,
                                                        s.scan_tiles_cap, s.derr, K_SCAN_HEADS);
  ++*env.launches;
  k_scatter<<<grid_for(g.n, env), kBlock, 0, env.stream>>>(g, s);
  ++*env.launches;
  // scan 2 (count = walk positions, known on the device only; bounded by n)
  cudaMemsetAsync(s.scan_state, 0, (size_t)(s.scan_tiles_cap + 1) * sizeof(unsigned long long), env.stream);
  PieceLoad pl{s.wlen};
  PieceStore ps{s.wlen, s.out_off, s.tile_seg, s.tiles_cap, t.tile_bytes, s.ctr, s.derr};
  if (g.n > 0)
    k_scan<<<(unsigned)tiles_n, kBlock, 0, env.stream>>>(pl, ps, 0, &s.ctr->n_emit, s.scan_state, s.scan_tiles_cap,
                                                        s.derr, K_SCAN_OFFSETS);
  ++*env.launches;
  k_contig_off<<<grid_for(g.n + 1, env), kBlock, 0, env.stream>>>(s);
  ++*env.launches;
  return cudaGetLastError();
}

cudaError_t launch_export_contig_off(const Scratch& s, int64_t* out, int64_t cap, const LaunchEnv& env) {
  k_export_contig_off<<<env.num_sms, kBlock, 0, env.stream>>>(s, out, cap);
  ++*env.launches;
  return cudaGetLastError();
}

}  // namespace cg
