// cg_lookback.cuh - single-pass exclusive scan over 64-bit values with
// decoupled look-back (sm_103a), shared by the kernels that lay out outputs.
// Tiles take tickets in order, publish their aggregate, then look back over
// their predecessors with one warp (32 descriptors at a time) until an
// inclusive prefix is found. The wait on a predecessor is bounded; on timeout
// the kernel records DERR_TIMEOUT and stops.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

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

// A load may gather its inputs first: with
//   using Item = ...; Item fetch(long long i) const; unsigned long long value(long long i, const Item&) const
// the scan fetches all of a thread's items before computing any value, so
// that their loads overlap, and hands each item to the store:
//   void item(long long i, unsigned long long exclusive, const Item&) const
struct NoItem {
  using Item = char;
};
template <class L, class = void>
struct has_item : std::false_type {};
template <class L>
struct has_item<L, std::void_t<typename L::Item>> : std::true_type {};

// Generic single-pass exclusive scan of `count` 64-bit values.
//   Load:  unsigned long long operator()(long long i)
//   Store: void item(long long i, unsigned long long exclusive)   (or with the load's Item, above)
//          void last(long long count, unsigned long long total)
// Blocks loop over tiles by ticket (state[ticket_index], zero before the
// scan), so every tile a block waits for was taken earlier by a block that is
// already running, whatever the grid and however many blocks the GPU runs at
// once (a GPU shared with other work included). The blocks a count needs no
// tile of exit at once without taking one, so a grid sized for the largest
// count costs little when the count (read on the device) is small. A scan may
// also zero `clear` (clear_words words), another scan's descriptors, so that
// no separate memset runs before that one.
template <class Load, class Store>
__global__ void __launch_bounds__(kBlock) k_scan(Load ld, Store st, long long count_host, const unsigned* count_dev,
                                                 unsigned long long* state, long long ticket_index, DevError* derr,
                                                 int where, unsigned long long* clear = nullptr,
                                                 long long clear_words = 0) {
  pdl_enter();
  __shared__ unsigned long long sm[kTileItems];
  __shared__ unsigned long long warp_tot[kBlock / 32];
  __shared__ long long s_tile;
  __shared__ unsigned long long s_excl;
  for (long long i = (long long)blockIdx.x * kBlock + threadIdx.x; i < clear_words; i += (long long)gridDim.x * kBlock)
    clear[i] = 0ull;
  const long long count = count_dev ? (long long)*(const volatile unsigned*)count_dev : count_host;
  const long long tiles = (count + kTileItems - 1) / kTileItems;
  if ((long long)blockIdx.x >= tiles) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (;;) {
    if (tid == 0) s_tile = (long long)atomicAdd(&state[ticket_index], 1ull);
    __syncthreads();
    const long long tile = s_tile;
    if (tile >= tiles) return;                       // block-uniform
    const long long base = tile * kTileItems;
    typename std::conditional<has_item<Load>::value, Load, NoItem>::type::Item it[kItems];
    if constexpr (has_item<Load>::value) {
#pragma unroll
      for (int k = 0; k < kItems; ++k) {
        long long i = base + k * kBlock + tid;
        it[k] = i < count ? ld.fetch(i) : typename Load::Item{};
      }
#pragma unroll
      for (int k = 0; k < kItems; ++k) {
        long long i = base + k * kBlock + tid;
        sm[k * kBlock + tid] = i < count ? ld.value(i, it[k]) : 0ull;
      }
    } else {
      for (int k = 0; k < kItems; ++k) {
        long long i = base + k * kBlock + tid;
        sm[k * kBlock + tid] = i < count ? ld(i) : 0ull;
      }
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
    if constexpr (has_item<Load>::value) {
#pragma unroll
      for (int k = 0; k < kItems; ++k) {
        long long i = base + k * kBlock + tid;
        if (i < count) {
          unsigned long long e = sm[k * kBlock + tid];
          // the total before the item's store: a store may reuse its load's inputs
          const unsigned long long tot = i == count - 1 ? e + ld.value(i, it[k]) : 0ull;
          st.item(i, e, it[k]);
          if (i == count - 1) st.last(count, tot);
        }
      }
    } else {
      for (int k = 0; k < kItems; ++k) {
        long long i = base + k * kBlock + tid;
        if (i < count) {
          unsigned long long e = sm[k * kBlock + tid];
          const unsigned long long tot = i == count - 1 ? e + ld(i) : 0ull;
          st.item(i, e);
          if (i == count - 1) st.last(count, tot);
        }
      }
    }
    __syncthreads();                                 // sm and s_tile are reused by the next tile
  }
}

}  // namespace

// Grid of a scan over at most `tiles` tiles: blocks loop over tiles by
// ticket, so the grid need not exceed what runs at once (every scan here fits
// three blocks per SM: at most 80 registers per thread and 16.5 KB of shared
// memory per block).
inline unsigned scan_grid(long long tiles, const LaunchEnv& env) {
  const long long cap = (long long)env.num_sms * 3;
  return (unsigned)(tiles < 1 ? 1 : (tiles < cap ? tiles : cap));
}

}  // namespace cg
