// cg_lookback.cuh - single-pass exclusive scan over 64-bit values with
// decoupled look-back (sm_103a), shared by the kernels that lay out outputs.
// Tiles take tickets in order, publish their aggregate, then look back over
// their predecessors with one warp (32 descriptors at a time) until an
// inclusive prefix is found. The wait on a predecessor is bounded; on timeout
// the kernel records DERR_TIMEOUT and stops.
#pragma once

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

}  // namespace

}  // namespace cg
