// cg_noalloc.cu - cg_offsets_noalloc: the exclusive-prefix offset scan of the
// library (the one that places contigs and read pieces in the output), in a
// form that allocates no device memory. Its look-back scratch lives in one
// fixed file-scope device array instead of buffers from cudaMalloc.
#include <cuda_runtime.h>

#include <mutex>

#include "cg.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 8;
constexpr long long kTile = kThreads * kPerThread;                // 2048 lengths per block
constexpr long long kMaxTiles = CG_NOALLOC_MAX_COUNT / kTile;      // 8192
constexpr unsigned long long kAgg = 1ull << 62, kPre = 2ull << 62, kVal = (1ull << 62) - 1;
constexpr long long kSpinLimit = 1ll << 22;

// Scratch shared by every call on a device: [0] tile ticket, [1] error word,
// [2, 2 + tiles) tile descriptors (status in the top two bits, sum below).
// 8 * (kMaxTiles + 2) bytes = 64 KiB + 16 bytes, held by the GPU until exit.
static __device__ __align__(256) unsigned long long g_scan_scratch[kMaxTiles + 2];

static_assert(CG_NOALLOC_MAX_COUNT % kTile == 0, "max count must be whole tiles");

__global__ void __launch_bounds__(kThreads) k_offsets_noalloc(const int32_t* len, long long count, int64_t* out,
                                                              unsigned long long* scratch) {
  __shared__ unsigned long long sm[kTile];
  __shared__ unsigned long long warp_tot[kThreads / 32];
  __shared__ long long s_tile;
  __shared__ unsigned long long s_excl;
  unsigned long long* desc = scratch + 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = (long long)atomicAdd(&scratch[0], 1ull);
  __syncthreads();
  const long long tile = s_tile, base = tile * kTile;
  if (base >= count) return;
  for (int k = 0; k < kPerThread; ++k) {
    long long i = base + k * kThreads + tid;
    sm[k * kThreads + tid] = i < count ? (unsigned long long)(unsigned)len[i] : 0ull;
  }
  __syncthreads();
  unsigned long long v[kPerThread], sum = 0;
  for (int k = 0; k < kPerThread; ++k) { v[k] = sm[tid * kPerThread + k]; sum += v[k]; }
  unsigned long long inc = sum;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  unsigned long long warp_excl = 0, agg = 0;
  for (int w = 0; w < kThreads / 32; ++w) {
    if (w < warp) warp_excl += warp_tot[w];
    agg += warp_tot[w];
  }
  if (warp == 0) {
    // publish the tile sum, then look back over predecessors 32 at a time
    unsigned long long excl = 0;
    if (tile == 0) {
      if (lane == 0) atomicExch(&desc[0], kPre | agg);
    } else {
      if (lane == 0) atomicExch(&desc[tile], kAgg | agg);
      long long back = tile - 1, spins = 0;
      for (;;) {
        long long idx = back - lane;
        unsigned long long w = idx >= 0 ? *(const volatile unsigned long long*)&desc[idx] : kPre;
        unsigned st = (unsigned)(w >> 62);
        if (__any_sync(0xffffffffu, st == 0)) {
          if (++spins > kSpinLimit) {           // bounded wait: record and stop
            if (lane == 0) atomicExch(&scratch[1], 1ull);
            break;
          }
          __nanosleep(spins < 32 ? 20 : 200);
          continue;
        }
        unsigned pm = __ballot_sync(0xffffffffu, st == 2);
        int first = pm ? __ffs(pm) - 1 : 32;
        unsigned long long x = lane <= first ? (w & kVal) : 0ull;
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        excl += __shfl_sync(0xffffffffu, x, 0);
        if (pm) break;
        back -= 32;
      }
      if (lane == 0) atomicExch(&desc[tile], kPre | (excl + agg));
    }
    if (lane == 0) s_excl = excl;
  }
  __syncthreads();
  unsigned long long run = s_excl + warp_excl + inc - sum;
  for (int k = 0; k < kPerThread; ++k) { sm[tid * kPerThread + k] = run; run += v[k]; }
  __syncthreads();
  for (int k = 0; k < kPerThread; ++k) {
    long long i = base + k * kThreads + tid;
    if (i < count) {
      unsigned long long e = sm[k * kThreads + tid];
      out[i] = (int64_t)e;
      if (i == count - 1) out[count] = (int64_t)(e + (unsigned)len[i]);
    }
  }
}

std::mutex g_mu;
unsigned long long* g_addr[256] = {};   // device address of g_scan_scratch, per device

}  // namespace

extern "C" CG_API cg_status cg_offsets_noalloc(const int32_t* lengths, int64_t count, int64_t* offsets,
                                               void* cuda_stream) {
  if (count < 0 || count > CG_NOALLOC_MAX_COUNT || !offsets || (count > 0 && !lengths)) return CG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    cudaGetLastError();
    return CG_ECUDA;
  }
  unsigned long long* scratch = nullptr;
  {
    // Set-up, once per device with that device current: the host-side name
    // g_scan_scratch is only a stand-in, the kernel needs the device address.
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scan_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return CG_ECUDA;
      }
      g_addr[dev] = static_cast<unsigned long long*>(p);
    }
    scratch = g_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const long long tiles = (count + kTile - 1) / kTile;
  // the ticket, the error word and this call's tile descriptors start at zero
  if (cudaMemsetAsync(scratch, 0, (size_t)(tiles + 2) * sizeof(unsigned long long), s) != cudaSuccess) {
    cudaGetLastError();
    return CG_ECUDA;
  }
  if (count == 0) {
    if (cudaMemsetAsync(offsets, 0, sizeof(int64_t), s) != cudaSuccess) {
      cudaGetLastError();
      return CG_ECUDA;
    }
  } else {
    k_offsets_noalloc<<<(unsigned)tiles, kThreads, 0, s>>>(lengths, count, offsets, scratch);
    if (cudaGetLastError() != cudaSuccess) return CG_ECUDA;
  }
  unsigned long long err = 0;
  if (cudaMemcpyAsync(&err, scratch + 1, sizeof(err), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return CG_ECUDA;
  }
  return err ? CG_ETIMEOUT : CG_OK;
}
