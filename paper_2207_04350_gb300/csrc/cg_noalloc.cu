// cg_noalloc.cu - cg_offsets_noalloc: the library's exclusive-prefix offset
// scan (the look-back scan of cg_lookback.cuh that places contigs and read
// pieces in the output) in a form that allocates no device memory. Its
// look-back scratch lives in one fixed file-scope device array instead of
// buffers from cudaMalloc.
#include <cuda_runtime.h>

#include <mutex>

#include "cg.h"
#include "cg_lookback.cuh"

namespace {

using cg::kTileItems;                                                 // 2048 lengths per tile
constexpr long long kMaxTiles = CG_NOALLOC_MAX_COUNT / kTileItems;    // 8192

// Scratch shared by every call on a device, in 8-byte words:
//   [0, 2)                the first error a tile records (cg::DevError: code, kernel, tile);
//   [2, 2 + tiles)        the tiles' look-back descriptors (status in the top two bits, sum below);
//   [2 + tiles]           the ticket counter that hands out tiles in order.
// 8 * (kMaxTiles + 3) bytes = 64 KiB + 24 bytes, held by the GPU until exit.
static __device__ __align__(256) unsigned long long g_scan_scratch[kMaxTiles + 3];

static_assert(CG_NOALLOC_MAX_COUNT % kTileItems == 0, "max count must be whole tiles");
static_assert(sizeof(cg::DevError) == 2 * sizeof(unsigned long long), "error record must fill two words");

struct LenLoad {
  const int32_t* len;
  __device__ unsigned long long operator()(long long i) const { return (unsigned long long)(unsigned)len[i]; }
};

struct OffStore {
  int64_t* out;
  __device__ void item(long long i, unsigned long long excl) const { out[i] = (int64_t)excl; }
  __device__ void last(long long count, unsigned long long total) const { out[count] = (int64_t)total; }
};

struct DeviceSetup {
  unsigned long long* scratch = nullptr;   // device address of g_scan_scratch
  int num_sms = 0;
};

std::mutex g_mu;
DeviceSetup g_dev[256];

bool is_device_memory(const void* p) {
  cudaPointerAttributes a = {};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" CG_API cg_status cg_offsets_noalloc(const int32_t* lengths, int64_t count, int64_t* offsets,
                                               void* cuda_stream) {
  if (count < 0 || count > CG_NOALLOC_MAX_COUNT || !offsets || (count > 0 && !lengths)) return CG_EINVAL;
  if (reinterpret_cast<uintptr_t>(offsets) % alignof(int64_t) != 0 ||
      reinterpret_cast<uintptr_t>(lengths) % alignof(int32_t) != 0)
    return CG_EINVAL;
  if (!is_device_memory(offsets) || (count > 0 && !is_device_memory(lengths))) return CG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    cudaGetLastError();
    return CG_ECUDA;
  }
  DeviceSetup su;
  {
    // Set-up, once per device with that device current: in host code the
    // name g_scan_scratch is only a host-side stand-in, so the kernel is given
    // the array's device address instead.
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev[dev].scratch) {
      void* p = nullptr;
      int sms = 0;
      if (cudaGetSymbolAddress(&p, g_scan_scratch) != cudaSuccess || !p ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        return CG_ECUDA;
      }
      g_dev[dev].scratch = static_cast<unsigned long long*>(p);
      g_dev[dev].num_sms = sms;
    }
    su = g_dev[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const long long tiles = (count + kTileItems - 1) / kTileItems;
  cg::DevError* derr = reinterpret_cast<cg::DevError*>(su.scratch);
  unsigned long long* state = su.scratch + 2;
  // the error record, this call's tile descriptors and the ticket start at zero
  if (cudaMemsetAsync(su.scratch, 0, (size_t)(tiles + 3) * sizeof(unsigned long long), s) != cudaSuccess) {
    cudaGetLastError();
    return CG_ECUDA;
  }
  if (count == 0) {
    if (cudaMemsetAsync(offsets, 0, sizeof(int64_t), s) != cudaSuccess) {
      cudaGetLastError();
      return CG_ECUDA;
    }
  } else {
    cg::LaunchEnv env = {};
    env.num_sms = su.num_sms;
    const unsigned grid = cg::scan_grid(tiles, env);
    cg::k_scan<LenLoad, OffStore><<<grid, cg::kBlock, 0, s>>>(LenLoad{lengths}, OffStore{offsets}, count, nullptr,
                                                              state, tiles, derr, (int)cg::K_SCAN_OFFSETS);
    if (cudaGetLastError() != cudaSuccess) return CG_ECUDA;
  }
  int err = 0;
  if (cudaMemcpyAsync(&err, &derr->err, sizeof(err), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return CG_ECUDA;
  }
  if (err == cg::DERR_TIMEOUT) return CG_ETIMEOUT;
  return err ? CG_EKERNEL : CG_OK;
}
