// cg_emit.cu - spelling the contigs (LocalAssembly concatenation, Alg. 2,
// Sec. 4.4) on sm_103a.
//
// The output is one byte stream holding every contig back to back; each read
// of a contig owns one piece [out_off[j], out_off[j+1]) of it (walk position
// j). The kernel tiles the OUTPUT: a persistent grid strides over fixed-size
// tiles, and inside a tile every thread produces aligned 16-byte chunks, so
// stores are full 128-bit, coalesced and independent of piece lengths (a
// long contig spreads over many blocks, short pieces share a chunk).
//
// A chunk inside one piece is read with two 32-bit words of the packed
// stream and one funnel shift (16 bases); a reverse-complement piece takes
// the 16 bases below it, reverses the 2-bit groups and complements them
// (complement of b is 3-b = b^3, i.e. bitwise NOT). Four lookups in a
// shared-memory table turn 4 bases (one byte) into 4 ASCII characters.
// Chunks that straddle pieces, or sit at the very start of the stream, take
// the base-by-base path.
#include <cuda_runtime.h>

#include "cg_internal.cuh"

namespace cg {

namespace {

__device__ __forceinline__ uint32_t load_word(const uint32_t* words, const uint8_t* bytes, long long full_words,
                                              long long packed_bytes, long long w) {
  if (w < full_words) return __ldg(words + w);
  uint32_t r = 0;
  for (int b = 0; b < 4; ++b) {
    long long i = 4 * w + b;
    if (i < packed_bytes) r |= (uint32_t)__ldg(bytes + i) << (8 * b);
  }
  return r;
}

// 16 bases starting at stored base p (p >= 0); base k at bits 2k.
__device__ __forceinline__ uint32_t get16(const uint32_t* words, const uint8_t* bytes, long long full_words,
                                          long long packed_bytes, long long p) {
  long long w = p >> 4;
  uint32_t lo = load_word(words, bytes, full_words, packed_bytes, w);
  uint32_t hi = load_word(words, bytes, full_words, packed_bytes, w + 1);
  return __funnelshift_r(lo, hi, (unsigned)(2 * (p & 15)));
}

// Reverse the order of the sixteen 2-bit groups.
__device__ __forceinline__ uint32_t rev2(uint32_t x) {
  x = __brev(x);
  return ((x >> 1) & 0x55555555u) | ((x & 0x55555555u) << 1);
}

__device__ __forceinline__ int stored_base(const uint8_t* bytes, long long i) {
  return (__ldg(bytes + (i >> 2)) >> (2 * (i & 3))) & 3;
}

__global__ void __launch_bounds__(kBlock) k_emit(Scratch s, const uint8_t* packed, long long packed_bytes,
                                                 uint8_t* out, long long cap, int tile_bytes) {
  __shared__ uint32_t lut[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    uint32_t v = 0;
    for (int k = 0; k < 4; ++k) v |= (uint32_t)("ACGT"[(i >> (2 * k)) & 3]) << (8 * k);
    lut[i] = v;
  }
  __syncthreads();
  const Counters* c = s.ctr;
  long long total = *(const volatile long long*)&c->total_bases;
  if (total > cap) {
    if (grid_tid() == 0) set_error(s.derr, DERR_CAPACITY, K_EMIT, total);
    return;
  }
  long long ntiles = (total + tile_bytes - 1) / tile_bytes;
  const uint32_t* words = reinterpret_cast<const uint32_t*>(packed);
  long long full_words = packed_bytes >> 2;
  const int64_t* oo = s.out_off;
  const unsigned long long* ws = s.wsrc;
  int chunks = tile_bytes >> 4;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int lo = s.tile_seg[t], hi = s.tile_seg[t + 1];
    long long tbase = t * (long long)tile_bytes;
    for (int k = threadIdx.x; k < chunks; k += blockDim.x) {
      long long X = tbase + 16ll * k;
      if (X >= total) break;
      int a = lo, b = hi;                       // last piece starting at or before X
      while (a < b) {
        int mid = (a + b + 1) >> 1;
        if (oo[mid] <= X) a = mid; else b = mid - 1;
      }
      int j = a;
      long long oj = oo[j], oe = oo[j + 1];
      uint32_t r0, r1, r2, r3;
      bool fast = X + 16 <= oe;
      if (fast) {
        unsigned long long w = ws[j];
        long long src = (long long)(w & ~(1ull << 63));
        long long k0 = X - oj;
        uint32_t bits;
        if (!(w >> 63)) {
          bits = get16(words, packed, full_words, packed_bytes, src + k0);
        } else {
          long long q = src - k0 - 15;
          if (q < 0) {
            fast = false;
          } else {
            bits = ~rev2(get16(words, packed, full_words, packed_bytes, q));
          }
        }
        if (fast) {
          r0 = lut[bits & 255u];
          r1 = lut[(bits >> 8) & 255u];
          r2 = lut[(bits >> 16) & 255u];
          r3 = lut[bits >> 24];
        }
      }
      if (!fast) {
        uint32_t r[4] = {0u, 0u, 0u, 0u};
        int jj = j;
        for (int bb = 0; bb < 16; ++bb) {
          long long Xb = X + bb;
          if (Xb >= total) break;
          while (jj < hi && Xb >= oo[jj + 1]) ++jj;
          unsigned long long w = ws[jj];
          long long src = (long long)(w & ~(1ull << 63));
          long long kk = Xb - oo[jj];
          int base = (w >> 63) ? (stored_base(packed, src - kk) ^ 3) : stored_base(packed, src + kk);
          r[bb >> 2] |= (uint32_t)("ACGT"[base]) << (8 * (bb & 3));
        }
        r0 = r[0]; r1 = r[1]; r2 = r[2]; r3 = r[3];
      }
      if (X + 16 <= total) {
        *reinterpret_cast<uint4*>(out + X) = make_uint4(r0, r1, r2, r3);
      } else {
        uint32_t r[4] = {r0, r1, r2, r3};
        for (long long bb = 0; X + bb < total; ++bb) out[X + bb] = (uint8_t)(r[bb >> 2] >> (8 * (bb & 3)));
      }
    }
  }
}

}  // namespace

cudaError_t launch_emit(const DevGraph& g, const Scratch& s, const Tuning& t, uint8_t* out, int64_t cap,
                        const LaunchEnv& env) {
  int blocks = env.num_sms * t.emit_blocks_per_sm;
  k_emit<<<blocks, kBlock, 0, env.stream>>>(s, g.packed, g.packed_bytes, out, cap, t.tile_bytes);
  ++*env.launches;
  return cudaGetLastError();
}

}  // namespace cg
