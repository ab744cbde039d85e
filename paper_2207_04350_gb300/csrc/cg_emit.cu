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

// Reverse the order of the sixteen 2-bit groups.
__device__ __forceinline__ uint32_t rev2(uint32_t x) {
  x = __brev(x);
  return ((x >> 1) & 0x55555555u) | ((x & 0x55555555u) << 1);
}

// Eight 2-bit codes (bits 0..15) spread to one code per nibble.
__device__ __forceinline__ uint32_t spread8(uint32_t t) {
  t &= 0xFFFFu;
  t = (t | (t << 8)) & 0x00FF00FFu;
  t = (t | (t << 4)) & 0x0F0F0F0Fu;
  t = (t | (t << 2)) & 0x33333333u;
  return t;
}

// 16 codes -> 16 ASCII bytes: each nibble selects a byte of "ACGT".
__device__ __forceinline__ uint4 ascii16(uint32_t bits) {
  const uint32_t acgt = 0x54474341u;   // 'T' 'G' 'C' 'A' from the high byte down
  uint32_t lo = spread8(bits), hi = spread8(bits >> 16);
  return make_uint4(__byte_perm(acgt, 0u, lo & 0xFFFFu), __byte_perm(acgt, 0u, lo >> 16),
                    __byte_perm(acgt, 0u, hi & 0xFFFFu), __byte_perm(acgt, 0u, hi >> 16));
}

__device__ __forceinline__ int stored_base(const uint8_t* bytes, long long i) {
  return (__ldg(bytes + (i >> 2)) >> (2 * (i & 3))) & 3;
}

__device__ __forceinline__ long long shfl64(long long v, int src) {
  int lo = __shfl_sync(0xffffffffu, (int)(v & 0xffffffffll), src);
  int hi = __shfl_sync(0xffffffffu, (int)(v >> 32), src);
  return ((long long)hi << 32) | (unsigned)lo;
}

// One ASCII base at output position X of a piece: source word w (first stored
// base | reverse flag << 63), piece starts at output offset oj.
__device__ __forceinline__ uint8_t base_at(const uint8_t* packed, unsigned long long w, long long oj, long long X) {
  const long long src = (long long)(w & ~(1ull << 63));
  const long long k = X - oj;
  const int b = (w >> 63) ? (stored_base(packed, src - k) ^ 3) : stored_base(packed, src + k);
  return (uint8_t)(0x54474341u >> (8 * b));
}

// One warp per output tile (persistent grid). The warp takes the pieces of its
// tile, [tile_seg[t], tile_seg[t+1]], in order; of each piece it writes the
// 16-byte-aligned interior inside the tile with full chunks (U chunks per lane
// whose packed words are loaded together before any is used), and the at most
// 30 bytes at its two ragged ends byte by byte. Chunks shared by two pieces
// are thus written as disjoint bytes by each piece; no search per chunk.
template <int U>
__global__ void __launch_bounds__(kBlock) k_emit(Scratch s, const uint8_t* packed, long long packed_bytes,
                                                 uint8_t* out, long long cap, int tile_bytes) {
  const Counters* c = s.ctr;
  const long long total = *(const volatile long long*)&c->total_bases;
  if (total > cap) {
    if (grid_tid() == 0) set_error(s.derr, DERR_CAPACITY, K_EMIT, total);
    return;
  }
  const int lane = threadIdx.x & 31;
  const long long ntiles = (total + tile_bytes - 1) / tile_bytes;
  const uint32_t* words = reinterpret_cast<const uint32_t*>(packed);
  const long long full_words = packed_bytes >> 2;
  const int64_t* oo = s.out_off;
  const unsigned long long* ws = s.wsrc;
  for (long long t = grid_tid() >> 5; t < ntiles; t += grid_threads() >> 5) {
    const int lo = s.tile_seg[t], hi = s.tile_seg[t + 1];
    const long long tbase = t * (long long)tile_bytes;
    const long long tend = min(tbase + (long long)tile_bytes, total);
    for (int jb = lo; jb <= hi; jb += 32) {
      const int jl = jb + lane;
      const long long my_o = jl <= hi ? oo[jl] : 0, my_e = jl <= hi ? oo[jl + 1] : 0;
      const long long my_w = jl <= hi ? (long long)ws[jl] : 0;
      const int cnt = min(32, hi - jb + 1);
      for (int q = 0; q < cnt; ++q) {
        const long long oj = shfl64(my_o, q), oe = shfl64(my_e, q);
        const unsigned long long w = (unsigned long long)shfl64(my_w, q);
        const long long a = max(oj, tbase), b = min(oe, tend);   // the piece's bytes in this tile
        if (a >= b) continue;
        const long long A = (a + 15) & ~15ll, B = b & ~15ll;     // aligned interior [A, B)
        const bool rc = (w >> 63) != 0;
        const long long src = (long long)(w & ~(1ull << 63));
        for (long long X0 = A + 16ll * lane; X0 < B; X0 += 512ll * U) {
          uint32_t wlo[U], whi[U];
          int sh[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const long long X = X0 + 512ll * u;
            wlo[u] = whi[u] = 0u;
            sh[u] = 0;
            if (X >= B) continue;
            const long long k0 = X - oj;
            const long long p = rc ? src - k0 - 15 : src + k0;   // lowest stored base of the 16
            sh[u] = (int)(2 * (p & 15));
            wlo[u] = load_word(words, packed, full_words, packed_bytes, p >> 4);
            whi[u] = load_word(words, packed, full_words, packed_bytes, (p >> 4) + 1);
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const long long X = X0 + 512ll * u;
            if (X >= B) continue;
            uint32_t bits = __funnelshift_r(wlo[u], whi[u], (unsigned)sh[u]);
            if (rc) bits = ~rev2(bits);
            __stcs(reinterpret_cast<uint4*>(out + X), ascii16(bits));
          }
        }
        // ragged ends: [a, head_end) and, when there is an interior, [B, b)
        const long long head_end = A < B ? A : b;
        if (a + lane < head_end) out[a + lane] = base_at(packed, w, oj, a + lane);
        if (A < B && B + lane < b) out[B + lane] = base_at(packed, w, oj, B + lane);
      }
    }
  }
}

}  // namespace

cudaError_t launch_emit(const DevGraph& g, const Scratch& s, const Tuning& t, uint8_t* out, int64_t cap,
                        const LaunchEnv& env) {
  // a persistent grid: never more blocks than can be resident at once
  static int resident = 0;
  if (resident == 0) {
    int r = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_emit<4>, kBlock, 0);
    resident = r > 0 ? r : 1;
  }
  int per_sm = t.emit_blocks_per_sm < resident ? t.emit_blocks_per_sm : resident;
  int blocks = env.num_sms * per_sm;
  k_emit<4><<<blocks, kBlock, 0, env.stream>>>(s, g.packed, g.packed_bytes, out, cap, t.tile_bytes);
  ++*env.launches;
  return cudaGetLastError();
}

}  // namespace cg
