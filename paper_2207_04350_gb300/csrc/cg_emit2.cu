// cg_emit2.cu - spelling the contigs (LocalAssembly concatenation, Alg. 2,
// Sec. 4.4) into a 2-bit output stream: the same contigs as the ASCII form,
// base i of the stream at byte i >> 2, bits 2 (i & 3), A=0 C=1 G=2 T=3 (the
// convention of the packed reads), a quarter of the bytes.
//
// The output is tiled like the ASCII form (tiles of tile_bytes bases, one warp
// per tile, persistent grid) and written in 16-byte chunks of 64 bases. A
// forward piece is a bit-granular copy of the packed read: five words and four
// funnel shifts per chunk. A reverse-complement piece takes the 64 stored
// bases below it, reverses the order of the 2-bit fields of each word and
// complements them (b -> 3 - b is a bitwise NOT of the field).
//
// The warp takes the tile's pieces 32 at a time, one per lane, and flattens
// every chunk they touch into one work list, one chunk per lane at a time,
// read with two aligned 16-byte loads (a warp reads contiguous memory). A chunk
// wholly inside one piece is stored as is. A chunk holding piece boundaries
// gets bits from consecutive pieces: the piece that covers its first base
// stores it (zeros elsewhere) and the later ones OR their bits in with
// atomics, after a warp barrier; pieces are contiguous in the output and the
// list is in piece order, so that first piece always comes first.
#include <cuda_runtime.h>

#include "cg_internal.cuh"

namespace cg {

namespace {

struct Chunk {
  uint32_t v[4];   // word k: bases 16k .. 16k + 15 of the chunk
};

__device__ __forceinline__ uint32_t load_word_checked(const uint32_t* words, const uint8_t* bytes,
                                                      long long full_words, long long packed_bytes, long long w) {
  if (w < 0) return 0u;                         // below the stream: only masked-off bases come from here
  if (w < full_words) return __ldg(words + w);
  uint32_t r = 0;
  for (int b = 0; b < 4; ++b) {
    const long long i = 4 * w + b;
    if (i < packed_bytes) r |= (uint32_t)__ldg(bytes + i) << (8 * b);
  }
  return r;
}

// Reverse the order of the sixteen 2-bit fields and complement each.
__device__ __forceinline__ uint32_t revcomp16(uint32_t x) {
  x = __brev(x);                                            // fields reversed, their two bits swapped
  x = ((x >> 1) & 0x55555555u) | ((x & 0x55555555u) << 1);
  return ~x;
}

// Bits of the fields [lo, hi) of a 16-field word (0 <= lo, hi <= 16).
__device__ __forceinline__ uint32_t field_mask(int lo, int hi) {
  if (hi <= lo) return 0u;
  const uint32_t up = hi >= 16 ? 0xffffffffu : (1u << (2 * hi)) - 1u;
  const uint32_t down = (1u << (2 * lo)) - 1u;              // lo < 16 here
  return up & ~down;
}

// The 64 bases of output chunk x0 (a multiple of 64) as if piece (oj, src,
// rc) covered all of them. Checked: word indices outside the stream read 0.
template <bool Checked>
__device__ __forceinline__ Chunk chunk_bits(const uint32_t* words, const uint8_t* bytes, long long full_words,
                                            long long packed_bytes, long long x0, long long oj, long long src, int rc) {
  // lowest stored base of the chunk: forward, the base at output x0; reverse, the base at output x0 + 63
  const long long p = rc ? src - (x0 - oj) - 63 : src + (x0 - oj);
  const long long w0 = p >> 4;                   // floor, also for p < 0
  const unsigned sh = (unsigned)(2 * (p & 15));
  uint32_t W[5];
#pragma unroll
  for (int k = 0; k < 5; ++k)
    W[k] = Checked ? load_word_checked(words, bytes, full_words, packed_bytes, w0 + k) : __ldg(words + w0 + k);
  Chunk c;
  if (rc) {
#pragma unroll
    for (int k = 0; k < 4; ++k) c.v[k] = revcomp16(__funnelshift_r(W[3 - k], W[4 - k], sh));
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) c.v[k] = __funnelshift_r(W[k], W[k + 1], sh);
  }
  return c;
}

// Keep output positions [lo, hi) of chunk x0 (absolute base positions).
__device__ __forceinline__ void keep(Chunk& c, long long x0, long long lo, long long hi) {
  const int l = (int)(max(lo, x0) - x0), h = (int)(min(hi, x0 + 64) - x0);
#pragma unroll
  for (int k = 0; k < 4; ++k) c.v[k] &= field_mask(min(max(l - 16 * k, 0), 16), min(max(h - 16 * k, 0), 16));
}

__device__ __forceinline__ void store_chunk(uint4* out, long long idx, const Chunk& c) {
  __stcs(out + idx, make_uint4(c.v[0], c.v[1], c.v[2], c.v[3]));
}

// The same chunk from two aligned 16-byte loads: the five words from the
// chunk's lowest stored base sit at d = (p >> 4) & 3 within the eight loaded.
__device__ __forceinline__ Chunk chunk_bits_aligned(const uint32_t* words, long long x0, long long oj, long long src,
                                                    int rc) {
  const long long p = rc ? src - (x0 - oj) - 63 : src + (x0 - oj);
  const long long wq = p >> 4;
  const unsigned sh = (unsigned)(2 * (p & 15));
  const uint4* q = reinterpret_cast<const uint4*>(words + (wq & ~3ll));
  const uint4 r0 = __ldg(q), r1 = __ldg(q + 1);
  const uint32_t R[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
  const int d = (int)(wq & 3);
  uint32_t W[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) W[k] = d == 0 ? R[k] : d == 1 ? R[k + 1] : d == 2 ? R[k + 2] : R[k + 3];
  Chunk c;
  if (rc) {
#pragma unroll
    for (int k = 0; k < 4; ++k) c.v[k] = revcomp16(__funnelshift_r(W[3 - k], W[4 - k], sh));
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) c.v[k] = __funnelshift_r(W[k], W[k + 1], sh);
  }
  return c;
}

constexpr int kWarps = kBlock / 32;
constexpr int kU = 2;              // chunks per lane in flight

__global__ void __launch_bounds__(kBlock) k_emit2(Scratch s, const uint8_t* packed, long long packed_bytes,
                                                  long long readable_words, bool aligned16, uint4* out,
                                                  long long cap_bytes, int tile_bases, long long t_begin,
                                                  long long t_end) {
  pdl_enter();
  __shared__ long long s_oj[kWarps][32], s_w[kWarps][32], s_a[kWarps][32], s_b[kWarps][32];
  __shared__ int s_start[kWarps][32];
  const Counters* c = s.ctr;
  const long long total = *(const volatile long long*)&c->total_bases;
  const long long need = 16 * ((total + 63) / 64);
  if (need > cap_bytes) {
    if (grid_tid() == 0) set_error(s.derr, DERR_CAPACITY, K_EMIT, need);
    return;
  }
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const unsigned full = 0xffffffffu;
  const long long ntiles = (total + tile_bases - 1) / tile_bases;
  const uint32_t* words = reinterpret_cast<const uint32_t*>(packed);
  uint32_t* out_words = reinterpret_cast<uint32_t*>(out);
  const long long full_words = packed_bytes >> 2;
  const long long t_stop = min(ntiles, t_end);          // the tiles [t_begin, t_end) of this launch
  for (long long t = t_begin + (grid_tid() >> 5); t < t_stop; t += grid_threads() >> 5) {
    const int lo = s.tile_seg[t], hi = s.tile_seg[t + 1];
    const long long tbase = t * (long long)tile_bases;
    const long long tend = min(tbase + (long long)tile_bases, total);
    for (int jb = lo; jb <= hi; jb += 32) {
      const int j = jb + lane;
      long long oj = 0, a = 0, b = 0;
      unsigned long long w = 0;
      int plen = 0;
      if (j <= hi) {
        oj = s.out_off[j];
        const long long oe = s.out_off[j + 1];
        w = s.wsrc[j];
        plen = (int)(oe - oj);
        a = max(oj, tbase);
        b = min(oe, tend);
      }
      const bool valid = a < b;
      const int rc = (int)(w >> 63);
      const long long src = (long long)(w & ~(1ull << 63));
      // chunks the piece touches: [a >> 6, (b - 1) >> 6]
      const int n = valid ? (int)(((b - 1) >> 6) - (a >> 6) + 1) : 0;
      // aligned loads are safe for the group when every piece's stored bases
      // stay 64 bases above the stream start and 9 words below the readable end
      const long long low = rc ? src - plen + 1 : src, top = rc ? src : src + plen - 1;
      const bool safe = aligned16 && __all_sync(full, !valid || (low >= 64 && (top >> 4) + 9 < readable_words));
      int incl = n;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += v;
      }
      const int T = __shfl_sync(full, incl, 31);
      s_oj[wq][lane] = oj;
      s_w[wq][lane] = (long long)w;
      s_a[wq][lane] = a;
      s_b[wq][lane] = b;
      s_start[wq][lane] = incl - n;
      __syncwarp();
      // warp-uniform trip count: every lane reaches the warp barriers below
      for (int f0 = 0; f0 < T; f0 += 32 * kU) {
        Chunk v[kU];
        long long ci[kU];
        bool fresh[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int f = f0 + 32 * u + lane;
          ci[u] = -1;
          fresh[u] = false;
          if (f < T) {
            // the piece of item f: the last lane whose first item is <= f
            // (starts are nondecreasing; l + step never exceeds 31)
            int l = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
              if (s_start[wq][l + step] <= f) l += step;
            const long long al = s_a[wq][l], bl = s_b[wq][l];
            const long long x0 = ((al >> 6) + (f - s_start[wq][l])) << 6;
            const unsigned long long wl = (unsigned long long)s_w[wq][l];
            const long long srcl = (long long)(wl & ~(1ull << 63));
            const int rcl = (int)(wl >> 63);
            v[u] = safe ? chunk_bits_aligned(words, x0, s_oj[wq][l], srcl, rcl)
                        : chunk_bits<true>(words, packed, full_words, packed_bytes, x0, s_oj[wq][l], srcl, rcl);
            if (al > x0 || bl < x0 + 64) keep(v[u], x0, al, bl);
            ci[u] = x0 >> 6;
            fresh[u] = al <= x0;               // this piece covers the chunk's first base
          }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u)
          if (ci[u] >= 0 && fresh[u]) store_chunk(out, ci[u], v[u]);
        __syncwarp();
#pragma unroll
        for (int u = 0; u < kU; ++u)
          if (ci[u] >= 0 && !fresh[u]) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
              if (v[u].v[k]) atomicOr(out_words + 4 * ci[u] + k, v[u].v[k]);
          }
        __syncwarp();
      }
    }
  }
}

}  // namespace

cudaError_t launch_emit2(const DevGraph& g, const Scratch& s, const Tuning& t, uint8_t* out, int64_t cap,
                         const LaunchEnv& env, long long t_begin, long long t_end) {
  static const int resident = resident_blocks(k_emit2);   // once, safely across threads
  const int per_sm = t.emit_blocks_per_sm < resident ? t.emit_blocks_per_sm : resident;
  const bool aligned16 = (reinterpret_cast<uintptr_t>(g.packed) & 15) == 0;
  cudaError_t e = launch_k(k_emit2, env.num_sms * per_sm, env, env.pdl_first, s, g.packed,
                           (long long)g.packed_bytes, (long long)(g.packed_readable / 4), aligned16,
                           reinterpret_cast<uint4*>(out), (long long)cap, t.tile_bytes, t_begin, t_end);
  if (e != cudaSuccess) return e;
  mark(env, "k_emit2");
  return cudaGetLastError();
}

}  // namespace cg
