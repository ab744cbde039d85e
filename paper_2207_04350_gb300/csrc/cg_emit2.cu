// cg_emit2.cu - spelling the contigs (LocalAssembly concatenation, Alg. 2,
// Sec. 4.4) into a 2-bit output stream: the same contigs as the ASCII form,
// base i of the stream at byte i >> 2, bits 2 (i & 3), A=0 C=1 G=2 T=3 (the
// convention of the packed reads), a quarter of the bytes.
//
// The output is tiled like the ASCII form (tiles of tile_bytes bases, one warp
// per tile, persistent grid, tiles taken as the warps free up (TileQueue):
// 0.309 ms on the 3.1 Gb graph against 0.326 in a fixed stride) and written
// in 16-byte chunks of
// 64 bases. A
// forward piece is a bit-granular copy of the packed read: five words and four
// funnel shifts per chunk. A reverse-complement piece takes the 64 stored
// bases below it, reverses the order of the 2-bit fields of each word and
// complements them (b -> 3 - b is a bitwise NOT of the field).
//
// At a tile's start the warp asks L2 for the source bytes of all the tile's
// pieces (they lie at unrelated places of the read stream). The interior
// chunks of the tile's pieces (all 64 bases inside one piece) are one work
// list that the warp's lanes walk with forward-only cursors; a chunk with a
// piece boundary inside is assembled by one lane from the pieces overlapping
// it and stored once (spell_tile_global below).
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

// Chunks per lane in flight and the blocks (of 256 threads) per SM the
// registers must allow. On the 3.1 Gb graph, with each tile's sources
// prefetched to L2: 2 chunks at 5 blocks (48 registers) 0.335 ms, at 6 0.360; 1 at 6 0.346, at 8 0.387; 3
// at 5 0.354, at 4 0.346; 4 at 4 0.345. The loads wait on memory, and
// resident warps hide that wait better than more chunks per lane. Keeping
// more chunks in flight without registers, through a per-lane ring in shared
// memory filled by 4-byte cp.async copies (2 to 4 chunks ahead), ran 0.367-
// 0.383 ms; two aligned 16-byte loads per chunk instead of five 4-byte ones
// (fewer L1 wavefronts, eight words selected down to five) 0.333 ms against
// 0.325-0.328, and slower from pinned host reads too. A variant that staged each tile's input in shared memory with
// TMA bulk copies (one per piece, on an mbarrier, the next tiles' copies in
// flight while the current one was spelled) ran 0.45-1.6 ms: the smem
// buffers left too few warps resident, and the spelling itself, not the
// loads, then bounds a warp.
#ifndef CG_EMIT2_U
#define CG_EMIT2_U 2
#endif
#ifndef CG_EMIT2_MIN_BLOCKS
#define CG_EMIT2_MIN_BLOCKS 5
#endif
constexpr int kU = CG_EMIT2_U;     // interior chunks per lane in flight

// Aligned 16-byte loads may serve a piece when its stored bases, widened by
// one chunk on either side, stay inside the stream's readable words.
__device__ __forceinline__ bool aligned_ok(bool aligned16, long long src, int rc, long long plen,
                                           long long readable_words) {
  const long long low = rc ? src - plen + 1 : src, top = rc ? src : src + plen - 1;
  return aligned16 && low >= 64 && (top >> 4) + 9 < readable_words;
}

// The 64 bases whose lowest stored base is base sh / 2 of word q[0] (forward:
// in stored order; reverse complement: reversed and complemented): five
// words, four funnel shifts. Unchecked: every word must be readable.
__device__ __forceinline__ Chunk chunk_words(const uint32_t* q, unsigned sh, int rc) {
  uint32_t W[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) W[k] = __ldg(q + k);
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

// The same with every word checked against the stream (outside it: 0).
__device__ __forceinline__ Chunk chunk_at_checked(const uint32_t* words, const uint8_t* bytes, long long full_words,
                                                  long long packed_bytes, long long p, int rc) {
  const long long w0 = p >> 4;                  // floor, also for p < 0
  const unsigned sh = (unsigned)(2 * (p & 15));
  uint32_t W[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) W[k] = load_word_checked(words, bytes, full_words, packed_bytes, w0 + k);
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

// Asks L2 for the packed bytes that the pieces of output tile t (tiles of
// tile_bases bases, pieces [tile_seg[t], tile_seg[t+1]] of the walk) read:
// one bulk prefetch per piece, by the warp's lanes, rounded out to 16 bytes
// (and past the last chunk's fifth word) and kept inside the first
// readable_words words of `packed` (16-byte aligned). The tile's loads then
// find their lines in L2 or on their way instead of each waiting on DRAM in
// turn: the pieces of a tile lie at unrelated places of the read stream. On
// the 3.1 Gb graph (tiles of 32768 bases) k_emit2 went from 0.361 to 0.335
// ms with it. Prefetching the warp's next tile instead (0.441 ms), or the
// first 32 pieces of the next tile with the rest of the current one (0.435),
// was slower, and so was the same prefetch in the ASCII kernel (0.696 to
// 0.758 ms), whose time the output writes set.
__device__ __forceinline__ void prefetch_tile_sources(const Scratch& s, const uint8_t* packed,
                                                      long long readable_words, int tile_bases, long long total,
                                                      long long t, long long t_hi, int lane) {
  const int64_t* oo = s.out_off;
  const unsigned long long* ws = s.wsrc;
  const int lo = s.tile_seg[t], hi = s.tile_seg[t_hi];
  const long long tbase = t * (long long)tile_bases;
  const long long tend = min(t_hi * (long long)tile_bases, total);
  const long long top = (readable_words * 4) & ~15ll;
  for (int j = lo + lane; j <= hi; j += 32) {
    const long long oj = oo[j], oe = oo[j + 1];
    const unsigned long long w = ws[j];
    const long long a = max(oj, tbase), b = min(oe, tend);    // the piece's bases in this tile
    if (a >= b) continue;
    const int rc = (int)(w >> 63);
    const long long src = (long long)(w & ~(1ull << 63));
    const long long lo_base = rc ? src - (b - 1 - oj) : src + (a - oj);   // stored bases [lo_base, hi_base]
    const long long hi_base = rc ? src - (a - oj) : src + (b - 1 - oj);
    const long long b0 = max((lo_base >> 2) & ~15ll, 0ll);
    const long long b1 = min(((hi_base >> 2) + 32) & ~15ll, top);
    if (b1 > b0)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(packed + b0), "r"((unsigned)(b1 - b0))
                   : "memory");
  }
}

// Per-warp fields of the group of pieces being spelled.
struct PieceList {
  long long oj[32];          // output offset of each piece and of its end
  long long oe[32];
  unsigned long long w[32];
  int start[33];             // first interior chunk of each piece in the work list; [32] = the total
  long long ca[32];          // first interior chunk of each piece in the output
  bool safe[32];
};

// Spells output tile t from global memory: the tile's pieces 32 at a time, one
// per lane. The interior chunks of the 32 pieces (chunks whose 64 bases all
// lie inside one piece) form one work list in piece order, kU chunks per lane
// in flight; a lane's chunks only move forward through the list, so it finds
// each chunk's piece by stepping a cursor past the pieces it has left behind
// (no search), and the piece's address arithmetic is a few operations from
// the piece's fields in shared memory. A chunk with a piece boundary inside
// has one owner, the piece that covers its first base (the boundary is that
// piece's end): the owner's lane gathers the bits of every piece overlapping
// the chunk (reading their offsets and sources) and stores the chunk once, so
// no chunk is written twice and nothing needs an atomic. Tiles are whole
// chunks, so a chunk never spans two tiles.
__device__ void spell_tile_global(const Scratch& s, const uint8_t* packed, long long packed_bytes,
                                  long long readable_words, bool aligned16, uint4* out, int tile_bases,
                                  long long total, long long t, long long t_hi, int lane, PieceList& L) {
  const unsigned full = 0xffffffffu;
  const uint32_t* words = reinterpret_cast<const uint32_t*>(packed);
  const long long full_words = packed_bytes >> 2;
  const int64_t* oo = s.out_off;
  const unsigned long long* ws = s.wsrc;
  const int lo = s.tile_seg[t], hi = s.tile_seg[t_hi];
  const long long tbase = t * (long long)tile_bases;
  const long long tend = min(t_hi * (long long)tile_bases, total);
  for (int jb = lo; jb <= hi; jb += 32) {
    const int j = jb + lane;
    int T;
    {
      long long oj = 0, oe = 0, a = 0, b = 0;
      unsigned long long w = 0;
      if (j <= hi) {
        oj = oo[j];
        oe = oo[j + 1];
        w = ws[j];
        a = max(oj, tbase);
        b = min(oe, tend);
      }
      const long long ca = (a + 63) >> 6, cb = b >> 6;  // chunks wholly inside [a, b)
      const int n = a < b && ca < cb ? (int)(cb - ca) : 0;
      int incl = n;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += v;
      }
      T = __shfl_sync(full, incl, 31);
      L.oj[lane] = oj;
      L.oe[lane] = oe;
      L.w[lane] = w;
      L.start[lane] = incl - n;
      if (lane == 31) L.start[32] = T;
      L.ca[lane] = ca;
      L.safe[lane] = aligned_ok(aligned16, (long long)(w & ~(1ull << 63)), (int)(w >> 63), oe - oj, readable_words);
    }
    __syncwarp();
    // this lane's cursor: the piece of its next chunk, with that piece's fields
    // kept in registers until the lane's chunks move past it. Inside a piece
    // the lowest stored base of chunk f moves by 64 per chunk (up forward, down
    // reverse-complemented): its first word by 4, its shift not at all.
    int pc = -1, p_next = 0, p_rc = 0;
    unsigned p_sh = 0;
    long long p_w = 0;                                // first word of chunk f = 0 of the piece's progression
    uint4* p_o = out;                                 // chunk f goes to p_o[f]
    bool p_safe = false;
    for (int f0 = 0; f0 < T; f0 += 32 * kU) {         // warp-uniform trip count
      Chunk v[kU];
      uint4* dst[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int f = f0 + 32 * u + lane;
        dst[u] = nullptr;
        if (f < T) {
          if (f >= p_next) {                          // chunks only move forward
            do {
              ++pc;
              p_next = L.start[pc + 1];
            } while (p_next <= f);
            const int p_first = L.start[pc];
            const unsigned long long wl = L.w[pc];
            p_rc = (int)(wl >> 63);
            const long long src = (long long)(wl & ~(1ull << 63));
            const long long x_first = L.ca[pc] << 6, oj = L.oj[pc];
            // lowest stored base of the piece's first interior chunk
            const long long p0 = p_rc ? src - (x_first - oj) - 63 : src + (x_first - oj);
            p_sh = (unsigned)(2 * (p0 & 15));
            p_w = p_rc ? (p0 >> 4) + 4ll * p_first : (p0 >> 4) - 4ll * p_first;
            p_o = out + (L.ca[pc] - p_first);
            p_safe = L.safe[pc];
          }
          const long long wq = p_rc ? p_w - 4ll * f : p_w + 4ll * f;
          v[u] = p_safe ? chunk_words(words + wq, p_sh, p_rc)
                        : chunk_at_checked(words, packed, full_words, packed_bytes, (wq << 4) | (p_sh >> 1), p_rc);
          dst[u] = p_o + f;
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (dst[u] != nullptr) __stcs(dst[u], make_uint4(v[u].v[0], v[u].v[1], v[u].v[2], v[u].v[3]));
    }
    // the chunk at this piece's end, when a boundary falls inside it and this
    // piece covers its first base. Mostly the next piece covers the rest of
    // the chunk (pieces are longer than a chunk): both pieces' words are
    // loaded at once and the two parts merged under one mask. Otherwise every
    // piece overlapping the chunk adds its part in turn.
    // (this lane's piece fields come back from shared memory: registers are
    // what limits the resident warps)
    const long long oj = L.oj[lane], oe = L.oe[lane];
    const unsigned long long w = L.w[lane];
    const long long a = max(oj, tbase), b = min(oe, tend);
    long long oe_next = __shfl_down_sync(full, oe, 1);   // the next piece's end and source, from the next lane
    unsigned long long w_next = __shfl_down_sync(full, w, 1);
    if (j <= hi && a < b && (b & 63) != 0) {
      const long long x0 = ((b - 1) >> 6) << 6;
      if (a <= x0) {
        const bool last = oe >= total;                // the stream ends in this chunk, inside this piece
        if (!last && (lane == 31 || j + 1 > hi)) {
          oe_next = oo[j + 2];
          w_next = ws[j + 1];
        }
        if (last || oe_next >= x0 + 64 || oe_next >= total) {
          const int rc = (int)(w >> 63);
          const long long src = (long long)(w & ~(1ull << 63));
          Chunk va = aligned_ok(aligned16, src, rc, oe - oj, readable_words)
                         ? chunk_bits_aligned(words, x0, oj, src, rc)
                         : chunk_bits<true>(words, packed, full_words, packed_bytes, x0, oj, src, rc);
          Chunk vb;
#pragma unroll
          for (int k = 0; k < 4; ++k) vb.v[k] = 0u;
          if (!last) {
            const int rc2 = (int)(w_next >> 63);
            const long long src2 = (long long)(w_next & ~(1ull << 63));
            vb = aligned_ok(aligned16, src2, rc2, oe_next - oe, readable_words)
                     ? chunk_bits_aligned(words, x0, oe, src2, rc2)
                     : chunk_bits<true>(words, packed, full_words, packed_bytes, x0, oe, src2, rc2);
          }
          // bases [0, m) of the chunk from this piece, [m, m2) from the next
          const int m = (int)(oe - x0), m2 = last ? m : (int)(min(oe_next, x0 + 64) - x0);
          Chunk acc;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t lo_k = field_mask(0, min(max(m - 16 * k, 0), 16));
            const uint32_t hi_k = field_mask(0, min(max(m2 - 16 * k, 0), 16));
            acc.v[k] = (va.v[k] & lo_k) | (vb.v[k] & hi_k & ~lo_k);
          }
          store_chunk(out, x0 >> 6, acc);
        } else {
          Chunk acc;
#pragma unroll
          for (int k = 0; k < 4; ++k) acc.v[k] = 0u;
          long long pj = j, po = oj, pe = oe;
          unsigned long long pw = w;
          for (;;) {
            const long long lo2 = max(po, x0), hi2 = min(pe, x0 + 64);
            if (lo2 < hi2) {
              const int rc = (int)(pw >> 63);
              const long long src = (long long)(pw & ~(1ull << 63));
              Chunk v = aligned_ok(aligned16, src, rc, pe - po, readable_words)
                            ? chunk_bits_aligned(words, x0, po, src, rc)
                            : chunk_bits<true>(words, packed, full_words, packed_bytes, x0, po, src, rc);
              keep(v, x0, lo2, hi2);
#pragma unroll
              for (int k = 0; k < 4; ++k) acc.v[k] |= v.v[k];
            }
            if (pe >= x0 + 64 || pe >= total) break;        // the chunk (or the stream) ends in this piece
            ++pj;
            po = pe;
            pe = oo[pj + 1];
            pw = ws[pj];
          }
          store_chunk(out, x0 >> 6, acc);
        }
      }
    }
    __syncwarp();                                     // the group's fields are reused by the next group
  }
}

// One warp per output tile, persistent grid (spell_tile_global). Blocks of BT
// threads; the launch bounds keep CG_EMIT2_MIN_BLOCKS blocks of 256 threads'
// worth of warps resident (two blocks of 512).
template <int BT>
__global__ void __launch_bounds__(BT, BT >= 512 ? 2 : CG_EMIT2_MIN_BLOCKS * 256 / BT)
    k_emit2(Scratch s, const uint8_t* packed, long long packed_bytes, long long readable_words, bool aligned16,
            bool prefetch, uint4* out, long long cap_bytes, int tile_bases, int emit_tile, long long t_begin,
            long long t_end) {
  pdl_enter();
  __shared__ PieceList lists[BT / 32];
  const Counters* c = s.ctr;
  const long long total = *(const volatile long long*)&c->total_bases;
  const long long need = 16 * ((total + 63) / 64);
  if (need > cap_bytes) {
    if (grid_tid() == 0) set_error(s.derr, DERR_CAPACITY, K_EMIT, need);
    return;
  }
  const int lane = threadIdx.x & 31;
  const long long ntiles = (total + tile_bases - 1) / tile_bases;
  const long long t_stop = min(ntiles, t_end);          // the tiles [t_begin, t_end) of this launch
  // a warp spells `span` consecutive layout tiles at a time, spans taken as the warp frees up
  const int span = emit_span(t_stop - t_begin, grid_threads() >> 5, emit_tile, tile_bases, 2);
  const long long n_spans = (t_stop - t_begin + span - 1) / span;
  for (TileQueue q(0); q.t < n_spans; q.next(0, n_spans)) {
    q.ask(s.tickets, 0, n_spans, lane);
    const long long t = t_begin + q.t * span, t_hi = min(t + span, t_stop);
    if (prefetch) prefetch_tile_sources(s, packed, readable_words, tile_bases, total, t, t_hi, lane);
    spell_tile_global(s, packed, packed_bytes, readable_words, aligned16, out, tile_bases, total, t, t_hi, lane,
                      lists[threadIdx.x >> 5]);
  }
}

}  // namespace

namespace {

template <int BT>
cudaError_t launch_emit2_bt(const DevGraph& g, const Scratch& s, const Tuning& t, uint8_t* out, int64_t cap,
                            const LaunchEnv& env, long long t_begin, long long t_end) {
  const bool aligned16 = (reinterpret_cast<uintptr_t>(g.packed) & 15) == 0;
  // the L2 prefetch pays for HBM-resident reads only: with the reads in pinned
  // host memory it did not help (the 3.1 Gb end-to-end 2-bit step took 10.7 ms
  // with it, 9.9-10.6 ms without)
  const bool prefetch = aligned16 && !g.packed_host;
  static const int resident = resident_blocks(k_emit2<BT>, BT);   // once, safely across threads
  const int per_sm = t.emit_blocks_per_sm < resident ? t.emit_blocks_per_sm : resident;
  cudaError_t e = cudaMemsetAsync(s.tickets, 0, kTicketSets * kTicketStride * sizeof(unsigned long long), env.stream);
  if (e != cudaSuccess) return e;
  const bool chained = false;                     // a memset, not a kernel, comes right before
  return launch_kb(k_emit2<BT>, env.num_sms * per_sm, BT, env, chained, s, g.packed,
                   (long long)g.packed_bytes, (long long)(g.packed_readable / 4), aligned16, prefetch,
                   reinterpret_cast<uint4*>(out), (long long)cap, t.tile_bytes, t.emit_tile, t_begin, t_end);
}

}  // namespace

cudaError_t launch_emit2(const DevGraph& g, const Scratch& s, const Tuning& t, uint8_t* out, int64_t cap,
                         const LaunchEnv& env, long long t_begin, long long t_end) {
  cudaError_t e = t.emit_block_threads == 128 ? launch_emit2_bt<128>(g, s, t, out, cap, env, t_begin, t_end)
                  : t.emit_block_threads == 512 ? launch_emit2_bt<512>(g, s, t, out, cap, env, t_begin, t_end)
                                                : launch_emit2_bt<256>(g, s, t, out, cap, env, t_begin, t_end);
  if (e != cudaSuccess) return e;
  mark(env, "k_emit2");
  return cudaGetLastError();
}

}  // namespace cg
