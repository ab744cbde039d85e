// cg_emit.cu - spelling the contigs (LocalAssembly concatenation, Alg. 2,
// Sec. 4.4) on sm_103a.
//
// The output is one byte stream holding every contig back to back; each read
// of a contig owns one piece [out_off[j], out_off[j+1]) of it (walk position
// j). The kernel tiles the OUTPUT: the warps of a persistent grid take
// fixed-size tiles one at a time (TileQueue), and inside a tile every
// thread produces aligned 16-byte chunks, so stores are full 128-bit,
// coalesced and independent of piece lengths (a long contig spreads over many
// warps, short pieces share a chunk). Taking tiles as the warps free up rather
// than in a fixed stride lets them end together whatever each tile holds: on
// the 3.1 Gb graph 0.682 ms against 0.695.
//
// A chunk inside one piece is read with two 32-bit words of the packed
// stream and one funnel shift (16 bases); a reverse-complement piece takes
// the 16 bases below it. Four lookups in a shared-memory table turn 4 bases
// (one byte) into 4 ASCII characters; the reverse-complement table holds
// the complemented characters in reverse order (complement of b is 3-b).
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

// One warp per output tile (persistent grid; tiles from a TileQueue, its
// counters zeroed before the launch). The warp takes the pieces of its
// tile, [tile_seg[t], tile_seg[t+1]], in order; of each piece it writes the
// 16-byte-aligned interior inside the tile with full chunks, and the at most
// 30 bytes at its two ragged ends byte by byte (chunks shared by two pieces
// are thus written as disjoint bytes by each piece). Inside one piece every
// chunk starts 16 bases after the previous one, so the funnel-shift amount
// is the same for the whole piece and the packed word index moves by one per
// chunk (up for a forward piece, down for a reverse-complement one): all
// address arithmetic is done once per piece. Each chunk is two word loads,
// one funnel shift and four lookups in a shared table that maps a byte (four
// bases) to four ASCII characters, forward or reverse-complemented.
// With n_shares > 1 the launch spells share `share` of the stream cut into
// n_shares runs of whole tiles (tiles [share * T / n_shares, (share + 1) * T /
// n_shares) of the T tiles), written from out[0] on: out and cap then hold
// that share only.
template <int U, int BT>
__global__ void __launch_bounds__(BT, 1024 / BT) k_emit(Scratch s, const uint8_t* packed, long long packed_bytes,
                                                 long long readable_words, uint8_t* out, long long cap,
                                                 int tile_bytes, int emit_tile, long long t_begin, long long t_end,
                                                 int share, int n_shares) {
  __shared__ uint32_t lut[2][256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    uint32_t f = 0, r = 0;
    for (int k = 0; k < 4; ++k) {
      f |= (0x54474341u >> (8 * ((i >> (2 * k)) & 3)) & 255u) << (8 * k);             // base k -> byte k
      r |= (0x54474341u >> (8 * (3 - ((i >> (2 * (3 - k))) & 3))) & 255u) << (8 * k);  // complement of base 3-k
    }
    lut[0][i] = f;
    lut[1][i] = r;
  }
  pdl_enter();                 // the table needs nothing from the kernels before
  __syncthreads();
  const Counters* c = s.ctr;
  const long long total = *(const volatile long long*)&c->total_bases;
  const long long ntiles = (total + tile_bytes - 1) / tile_bytes;
  if (n_shares > 1) {
    t_begin = (long long)share * ntiles / n_shares;
    t_end = (long long)(share + 1) * ntiles / n_shares;
    const long long first = t_begin * tile_bytes;
    const long long bytes = max(0ll, min(total, t_end * (long long)tile_bytes) - first);
    if (bytes > cap) {
      if (grid_tid() == 0) set_error(s.derr, DERR_CAPACITY, K_EMIT, bytes);
      return;
    }
    out -= first;                                        // stream position X goes to out[X - first]
  } else if (total > cap) {
    if (grid_tid() == 0) set_error(s.derr, DERR_CAPACITY, K_EMIT, total);
    return;
  }
  const int lane = threadIdx.x & 31;
  const uint32_t* words = reinterpret_cast<const uint32_t*>(packed);
  const long long full_words = packed_bytes >> 2;
  const int64_t* oo = s.out_off;
  const unsigned long long* ws = s.wsrc;
  const long long t_stop = min(ntiles, t_end);          // the layout tiles [t_begin, t_end) of this launch
  // a warp spells `span` consecutive layout tiles at a time
  const int span = emit_span(t_stop - t_begin, grid_threads() >> 5, emit_tile, tile_bytes, 8);
  const long long n_spans = (t_stop - t_begin + span - 1) / span;
  TileQueue q(0);                                       // the warp's spans, from counters after the first
  for (; q.t < n_spans; q.next(0, n_spans)) {
    q.ask(s.tickets, 0, n_spans, lane);
    const long long t = t_begin + q.t * span, t_hi = min(t + span, t_stop);
    const int lo = s.tile_seg[t], hi = s.tile_seg[t_hi];
    const long long tbase = t * (long long)tile_bytes;
    const long long tend = min(t_hi * (long long)tile_bytes, total);
    for (int jb = lo; jb <= hi; jb += 32) {
      int jl = jb + lane;
      long long my_o = jl <= hi ? oo[jl] : 0, my_e = jl <= hi ? oo[jl + 1] : 0;
      if (jb + 31 <= hi && __all_sync(0xffffffffu, my_e == my_o)) {
        // 32 empty pieces in a row (another part's contigs, in one part's
        // layout): they all end at one offset X, and the next piece with bytes
        // is the first j >= jb + 32 with out_off[j+1] > X (offsets never
        // decrease), found by a 32-way search instead of stepping over the run
        const long long X = my_o;
        int L = jb + 32, R = hi + 1;                // the answer is in [L, R]; R = hi + 1: none
        while (R - L > 32) {
          const int step = (R - L + 31) / 32;
          const int pj = min(L + lane * step, R - 1);
          const unsigned hit = __ballot_sync(0xffffffffu, oo[pj + 1] > X);
          if (!hit) {
            L = __shfl_sync(0xffffffffu, pj, 31) + 1;
          } else {
            const int f = __ffs(hit) - 1;
            const int prev = __shfl_sync(0xffffffffu, pj, f > 0 ? f - 1 : 0);
            R = __shfl_sync(0xffffffffu, pj, f);
            if (f > 0) L = prev + 1;
          }
        }
        const unsigned hit = __ballot_sync(0xffffffffu, L + lane < R && oo[L + lane + 1] > X);
        jb = (hit ? L + __ffs(hit) - 1 : R) - 32;     // the loop step adds the 32 back
        continue;
      }
      const long long my_w = jl <= hi ? (long long)ws[jl] : 0;
      const int cnt = min(32, hi - jb + 1);
      for (int q = 0; q < cnt; ++q) {
        const long long oj = shfl64(my_o, q), oe = shfl64(my_e, q);
        const unsigned long long w = (unsigned long long)shfl64(my_w, q);
        const long long a = max(oj, tbase), b = min(oe, tend);   // the piece's bytes in this tile
        if (a >= b) continue;
        const long long A = (a + 15) & ~15ll, B = b & ~15ll;     // aligned interior [A, B)
        if (A < B) {
          const int rc = (int)(w >> 63);
          const long long src = (long long)(w & ~(1ull << 63));
          const long long p0 = rc ? src - (A - oj) - 15 : src + (A - oj);   // lowest stored base of chunk 0
          const unsigned sh = (unsigned)(2 * (p0 & 15));
          const int nch = (int)((B - A) >> 4);
          const long long w0 = p0 >> 4;
          const long long wmax = rc ? w0 + 1 : w0 + nch;             // highest word the piece reads
          const uint32_t* tab = lut[rc];
          uint4* dst = reinterpret_cast<uint4*>(out + A);
          if (wmax < readable_words) {
            const int step = rc ? -1 : 1;
            const uint32_t* wp = words + w0;
            for (int c0 = lane; c0 < nch; c0 += 32 * U) {
              uint32_t lo4[U], hi4[U];
#pragma unroll
              for (int u = 0; u < U; ++u) {
                const int ci = c0 + 32 * u;
                const int wi = ci < nch ? ci * step : 0;
                lo4[u] = __ldg(wp + wi);
                hi4[u] = __ldg(wp + wi + 1);
              }
#pragma unroll
              for (int u = 0; u < U; ++u) {
                const int ci = c0 + 32 * u;
                if (ci >= nch) continue;
                const uint32_t bits = __funnelshift_r(lo4[u], hi4[u], sh);
                uint4 v;
                if (rc) {
                  v = make_uint4(tab[bits >> 24], tab[(bits >> 16) & 255u], tab[(bits >> 8) & 255u], tab[bits & 255u]);
                } else {
                  v = make_uint4(tab[bits & 255u], tab[(bits >> 8) & 255u], tab[(bits >> 16) & 255u], tab[bits >> 24]);
                }
                __stcs(dst + ci, v);
              }
            }
          } else {                                                     // piece ends at the stream's end
            for (int ci = lane; ci < nch; ci += 32) {
              const long long wi = rc ? w0 - ci : w0 + ci;
              const uint32_t bits = __funnelshift_r(load_word(words, packed, full_words, packed_bytes, wi),
                                                    load_word(words, packed, full_words, packed_bytes, wi + 1), sh);
              const uint4 v = rc ? make_uint4(tab[bits >> 24], tab[(bits >> 16) & 255u], tab[(bits >> 8) & 255u],
                                              tab[bits & 255u])
                                 : make_uint4(tab[bits & 255u], tab[(bits >> 8) & 255u], tab[(bits >> 16) & 255u],
                                              tab[bits >> 24]);
              __stcs(dst + ci, v);
            }
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

namespace {

// One block size: a persistent grid of at most the blocks that can be resident
// at once (the function-local static is initialised once, safely across threads).
template <int BT>
cudaError_t launch_emit_bt(const DevGraph& g, const Scratch& s, const Tuning& t, uint8_t* out, int64_t cap,
                           const LaunchEnv& env, long long t_begin, long long t_end, int share, int n_shares) {
  static const int resident = resident_blocks(k_emit<4, BT>, BT);
  const int per_sm = t.emit_blocks_per_sm < resident ? t.emit_blocks_per_sm : resident;
  cudaError_t e = cudaMemsetAsync(s.tickets, 0, kTicketSets * kTicketStride * sizeof(unsigned long long), env.stream);
  if (e != cudaSuccess) return e;
  const bool chained = false;                     // a memset, not a kernel, comes right before
  return launch_kb(k_emit<4, BT>, env.num_sms * per_sm, BT, env, chained, s, g.packed,
                   (long long)g.packed_bytes, (long long)(g.packed_readable / 4), out, (long long)cap, t.tile_bytes,
                   t.emit_tile, t_begin, t_end, share, n_shares);
}

}  // namespace

cudaError_t launch_emit(const DevGraph& g, const Scratch& s, const Tuning& t, uint8_t* out, int64_t cap,
                        const LaunchEnv& env, long long t_begin, long long t_end, int share, int n_shares) {
  cudaError_t e = t.emit_block_threads == 128
                      ? launch_emit_bt<128>(g, s, t, out, cap, env, t_begin, t_end, share, n_shares)
                  : t.emit_block_threads == 512
                      ? launch_emit_bt<512>(g, s, t, out, cap, env, t_begin, t_end, share, n_shares)
                      : launch_emit_bt<256>(g, s, t, out, cap, env, t_begin, t_end, share, n_shares);
  if (e != cudaSuccess) return e;
  mark(env, "k_emit");
  return cudaGetLastError();
}

}  // namespace cg
