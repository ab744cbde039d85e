// cg_batch.cu - the batched form: many string graphs loaded as one disjoint
// union, so that every stage is one launch over all graphs' reads and pieces.
// Components never cross graphs and contigs are listed by smallest read id,
// so graph j's contigs are one contiguous run of the union's output.
#include <cuda_runtime.h>

#include "cg_internal.cuh"

namespace cg {

namespace {

__device__ __forceinline__ int graph_of(const int64_t* table, int k, long long x) {   // last j with table[j] <= x
  int a = 0, b = k - 1;
  while (a < b) {
    int mid = (a + b + 1) >> 1;
    if (table[mid] <= x) a = mid; else b = mid - 1;
  }
  return a;
}

// Union CSR: row_ptr[r] = graph's own row_ptr + its first entry; columns
// shifted by the graph's first read; base offsets by its packed start.
__global__ void k_batch_fixup(int k, const int64_t* R, const int64_t* E, const int64_t* PB, const int64_t* SR,
                              const void* stage_rp, int rp_bytes, int64_t* rp, int32_t* col, int64_t* off, long long N,
                              long long M) {
  for (long long r = grid_tid(); r < N; r += grid_threads()) {
    const int j = graph_of(R, k, r);
    const long long i = SR[j] + (r - R[j]);
    const long long v = rp_bytes == 8 ? reinterpret_cast<const int64_t*>(stage_rp)[i]
                                      : (long long)reinterpret_cast<const int32_t*>(stage_rp)[i];
    rp[r] = v + E[j];
    off[r] += 4 * PB[j];
  }
  for (long long e = grid_tid(); e < M; e += grid_threads()) col[e] += (int32_t)R[graph_of(E, k, e)];
  if (grid_tid() == 0) rp[N] = M;
}

// The input arrays of a batch's graphs into the union's arrays, read in place
// from pinned host memory (one launch instead of a copy call per graph and
// array): a warp per segment, four 16-byte loads per lane in flight when both
// ends are 16-byte aligned, else 4-byte words, else bytes.
__global__ void __launch_bounds__(kBlock) k_batch_copy(const CopySeg* __restrict__ seg, int n) {
  const int lane = threadIdx.x & 31;
  for (long long w = grid_tid() >> 5; w < n; w += grid_threads() >> 5) {
    const CopySeg sg = seg[w];
    const uintptr_t align = reinterpret_cast<uintptr_t>(sg.src) | reinterpret_cast<uintptr_t>(sg.dst);
    long long done = 0;
    if ((align & 15) == 0) {
      const uint4* __restrict__ src = reinterpret_cast<const uint4*>(sg.src);
      uint4* __restrict__ dst = reinterpret_cast<uint4*>(sg.dst);
      const long long n16 = sg.bytes >> 4;
      long long i = lane;
      for (; i + 96 < n16; i += 128) {
        const uint4 a = src[i], b = src[i + 32], c = src[i + 64], d = src[i + 96];
        dst[i] = a;
        dst[i + 32] = b;
        dst[i + 64] = c;
        dst[i + 96] = d;
      }
      for (; i < n16; i += 32) dst[i] = src[i];
      done = n16 << 4;
    } else if ((align & 3) == 0) {
      const uint32_t* __restrict__ src = reinterpret_cast<const uint32_t*>(sg.src);
      uint32_t* __restrict__ dst = reinterpret_cast<uint32_t*>(sg.dst);
      const long long n4 = sg.bytes >> 2;
      for (long long i = lane; i < n4; i += 32) dst[i] = src[i];
      done = n4 << 2;
    }
    for (long long i = done + lane; i < sg.bytes; i += 32) sg.dst[i] = sg.src[i];
  }
}

// First contig and first output base of every graph of the batch (and the
// totals at index k): heads before the graph's first read.
__global__ void k_batch_ranges(Scratch s, int k, const int64_t* R, long long N, int64_t* first_contig,
                               int64_t* first_base) {
  const Counters* c = s.ctr;
  for (long long j = grid_tid(); j <= k; j += grid_threads()) {
    const long long r = R[j];
    long long ci;
    if (r >= N) {
      ci = c->n_contigs;
    } else {
      const unsigned word = s.hb[r >> 5];
      ci = (long long)s.wp[r >> 5] + __popc(word & ((1u << (r & 31)) - 1u));
    }
    if (first_contig) first_contig[j] = ci;
    if (first_base) first_base[j] = s.contig_off[ci];
  }
}

}  // namespace

cudaError_t launch_batch_copy(const CopySeg* seg, int n, const LaunchEnv& env) {
  if (n <= 0) return cudaSuccess;
  static const int resident = resident_blocks(k_batch_copy);   // once, safely across threads
  const long long want = ((long long)n + kBlock / 32 - 1) / (kBlock / 32);
  const long long cap = (long long)env.num_sms * resident;
  k_batch_copy<<<(unsigned)(want < cap ? want : cap), kBlock, 0, env.stream>>>(seg, n);
  mark(env, "k_batch_copy");
  return cudaGetLastError();
}

cudaError_t launch_batch_fixup(int k, const int64_t* R, const int64_t* E, const int64_t* PB, const int64_t* SR,
                               const void* stage_rp, int rp_bytes, int64_t* rp, int32_t* col, int64_t* off,
                               long long N, long long M, const LaunchEnv& env) {
  k_batch_fixup<<<grid_for(N > M ? N : M, env), kBlock, 0, env.stream>>>(k, R, E, PB, SR, stage_rp, rp_bytes, rp,
                                                                         col, off, N, M);
  mark(env, "k_batch_fixup");
  return cudaGetLastError();
}

cudaError_t launch_batch_ranges(const Scratch& s, int k, const int64_t* R, long long N, int64_t* first_contig,
                                int64_t* first_base, const LaunchEnv& env) {
  k_batch_ranges<<<grid_for(k + 1, env), kBlock, 0, env.stream>>>(s, k, R, N, first_contig, first_base);
  mark(env, "k_batch_ranges");
  return cudaGetLastError();
}

}  // namespace cg

// ------------------------------------------------------------------------
// Batches whose reads stay in pinned host memory (CG_HOST_READS): the union
// keeps the virtual layout of the concatenated read streams (graph j's bytes
// at [PB[j], PB[j+1]), 16-byte aligned) without holding it. After the
// offsets stage every piece's words are gathered from its own graph's host
// stream into one device buffer, slot after slot, and the piece's source is
// rewritten into that buffer; the spelling kernels then run unchanged.
#include "cg_lookback.cuh"

namespace cg {

namespace {

// Words [lo >> 4, (hi >> 4) + 1] of a piece of stored bases [lo, hi]: the
// spelling reads the word after the last one for its funnel shifts.
__device__ __forceinline__ void piece_words(unsigned long long w, int32_t len, long long* w0, long long* nw) {
  const long long first = (long long)(w & ~(1ull << 63));
  const bool rc = (w >> 63) != 0;
  const long long lo = rc ? first - len + 1 : first, hi = rc ? first : first + len - 1;
  *w0 = lo >> 4;
  *nw = len > 0 ? (hi >> 4) - (lo >> 4) + 2 : 0;
}

struct SlotLoad {
  const unsigned long long* wsrc;
  const int32_t* wlen;
  __device__ unsigned long long operator()(long long j) const {
    long long w0, nw;
    piece_words(wsrc[j], wlen[j], &w0, &nw);
    return (unsigned long long)nw;
  }
};
struct SlotStore {
  unsigned long long* slot;
  __device__ void item(long long j, unsigned long long e) const { slot[j] = e; }
  __device__ void last(long long n, unsigned long long t) const { slot[n] = t; }
};

// One warp per piece: the graph holding its first word, the words copied
// with that graph's bounds (words past its stream read as 0), the source
// moved into the slot.
// With t_end > 0 only the pieces that output tiles [t_begin, t_end) need and
// that no earlier range took: (tile_seg[t_begin], tile_seg[t_end]] (from
// piece 0 when t_begin is 0), each piece once, as its source is moved.
__global__ void __launch_bounds__(kBlock) k_gather_pieces(Scratch s, int k, const int64_t* PB,
                                                          const uint8_t* const* base, const int64_t* bytes,
                                                          const unsigned long long* slot, uint32_t* dst,
                                                          long long cap_words, long long t_begin, long long t_end) {
  long long j_begin = 0, W = *(const volatile unsigned*)&s.ctr->n_walk;
  if (t_end > 0) {
    const long long nt = *(const volatile unsigned*)&s.ctr->n_tiles;
    j_begin = t_begin > 0 ? (long long)s.tile_seg[min(t_begin, nt)] + 1 : 0;
    W = min(W, (long long)s.tile_seg[min(t_end, nt)] + 1);
  }
  const int lane = threadIdx.x & 31;
  for (long long j = j_begin + (grid_tid() >> 5); j < W; j += grid_threads() >> 5) {
    const unsigned long long w = s.wsrc[j];
    long long w0, nw;
    piece_words(w, s.wlen[j], &w0, &nw);
    const long long o = (long long)slot[j];
    if (o + nw > cap_words) {
      if (lane == 0) set_error(s.derr, DERR_KERNEL, K_BATCH_GATHER, j);
      continue;
    }
    if (nw > 0) {
      const int g = graph_of(PB, k, 4 * w0);                 // the graph of the piece's first byte
      const long long gw0 = w0 - PB[g] / 4;                  // its first word in that graph's stream
      const long long gbytes = bytes[g];
      const uint8_t* src = base[g];
      for (long long t = lane; t < nw; t += 32) {
        const long long x = gw0 + t;
        uint32_t v = 0;
        if (4 * x + 4 <= gbytes) {
          v = *reinterpret_cast<const uint32_t*>(src + 4 * x);
        } else {
          for (int b = 0; b < 4; ++b)
            if (4 * x + b < gbytes) v |= (uint32_t)src[4 * x + b] << (8 * b);
        }
        dst[o + t] = v;
      }
    }
    if (lane == 0) {
      const long long first = (long long)(w & ~(1ull << 63)) + 16 * (o - w0);
      s.wsrc[j] = (unsigned long long)first | (w & (1ull << 63));
    }
  }
}

}  // namespace

cudaError_t launch_gather_slots(const Scratch& s, long long W, unsigned long long* slot, unsigned long long* state,
                                long long state_cap, const LaunchEnv& env) {
  const long long tiles = (W + kTileItems - 1) / kTileItems;
  if (tiles > state_cap) return cudaErrorInvalidValue;
  cudaMemsetAsync(state, 0, (size_t)(state_cap + 1) * sizeof(unsigned long long), env.stream);
  if (W > 0) {
    k_scan<<<scan_grid(tiles, env), kBlock, 0, env.stream>>>(SlotLoad{s.wsrc, s.wlen}, SlotStore{slot}, W, nullptr, state,
                                                       state_cap, s.derr, K_BATCH_GATHER);
    mark(env, "k_scan_slots");
  } else {
    cudaMemsetAsync(slot, 0, sizeof(unsigned long long), env.stream);
  }
  return cudaGetLastError();
}

cudaError_t launch_gather_pieces(const Scratch& s, int k, const int64_t* PB, const uint8_t* const* base,
                                 const int64_t* bytes, const unsigned long long* slot, uint32_t* dst,
                                 long long cap_words, long long W, const LaunchEnv& env, long long t_begin,
                                 long long t_end) {
  k_gather_pieces<<<grid_for(32 * (W > 0 ? W : 1), env), kBlock, 0, env.stream>>>(s, k, PB, base, bytes, slot, dst,
                                                                                 cap_words, t_begin, t_end);
  mark(env, "k_gather_pieces");
  return cudaGetLastError();
}

}  // namespace cg
