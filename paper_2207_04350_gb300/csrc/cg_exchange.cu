// cg_exchange.cu - the read exchange of a run split over ranks that each hold
// only a slice of the reads (the paper's read exchange, Sec. 4.3), on sm_103a.
//
// Every rank lays out the whole graph (mask, chains, offsets) without the
// reads, so every rank knows every piece: its read, its stored range in a
// virtual 2-bit stream (the graph's `off`), and its place in the output. The
// output is cut into equal runs of output tiles, one per rank (the shares of
// cg_emit_share). Rank r owns reads [rf[r], rf[r+1]) and holds their bases in
// a stream of its own layout. For every share p, the pieces of p's range whose
// reads r owns go, in walk order, into r's segment for p: each as the 32-bit
// words covering its stored range in the virtual stream (word W0 = its lowest
// base / 16, through its highest base / 16 + 1), realigned on the way from r's
// own layout, so the receiver needs nothing but the virtual offsets. The
// receiver, its segments laid end to end by source rank (as an all-to-all
// delivers them), moves every piece's source into its buffer and spells its
// share from there.
#include <cuda_runtime.h>

#include "cg_internal.cuh"
#include "cg_lookback.cuh"

namespace cg {

namespace {

// The rank r with rf[r] <= v < rf[r + 1].
__device__ __forceinline__ int owner_of(const int64_t* rf, int n, long long v) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (rf[mid] <= v) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

struct XPiece {
  long long W0;      // first virtual word sent
  long long words;   // words sent (0 for an empty piece)
  int owner;
};

__device__ __forceinline__ XPiece x_piece(const Scratch& s, const XchgArgs& x, long long j) {
  XPiece p;
  p.owner = owner_of(x.rf, x.n_shares, s.wread[j]);
  const long long L = s.wlen[j];
  if (L <= 0) {
    p.W0 = 0;
    p.words = 0;
    return p;
  }
  const unsigned long long w = s.wsrc[j];
  const long long src = (long long)(w & ~(1ull << 63));
  const int rc = (int)(w >> 63);
  const long long lo = rc ? src - L + 1 : src, hi = rc ? src : src + L - 1;
  p.W0 = lo >> 4;
  p.words = (hi >> 4) + 2 - p.W0;              // words W0 .. hi / 16 + 1: the spelling's two-word windows
  return p;
}

// The share of pair i (pairs are the shares' ranges laid end to end).
__device__ __forceinline__ int share_of_pair(const XchgArgs& x, long long i) {
  int lo = 0, hi = x.n_shares - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (x.pair0[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_x_ranges(Scratch s, int n_shares, int tile_bytes, long long* range) {
  const int p = (int)grid_tid();
  if (p >= n_shares) return;
  const long long total = *(const volatile long long*)&s.ctr->total_bases;
  const long long T = (total + tile_bytes - 1) / tile_bytes;
  const long long t0 = (long long)p * T / n_shares, t1 = (long long)(p + 1) * T / n_shares;
  if (t0 >= t1) {
    range[2 * p] = 1;
    range[2 * p + 1] = 0;
  } else {
    range[2 * p] = s.tile_seg[t0];
    range[2 * p + 1] = s.tile_seg[t1];
  }
}

// Words to each share (send) and from each rank (recv), summed per warp over
// the lanes with the same share or owner before one atomic each.
__global__ void k_x_sizes(Scratch s, XchgArgs x, unsigned long long* send_words, unsigned long long* recv_words,
                          long long n_pairs) {
  const long long T = grid_threads();
  const long long n_iter = (n_pairs + T - 1) / T * T;  // whole warps iterate together
  for (long long i = grid_tid(); i < n_iter; i += T) {
    int p = -1, owner = -1;
    unsigned long long words = 0;
    if (i < n_pairs) {
      p = share_of_pair(x, i);
      const long long j = x.range[2 * p] + (i - x.pair0[p]);
      const XPiece q = x_piece(s, x, j);
      owner = q.owner;
      words = (unsigned long long)q.words;
    }
    {
      const int key = owner == x.rank ? p : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      unsigned long long sum = 0;
      for (unsigned m = peers; m; m &= m - 1) sum += __shfl_sync(peers, words, __ffs(m) - 1);
      if (key >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&send_words[key], sum);
    }
    {
      const int key = p == x.rank ? owner : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      unsigned long long sum = 0;
      for (unsigned m = peers; m; m &= m - 1) sum += __shfl_sync(peers, words, __ffs(m) - 1);
      if (key >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&recv_words[key], sum);
    }
  }
}

// Scan loads: the words of a piece of one share's range when its owner is `who`.
struct XLoad {
  Scratch s;
  XchgArgs x;
  long long j0;
  int who;
  __device__ unsigned long long operator()(long long i) const {
    const XPiece q = x_piece(s, x, j0 + i);
    return q.owner == who ? (unsigned long long)q.words : 0ull;
  }
};
struct XStore {
  Scratch s;
  XchgArgs x;
  long long j0;
  int who;
  long long* slot;              // slot[i] for the items owned by `who`
  __device__ void item(long long i, unsigned long long e) const {
    if (x_piece(s, x, j0 + i).owner == who) slot[i] = (long long)e;
  }
  __device__ void last(long long, unsigned long long) const {}
};

// Scan over all pairs (the shares' ranges end to end): the words of the
// pieces this rank owns; every pair gets its exclusive prefix, so that a
// piece's offset in its share's segment is its prefix less the prefix at the
// share's first pair.
struct XPairLoad {
  Scratch s;
  XchgArgs x;
  __device__ unsigned long long operator()(long long i) const {
    const int p = share_of_pair(x, i);
    const XPiece q = x_piece(s, x, x.range[2 * p] + (i - x.pair0[p]));
    return q.owner == x.rank ? (unsigned long long)q.words : 0ull;
  }
};
struct XPairStore {
  long long* slot;
  __device__ void item(long long i, unsigned long long e) const { slot[i] = (long long)e; }
  __device__ void last(long long, unsigned long long) const {}
};

__device__ __forceinline__ uint32_t word_checked(const uint32_t* words, const uint8_t* bytes, long long n_bytes,
                                                 long long w) {
  if (w < 0) return 0u;
  if (4 * w + 4 <= n_bytes) return __ldg(words + w);
  uint32_t r = 0;
  for (int b = 0; b < 4; ++b) {
    const long long i = 4 * w + b;
    if (i < n_bytes) r |= (uint32_t)__ldg(bytes + i) << (8 * b);
  }
  return r;
}

// One warp per pair this rank owns: the piece's virtual words W0 .. W0 +
// words - 1, each built from the rank's own stream (read v's bases start at
// my_off[v - rf[rank]] there and at off[v] in the virtual stream) with one
// funnel shift; words outside the rank's stream read as 0.
__global__ void k_x_pack(DevGraph g, Scratch s, XchgArgs x, const uint8_t* my_packed, long long my_bytes,
                         const int64_t* my_off, const long long* seg, const long long* slot, uint32_t* send,
                         long long n_pairs) {
  const int lane = threadIdx.x & 31;
  const uint32_t* mw = reinterpret_cast<const uint32_t*>(my_packed);
  const long long my_first = x.rf[x.rank];
  for (long long i = grid_tid() >> 5; i < n_pairs; i += grid_threads() >> 5) {
    const int p = share_of_pair(x, i);
    const long long j = x.range[2 * p] + (i - x.pair0[p]);
    const XPiece q = x_piece(s, x, j);
    if (q.owner != x.rank || q.words == 0) continue;        // uniform across the warp
    const long long v = s.wread[j];
    const long long delta = my_off[v - my_first] - g.off[v];
    uint32_t* dst = send + seg[p] + (slot[i] - slot[x.pair0[p]]);
    for (long long k = lane; k < q.words; k += 32) {
      const long long b = 16 * (q.W0 + k) + delta;          // the word's first base in this rank's stream
      const long long w = b >> 4;                            // floor, also below 0
      const unsigned sh = (unsigned)(2 * (b & 15));
      dst[k] = __funnelshift_r(word_checked(mw, my_packed, my_bytes, w), word_checked(mw, my_packed, my_bytes, w + 1),
                               sh);
    }
  }
}

// The receiver: every piece of its range, its source moved into the receive
// buffer (16 bases per word, the piece's phase within its first word kept).
__global__ void k_x_rewrite(Scratch s, XchgArgs x, const long long* seg, const long long* slot) {
  const long long j0 = x.range[2 * x.rank], j1 = x.range[2 * x.rank + 1];
  for (long long i = grid_tid(); j0 + i <= j1; i += grid_threads()) {
    const long long j = j0 + i;
    const XPiece q = x_piece(s, x, j);
    if (q.words == 0) continue;
    const unsigned long long w = s.wsrc[j];
    const long long src = (long long)(w & ~(1ull << 63));
    const long long at = 16 * (seg[q.owner] + slot[i]) + (src - 16 * q.W0);
    s.wsrc[j] = (unsigned long long)at | (w & (1ull << 63));
  }
}

}  // namespace

cudaError_t launch_x_ranges(const Scratch& s, int n_shares, int tile_bytes, long long* range, const LaunchEnv& env) {
  k_x_ranges<<<(n_shares + kBlock - 1) / kBlock, kBlock, 0, env.stream>>>(s, n_shares, tile_bytes, range);
  mark(env, "k_x_ranges");
  return cudaGetLastError();
}

cudaError_t launch_x_sizes(const Scratch& s, const XchgArgs& x, unsigned long long* send_words,
                           unsigned long long* recv_words, long long n_pairs, const LaunchEnv& env) {
  cudaMemsetAsync(send_words, 0, (size_t)x.n_shares * 8, env.stream);
  cudaMemsetAsync(recv_words, 0, (size_t)x.n_shares * 8, env.stream);
  if (n_pairs > 0) {
    k_x_sizes<<<grid_for(n_pairs, env), kBlock, 0, env.stream>>>(s, x, send_words, recv_words, n_pairs);
    mark(env, "k_x_sizes");
  }
  return cudaGetLastError();
}

cudaError_t launch_x_pack(const DevGraph& g, const Scratch& s, const XchgArgs& x, const uint8_t* my_packed,
                          long long my_bytes, const int64_t* my_off, const long long* seg, const long long* slot,
                          uint32_t* send, long long n_pairs, const LaunchEnv& env) {
  if (n_pairs <= 0) return cudaSuccess;
  k_x_pack<<<grid_for(32 * n_pairs, env), kBlock, 0, env.stream>>>(g, s, x, my_packed, my_bytes, my_off, seg, slot,
                                                                     send, n_pairs);
  mark(env, "k_x_pack");
  return cudaGetLastError();
}

cudaError_t launch_x_rewrite(const Scratch& s, const XchgArgs& x, const long long* seg, const long long* slot,
                             const LaunchEnv& env) {
  k_x_rewrite<<<env.num_sms * 4, kBlock, 0, env.stream>>>(s, x, seg, slot);
  mark(env, "k_x_rewrite");
  return cudaGetLastError();
}

cudaError_t launch_x_scan_pairs(const Scratch& s, const XchgArgs& x, long long n_pairs, long long* slot,
                                unsigned long long* state, long long state_cap, const LaunchEnv& env) {
  if (n_pairs <= 0) return cudaSuccess;
  const long long tiles = (n_pairs + kTileItems - 1) / kTileItems;
  if (tiles > state_cap) return cudaErrorInvalidValue;
  cudaMemsetAsync(state, 0, (size_t)(state_cap + 1) * sizeof(unsigned long long), env.stream);
  k_scan<<<scan_grid(tiles, env), kBlock, 0, env.stream>>>(XPairLoad{s, x}, XPairStore{slot}, n_pairs, nullptr, state,
                                                           state_cap, s.derr, (int)K_SCAN_OFFSETS);
  mark(env, "k_scan_exchange_pairs");
  return cudaGetLastError();
}

// One exclusive scan over a share's range [j0, j0 + count): the word offset,
// among the pieces owned by `who`, of each piece owned by `who`.
cudaError_t launch_x_scan(const Scratch& s, const XchgArgs& x, long long j0, long long count, int who,
                          long long* slot, unsigned long long* state, long long state_cap, const LaunchEnv& env) {
  if (count <= 0) return cudaSuccess;
  const long long tiles = (count + kTileItems - 1) / kTileItems;
  if (tiles > state_cap) return cudaErrorInvalidValue;
  cudaMemsetAsync(state, 0, (size_t)(state_cap + 1) * sizeof(unsigned long long), env.stream);
  k_scan<<<scan_grid(tiles, env), kBlock, 0, env.stream>>>(XLoad{s, x, j0, who}, XStore{s, x, j0, who, slot}, count,
                                                           nullptr, state, state_cap, s.derr, (int)K_SCAN_OFFSETS);
  mark(env, "k_scan_exchange");
  return cudaGetLastError();
}

}  // namespace cg
