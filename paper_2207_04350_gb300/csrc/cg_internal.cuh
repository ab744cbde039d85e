// cg_internal.cuh - device data layout and kernel launchers shared by the
// translation units of the contig-generation library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace cg {

constexpr int kBlock = 256;

// First device-side error wins (atomicCAS from 0).
enum : int32_t {
  DERR_NONE = 0,
  DERR_GRAPH = 1,     // input check failed
  DERR_TIMEOUT = 2,   // a bounded wait gave up
  DERR_KERNEL = 3,    // an internal consistency check failed
  DERR_CAPACITY = 4   // an output buffer is too small
};

// Device-side error word of a context: the first error a kernel finds stays
// until the host reads and clears it.
// Per-graph counters of one run: each stage zeroes its own part.
struct DevError {
  int err;                     // DERR_*
  int where;                   // kernel id of the first error
  long long index;             // element index of the first error
};

struct Counters {
  // mask stage
  unsigned long long n_branch;
  unsigned int n_cand;         // unmasked reads with at least one overlap
  unsigned int n_lone;         // reads without overlaps spelled as one-read contigs (min_chain <= 1)
  // chain stage
  unsigned int n_rulers;       // sublist starts of the list ranking
  unsigned int n_hlist;        // sublists that start a list
  unsigned int n_cycle_reads;  // reads on closed chains
  unsigned int n_cycles;
  unsigned int n_heads;        // contigs found by the chain stage
  unsigned int need_jump;      // a list had more sublists than the list walk follows
  unsigned int final_buf;      // which pointer-jumping buffer holds the result
  unsigned int bar_count;      // grid barrier arrival counter
  unsigned int bar_gen;        // grid barrier generation
  unsigned int round_flag[64]; // "some pointer still moves" per jumping round
  // offsets stage
  unsigned int n_contigs;
  unsigned int n_walk;         // walk positions = reads spelled
  unsigned int n_tiles;        // emission tiles
  unsigned int pad;
  long long total_bases;
};

// The graph as kernels see it (all device pointers).
struct DevGraph {
  int64_t n, m;
  const void* row_ptr;
  int rp64;                    // 1: int64 row_ptr, 0: int32
  int min_chain;               // >= 1
  const int32_t* col;
  const uint8_t* code;
  const int32_t* suf;          // suffix form, or
  const int32_t* pre;          // x-drop form (Sec. 4.4): pre and post per entry, nullptr in the suffix form
  const int32_t* post;
  const int32_t* len;
  const int64_t* off;
  const uint8_t* packed;
  int64_t packed_bytes;
  int64_t packed_readable;     // bytes of `packed` that may be read (>= packed_bytes: padding of owned copies)
  bool packed_host = false;    // `packed` is pinned host memory read in place over the host link
  bool no_reads = false;       // loaded without its reads: `off` places reads in a virtual stream
};

// Scratch owned by a loaded graph. Sizes in elements (n reads).
struct Scratch {
  uint8_t* branch;      // n
  int32_t* cand;        // n: candidate reads (unmasked, with overlaps), in candidate order
  int32_t* cidx;        // n: per read with overlaps, its candidate index, -1 for a branch read
  int32_t* lone;        // n: reads without overlaps spelled alone
  unsigned* hb_mask;    // n/32+1: heads bitmap words of the mask stage
  unsigned* hb;         // n/32+1: bit m set when read m is the smallest read of a contig
  // The chain stage indexes candidates, c = cidx[v], and their oriented
  // copies u = 2c + o: its records sit together in candidate order instead
  // of spreading over arrays of n reads.
  int4* succ;           // n: (successor of (c,fwd), successor of (c,rc) as oriented candidates, or -1; read id;
                        //     the sublist (c,fwd) starts, when it starts one)
  int32_t* sufin;       // 2n: suffix (x-drop form: post) of the overlap entering oriented candidate u
  int32_t* preout;      // 2n, x-drop form only: pre of the overlap leaving oriented candidate u
  int32_t* pfirst;      // n, x-drop form only: per candidate, stored index of the piece's first base
  // Records read together sit together: one sector per random access.
  int2* rr;             // 2n: oriented candidate u -> (sublist, -1 when not reached; position inside it);
                        //     rr[2c] and rr[2c+1] form one 16-byte record
  // sublists (capacity 2n)
  int32_t* rlist;       // first oriented candidate of each sublist
  int32_t* hlist;       // sublists that start a list
  int4* rec;            // sublist -> (the next sublist, -1 at the list end;
                        //             length; smallest read id inside; last oriented read, 2v + o)
  int4* pj[2];          // sublist -> (next: -1 resolved, -2 unresolved; oriented reads to the list tail;
                        //             smallest read id to the tail; the list's last oriented read);
                        //             jumping double buffers
  // per candidate
  int4* prd;            // n: (smallest read id of the chain, -1 in no contig; walk position;
                        //     bases this read adds to its contig; orientation 0 / 1, 255 in no contig)
  int32_t* headq;       // per read, at a contig's smallest read: its number of reads
  // closed chains (oriented candidates)
  int32_t* cyc;         // n: candidates on closed chains
  int32_t* c_ptr[2];    // 2n
  long long* c_val[2];  // 2n: (2v + o) << 32 | u while finding each cycle's smallest read, then distances
  int32_t* c_head;      // 2n
  // contig order and walk order
  unsigned* wp;         // n/32+1: heads before each bitmap word
  int32_t* qd;          // n: reads per contig, in contig order
  unsigned long long* cbase; // n+1: first walk position of each contig
  unsigned long long* wsrc;  // n: first stored base of the piece | reverse flag << 63
  int32_t* wlen;        // n: piece length
  int64_t* out_off;     // n+1
  int32_t* wfirst;      // n: per walk position, the contig whose first read it holds, or -1
  int32_t* wread;       // n, graphs loaded without their reads only: the read at each walk position
  int64_t* contig_off;  // n+1
  int32_t* tile_seg;    // tiles_cap+1: walk position holding the first byte of each emission tile
  int64_t tiles_cap;
  // one part's layout (Sec. 4.3): when part is set, the reads of a contig c with
  // part[c] != part_p add no bases, so the layout holds that part's contigs only
  const int32_t* part;  // n_contigs, or nullptr for the whole layout
  int32_t part_p;
  unsigned long long* scan_state[3];  // look-back tile descriptors (+1 ticket word) of the three scans
  int64_t scan_tiles_cap;
  Counters* ctr;
  DevError* derr;
  unsigned long long* tickets;  // kTicketSets counters, one 128-byte line each: a spelling launch's tiles
};

// Output tiles [t_begin, t_stop) for the W warps of a persistent grid: warp gw
// spells tile t_begin + gw first; the tiles from t_begin + W on go out one at a
// time, the tiles t_begin + W + c + kTicketSets * k from counter c (zeroed
// before the launch) to the warps gw = c mod kTicketSets, each warp asking for
// its next ticket while it spells its current tile. A warp thus takes its next
// tile when it finishes one, and the warps end together whatever each tile
// holds; no launch starts with every warp on one counter, and a launch with no
// more tiles than warps touches no counter.
constexpr int kTicketSets = 8, kTicketStride = 16;

struct TileQueue {
  long long t;                 // the warp's current tile (past t_stop: done)
  unsigned long long tk;
  __device__ static long long warp_id() {
    return (long long)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
  }
  __device__ static long long warps() { return (long long)gridDim.x * (blockDim.x >> 5); }
  __device__ TileQueue(long long t_begin) : t(t_begin + warp_id()), tk(0) {}
  // The warp's current tile is t while t < t_stop; call ask() as the tile is
  // started and next() when it is done (warp-uniform calls, with the launch's
  // counters and tile range; the queue keeps no copy, to spare registers). A
  // grid with no fewer warps than tiles takes no ticket.
  __device__ void ask(unsigned long long* tickets, long long t_begin, long long t_stop, int lane) {
    if (t_begin + warps() < t_stop && lane == 0)
      tk = atomicAdd(tickets + kTicketStride * (int)(warp_id() % kTicketSets), 1ull);
  }
  __device__ void next(long long t_begin, long long t_stop) {
    const long long k = (long long)__shfl_sync(0xffffffffu, tk, 0);
    t = t_begin + warps() < t_stop ? t_begin + warps() + warp_id() % kTicketSets + (long long)kTicketSets * k
                                   : 0x7fffffffffffffffll;
  }
};

// Tuning knobs (chosen by the autotuner per size class).
struct Tuning {
  int ruler_log2 = 3;      // a read starts a sublist with probability 2^-ruler_log2
  int tile_bytes = 4096;   // layout tile of the output (tile_seg, shares, chunks): set per graph
  int emit_tile = 0;       // spelling tile, a multiple of tile_bytes; 0: chosen per launch (emit_span)
  int emit_blocks_per_sm = 8;
  int emit_block_threads = 256;   // CTA size of the spelling kernels: 128, 256 or 512
  int grid_blocks_per_sm = 8;
};

// The spelling launch parameters as one value, for the keys of captured stages.
inline unsigned long long emit_launch_key(const Tuning& t) {
  return (unsigned long long)t.emit_blocks_per_sm | ((unsigned long long)t.emit_block_threads << 16) |
         ((unsigned long long)t.emit_tile << 32);
}

// Layout tiles a spelling warp takes at once: emit_tile / layout tile when the
// caller set one (at least one tile), else the largest span of at most 32 KiB
// that leaves every one of the launch's warps at least per_warp spans of the n
// layout tiles (big outputs: 32 KiB spans, few per-span overheads; small ones:
// one layout tile, enough spans to balance). The ASCII kernel asks for 8 per
// warp; the 2-bit one, whose fixed cost per span weighs four times more
// against its bytes, for 2.
__host__ __device__ inline int emit_span(long long n_tiles, long long warps, int emit_tile, int layout_tile,
                                         int per_warp) {
  if (emit_tile > 0) return emit_tile > layout_tile ? emit_tile / layout_tile : 1;
  int span = 1;
  while (2 * span * layout_tile <= 32768 && n_tiles / (2 * span) >= per_warp * warps) span *= 2;
  return span;
}

// CUDA events recorded after each kernel when timing is on.
struct KernelMarks {
  static constexpr int kMax = 64;
  bool on = false;
  int n = 0;
  cudaEvent_t ev[kMax + 1] = {};
  const char* name[kMax + 1] = {};
};

struct LaunchEnv {
  cudaStream_t stream;
  int num_sms;
  int coop_blocks;         // co-resident blocks for the grid-synchronised kernels
  unsigned long long* launches;  // host counter of kernel launches
  KernelMarks* marks;
  bool pdl;                // programmatic dependent launch between consecutive kernels
  bool pdl_first;          // the first kernel of a launch_* call directly follows a kernel
};

// Counts the kernel just launched and, with timing on, records an event after it.
inline void mark(const LaunchEnv& env, const char* name) {
  ++*env.launches;
  KernelMarks* m = env.marks;
  if (m && m->on && m->n < KernelMarks::kMax) {
    // inside a stream capture an external record becomes an event-record node
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(env.stream, &cs);
    if (cs == cudaStreamCaptureStatusActive)
      cudaEventRecordWithFlags(m->ev[m->n + 1], env.stream, cudaEventRecordExternal);
    else
      cudaEventRecord(m->ev[m->n + 1], env.stream);
    m->name[m->n + 1] = name;
    ++m->n;
  }
}

// ---- launchers (each returns cudaGetLastError()) ----
cudaError_t launch_validate(const DevGraph& g, DevError* derr, const LaunchEnv& env);
cudaError_t launch_mask(const DevGraph& g, const Scratch& s, const LaunchEnv& env);
cudaError_t launch_chains(const DevGraph& g, const Scratch& s, const Tuning& t, const LaunchEnv& env);
// With user_off, the piece scan also writes the caller's contig offsets
// (user_cap entries; a capacity error and nothing written when too small).
cudaError_t launch_offsets(const DevGraph& g, const Scratch& s, const Tuning& t, const LaunchEnv& env,
                           int64_t* user_off = nullptr, long long user_cap = 0);
// Spells the output tiles [t_begin, t_end) (all of them by default); with
// n_shares > 1, share `share` of the tiles cut into n_shares equal runs,
// written from out[0] on (out and cap hold that share only).
cudaError_t launch_emit(const DevGraph& g, const Scratch& s, const Tuning& t, uint8_t* out, int64_t cap,
                        const LaunchEnv& env, long long t_begin = 0, long long t_end = 1ll << 62, int share = 0,
                        int n_shares = 1);
cudaError_t launch_export_reads(const DevGraph& g, const Scratch& s, int32_t* cid, int32_t* rank, uint8_t* orient,
                                const LaunchEnv& env);
// 2-bit spelling: cap = bytes of `out`, which must hold 16 * ceil(total / 64).
// The 2-bit form of the tiles [t_begin, t_end) (tiles of tile_bytes bases; all by default).
cudaError_t launch_emit2(const DevGraph& g, const Scratch& s, const Tuning& t, uint8_t* out, int64_t cap,
                         const LaunchEnv& env, long long t_begin = 0, long long t_end = 1ll << 62);
cudaError_t launch_export_contig_off(const Scratch& s, int64_t* out, int64_t cap, const LaunchEnv& env);
cudaError_t launch_sum_len(const DevGraph& g, unsigned long long* out, const LaunchEnv& env);
// One copy of a batched load: `bytes` bytes from src (device memory, or the
// device alias of pinned host memory) to dst.
struct CopySeg {
  const uint8_t* src;
  uint8_t* dst;
  long long bytes;
};
// Every segment of seg[0, n) (device memory), a warp per segment.
cudaError_t launch_batch_copy(const CopySeg* seg, int n, const LaunchEnv& env);
cudaError_t launch_batch_fixup(int k, const int64_t* R, const int64_t* E, const int64_t* PB, const int64_t* SR,
                               const void* stage_rp, int rp_bytes, int64_t* rp, int32_t* col, int64_t* off,
                               long long N, long long M, const LaunchEnv& env);
cudaError_t launch_batch_ranges(const Scratch& s, int k, const int64_t* R, long long N, int64_t* first_contig,
                                int64_t* first_base, const LaunchEnv& env);
// Batches with host-resident reads: the slots of the pieces' words (exclusive
// scan over walk positions, total at [W]), then the gather into one device
// buffer, which rewrites every piece's source into it.
cudaError_t launch_gather_slots(const Scratch& s, long long W, unsigned long long* slot, unsigned long long* state,
                                long long state_cap, const LaunchEnv& env);
// With t_end > 0: only the pieces output tiles [t_begin, t_end) need that no
// earlier range of an increasing sequence took.
cudaError_t launch_gather_pieces(const Scratch& s, int k, const int64_t* PB, const uint8_t* const* base,
                                 const int64_t* bytes, const unsigned long long* slot, uint32_t* dst,
                                 long long cap_words, long long W, const LaunchEnv& env, long long t_begin = 0,
                                 long long t_end = 0);
// Buffers of the contig-weight sort (capacity: the number of contigs).
struct SortBuffers {
  unsigned long long* key[2];
  int32_t* val[2];
  unsigned* hist;              // 256 x tiles_cap digit counts
  unsigned long long* base;    // 256 x tiles_cap scatter bases
  unsigned long long* state;   // look-back descriptors of the digit scan, + 1 ticket
  long long tiles_cap, state_cap;
};
// Buffers of the transitive reduction (m entries, n rows).
struct TrBuffers {
  int32_t* row_of;             // m: row of every entry
  uint8_t* trans;              // m: entry is transitive
  uint8_t* keep;               // m: entry kept (its pair is not transitive)
  int32_t* row_cnt;            // n: kept entries per row
  int64_t* out_rp;             // n + 1: the reduced graph's row offsets
  unsigned long long* total;   // kept entries
  unsigned long long* state;   // look-back descriptors of the row scan, + 1 ticket
  long long state_cap;
  DevError* derr;
};
// TransitiveReduction: row checks (launch_transitive_check, then the entry
// checks), marks, keeps, scans (launch_transitive), then writes the kept
// entries (launch_transitive_scatter). Each step needs the checks before it
// to have passed: the later kernels index rows by column values.
cudaError_t launch_transitive_check(const DevGraph& g, DevError* derr, const LaunchEnv& env);
cudaError_t launch_transitive_entries(const DevGraph& g, const TrBuffers& t, const LaunchEnv& env);
cudaError_t launch_transitive(const DevGraph& g, int fuzz, const TrBuffers& t, const LaunchEnv& env);
cudaError_t launch_transitive_scatter(const DevGraph& g, const TrBuffers& t, int32_t* col, uint8_t* code, int32_t* suf,
                                      const LaunchEnv& env);
constexpr int kMaxParts = 1024;
// GreedyPartitioning of the C contigs of the last offsets stage into P parts
// (weight 0: reads per contig, 1: bases); max_weight bounds every part sum.
cudaError_t launch_partition(const Scratch& s, long long C, int weight, long long max_weight, int P,
                             const SortBuffers& b, int32_t* part, int64_t* psum, const LaunchEnv& env);
int coop_blocks_for_grid_kernels(int num_sms);
// The read exchange of a run split over ranks that each hold a slice of the
// reads (cg_exchange_*). rf: device, n_shares + 1 read-id bounds (rank r owns
// reads [rf[r], rf[r+1])). A share's pieces are the walk positions
// [range[2p], range[2p+1]] (inclusive; range[2p] > range[2p+1] when empty).
struct XchgArgs {
  const int64_t* rf;
  int n_shares;
  int rank;
  const long long* range;       // 2 x n_shares
  const long long* pair0;       // n_shares + 1: first pair index of each share's range
};
// share ranges from the tile map (needs the layout's counters)
cudaError_t launch_x_ranges(const Scratch& s, int n_shares, int tile_bytes, long long* range, const LaunchEnv& env);
// words (4 bytes) this rank sends to each share and receives from each rank
cudaError_t launch_x_sizes(const Scratch& s, const XchgArgs& x, unsigned long long* send_words,
                           unsigned long long* recv_words, long long n_pairs, const LaunchEnv& env);
// one exclusive scan over a share's walk positions [j0, j0 + count): for the
// pieces whose read `who` owns, their word offset among those pieces (slot[i])
cudaError_t launch_x_scan(const Scratch& s, const XchgArgs& x, long long j0, long long count, int who,
                          long long* slot, unsigned long long* state, long long state_cap, const LaunchEnv& env);
// the sender: one exclusive scan over all pairs of the words of the pieces it
// owns (slot[i] for every pair; a piece's offset in its share's segment is
// slot[i] - slot[first pair of that share])
cudaError_t launch_x_scan_pairs(const Scratch& s, const XchgArgs& x, long long n_pairs, long long* slot,
                                unsigned long long* state, long long state_cap, const LaunchEnv& env);
cudaError_t launch_x_pack(const DevGraph& g, const Scratch& s, const XchgArgs& x, const uint8_t* my_packed,
                          long long my_bytes, const int64_t* my_off, const long long* seg, const long long* slot,
                          uint32_t* send, long long n_pairs, const LaunchEnv& env);
// the receiver: every piece's source moved into the receive buffer
cudaError_t launch_x_rewrite(const Scratch& s, const XchgArgs& x, const long long* seg, const long long* slot,
                             const LaunchEnv& env);
// Self-test of the look-back scan's bounded wait: scans `tiles` tiles of
// zeros with `state` (tiles descriptors + the ticket word) prepared by the
// caller; a ticket that starts at 1 withholds tile 0, so the later tiles'
// waits run out and the kernel records DERR_TIMEOUT.
cudaError_t launch_selftest_wait(unsigned long long* state, long long tiles, DevError* derr, const LaunchEnv& env);

// ---- device helpers ----
__device__ __forceinline__ void set_error(DevError* e, int code, int where, long long index) {
  if (atomicCAS(&e->err, 0, code) == 0) {
    e->where = where;
    e->index = index;
  }
}

// Programmatic dependent launch (sm_90 and later): wait until the grid before this
// one on the stream has completed and its writes are visible. Every kernel of the
// path calls it before it touches global memory, so each kernel also completes
// after every kernel before it. No kernel signals its dependents early
// (griddepcontrol.launch_dependents): the next grid is launched once every block
// of this one has exited, ahead of the grid's completion. Signalling at kernel entry, which parks the next grid's blocks on the SMs
// while this one runs, made the 3.1 Gb step 14 us slower. For a kernel launched
// without the attribute the wait returns at once.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ long long grid_tid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long grid_threads() { return (long long)gridDim.x * blockDim.x; }

enum KernelId {
  K_VALIDATE1 = 1, K_VALIDATE2, K_MASK, K_SUCC, K_WALK, K_JUMP, K_FINAL, K_CYCLE, K_EXPORT,
  K_SCAN_HEADS, K_SCATTER, K_SCAN_OFFSETS, K_CONTIG_OFF, K_EMIT, K_SORT, K_TRANSITIVE, K_BATCH_GATHER,
  K_SELFTEST_WAIT
};

// Blocks of `threads` threads (kBlock by default) of `kernel` that fit on one SM at once.
template <typename Kernel>
inline int resident_blocks(Kernel kernel, int threads = kBlock) {
  int r = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, kernel, threads, 0);
  return r > 0 ? r : 1;
}

// Launches `kernel` with kBlock threads on env.stream. With `chained` (the stream's
// previous operation is one of these kernels, with no event or copy between) and
// programmatic dependent launch on, the launch carries the programmatic
// stream-serialization attribute: it is launched once the previous grid's blocks
// have exited rather than after the grid's completion, and each block waits in
// pdl_enter() for that completion. Per-kernel timing events sit between every two
// kernels, so they turn the attribute off.
template <typename... P, typename... A>
inline cudaError_t launch_kb(void (*kernel)(P...), int grid, int threads, const LaunchEnv& env, bool chained,
                             A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = env.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained && env.pdl && !(env.marks && env.marks->on) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}

template <typename... P, typename... A>
inline cudaError_t launch_k(void (*kernel)(P...), int grid, const LaunchEnv& env, bool chained, A&&... args) {
  return launch_kb(kernel, grid, kBlock, env, chained, static_cast<A&&>(args)...);
}

inline int grid_for(long long n, const LaunchEnv& env, int per_sm = 8) {
  long long b = (n + kBlock - 1) / kBlock;
  long long cap = (long long)env.num_sms * per_sm;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

__device__ __forceinline__ int64_t rowp(const DevGraph& g, int64_t v) {
  return g.rp64 ? reinterpret_cast<const int64_t*>(g.row_ptr)[v]
                : (int64_t)reinterpret_cast<const int32_t*>(g.row_ptr)[v];
}

// Warp-aggregated append to a list; returns the slot.
__device__ __forceinline__ unsigned warp_append(unsigned* counter, bool want) {
  unsigned mask = __ballot_sync(0xffffffffu, want);
  if (!want) return 0;
  int lane = threadIdx.x & 31;
  int leader = __ffs(mask) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return base + (unsigned)__popc(mask & ((1u << lane) - 1u));
}

}  // namespace cg
