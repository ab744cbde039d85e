// cg_api.cu - the C ABI of include/cg.h: contexts, graph loading, and the
// stage sequence mask -> chains -> offsets -> emission on one CUDA stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "cg.h"
#include "cg_fault.h"
#include <nvtx3/nvToolsExt.h>
#include "cg_internal.cuh"

struct cg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint64_t budget = 0, used = 0;
  cg::LaunchEnv env{};
  cg::Tuning tune{};
  cg::DevError* derr = nullptr;   // device
  cg::DevError* h_err = nullptr;  // pinned host mirror
  cg::Counters* h_ctr = nullptr;  // pinned host mirror of one graph's counters
  unsigned long long* h_u64 = nullptr;  // pinned host word
  cg_status sticky = CG_OK;
  std::string last_error;
  cudaMemPool_t mempool = nullptr;     // device memory of this context's graphs and scratch
  std::map<void*, size_t> sizes;       // every live allocation of this context
  unsigned long long launches = 0;
  bool timing = false;
  bool timing_emit_only = false;       // level 3: events around the spelling stage only
  cudaEvent_t ev[8] = {};              // start/end of mask, chains, offsets, emission
  bool recorded[4] = {false, false, false, false};
  cg::KernelMarks marks;               // per-kernel events of the last run (timing on)
  bool graphs = true;                  // replay each stage from a captured CUDA graph
  bool host_direct = true;             // kernels write pinned host outputs in place
  cudaStream_t copy_stream = nullptr;  // device-to-host copies overlapping the spelling (created on first use)
  cudaEvent_t copy_ev = nullptr;       //   a chunk spelled / the copies done
  cg::FaultPlan fault;                 // host-side fault injection (tests)
};

// A captured stage: the instantiated graph and what its capture recorded.
struct StageExec {
  cudaGraphExec_t exec = nullptr;
  uint64_t key = 0;
  unsigned long long kernels = 0;      // kernels in the graph
  int mark_end = 0;                    // per-kernel timing marks after the stage
};

struct cg_graph {
  cg_ctx* ctx = nullptr;
  cg::DevGraph g{};
  cg::Scratch s{};
  std::vector<void*> owned;
  int stage = 0;                  // 0 loaded, 1 masked, 2 chained, 3 offsets (launches issued)
  int want = 0;                   // a later stage asked for with nothing to return, not yet launched
  int64_t sum_len = 0;
  int layout_tile = 4096;         // output layout tile (gt)
  uint8_t* stage_bases = nullptr; // device staging for host outputs
  int64_t stage_bases_cap = 0;
  void* stage_reads = nullptr;
  int32_t* part_buf = nullptr;         // device copy of a host part assignment (cg_emit_part)
  int64_t part_buf_cap = 0;
  unsigned long long* d_sum = nullptr;
  StageExec execs[8];                  // mask, chains, offsets, emission, contig_off export, 2-bit emission,
                                       // offsets + emission + export in one graph, all stages in one graph
  int batch_k = 0;                     // graphs of a batch (0: a single graph)
  int64_t* batch_R = nullptr;          // device: first read of each graph, batch_k + 1 entries
  // a batch whose reads stay in pinned host memory: per graph its stream's
  // device alias, length and virtual start; the gathered pieces' words
  bool host_batch = false;
  const uint8_t** hb_base = nullptr;
  int64_t* hb_bytes = nullptr;
  const int64_t* hb_PB = nullptr;
  unsigned long long* hb_slot = nullptr;
  unsigned long long* hb_state = nullptr;
  long long hb_state_cap = 0;
  uint32_t* hb_dst = nullptr;
  int64_t hb_dst_words = 0;
  cg::DevGraph g_emit{};               // the graph as the spelling sees it (gathered reads)
  cg::Tuning tune{};                   // the context's launch parameters as this graph uses them
};

namespace {

cg_status fail(cg_ctx* c, cg_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->last_error = buf;
    if (s == CG_ETIMEOUT || s == CG_EKERNEL || s == CG_ECUDA) c->sticky = s;
  }
  return s;
}

cg_status cuda_fail(cg_ctx* c, cudaError_t e, const char* what) {
  return fail(c, CG_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                 \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

// Device allocation: stream-ordered suballocation from the context's CUDA
// memory pool (which keeps freed memory for reuse, up to the budget), under
// the context's HBM budget.
void* dalloc(cg_ctx* c, size_t bytes, cg_status* st) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (c->budget && c->used + bytes > c->budget) {
    *st = fail(c, CG_ENOMEM, "HBM budget: %zu bytes in use, %zu more requested, budget %llu", (size_t)c->used,
               bytes, (unsigned long long)c->budget);
    return nullptr;
  }
  if (c->fault.hit("alloc")) {
    *st = fail(c, CG_ENOMEM, "injected: device allocation of %zu bytes", bytes);
    return nullptr;
  }
  void* p = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, c->mempool, c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *st = fail(c, CG_ENOMEM, "device allocation of %zu bytes: %s", bytes, cudaGetErrorString(e));
    return nullptr;
  }
  c->used += bytes;
  c->sizes[p] = bytes;
  return p;
}

void dfree(cg_ctx* c, void* p) {
  if (!p) return;
  auto it = c->sizes.find(p);
  if (it == c->sizes.end()) return;
  cudaFreeAsync(p, c->stream);
  c->used -= it->second;
  c->sizes.erase(it);
}

template <class T>
T* galloc(cg_graph* g, size_t count, cg_status* st) {
  void* p = dalloc(g->ctx, count * sizeof(T), st);
  if (p) g->owned.push_back(p);
  return reinterpret_cast<T*>(p);
}

// Reads the context error word and the graph counters (waits for the stream).
cg_status flush(cg_graph* g);

cg_status wait_and_read(cg_graph* g) {
  cg_ctx* c = g->ctx;
  if (g->want) {                          // launches that still wait go first
    cg_status st0 = flush(g);
    if (st0 != CG_OK) return st0;
  }
  CK(cudaMemcpyAsync(c->h_err, c->derr, sizeof(cg::DevError), cudaMemcpyDeviceToHost, c->stream), "read error word");
  if (g->s.ctr)
    CK(cudaMemcpyAsync(c->h_ctr, g->s.ctr, sizeof(cg::Counters), cudaMemcpyDeviceToHost, c->stream), "read counters");
  CK(cudaStreamSynchronize(c->stream), "stream synchronize");
  cg::DevError e = *c->h_err;
  if (c->fault.hit("timeout")) return fail(c, CG_ETIMEOUT, "injected: device wait timed out");
  if (c->fault.hit("kernel")) return fail(c, CG_EKERNEL, "injected: kernel consistency check failed");
  if (e.err == cg::DERR_NONE) return CG_OK;
  if (e.err == cg::DERR_CAPACITY || e.err == cg::DERR_GRAPH) {
    CK(cudaMemsetAsync(c->derr, 0, sizeof(cg::DevError), c->stream), "clear error word");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    if (e.err == cg::DERR_CAPACITY)
      return fail(c, CG_EINVAL, "output buffer too small: %lld needed (kernel %d)", e.index, e.where);
    return fail(c, CG_EGRAPH, "invalid string graph: check %d failed at index %lld", e.where, e.index);
  }
  if (e.err == cg::DERR_TIMEOUT) return fail(c, CG_ETIMEOUT, "device wait timed out in kernel %d", e.where);
  return fail(c, CG_EKERNEL, "kernel %d found an inconsistency at index %lld", e.where, e.index);
}

cg_status check_ctx(cg_ctx* c) {
  if (!c) return CG_EINVAL;
  if (c->sticky != CG_OK) return c->sticky;
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  return CG_OK;
}

// An NVTX range around a host-side call (shown by profilers on the host
// timeline; without a tool attached it costs a few nanoseconds).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

// Brackets one stage with an NVTX range and, when timing is on, CUDA events.
struct StageTimer {
  cg_ctx* c;
  int k;
  bool on;
  Range range;
  static const char* name(int k) {
    static const char* const n[4] = {"cg.mask", "cg.chains", "cg.offsets", "cg.emit"};
    return n[k & 3];
  }
  StageTimer(cg_ctx* c_, int k_)
      : c(c_), k(k_), on(c_->timing && (!c_->timing_emit_only || k_ == 3)), range(name(k_)) {
    if (on) cudaEventRecord(c->ev[2 * k], c->stream);
  }
  ~StageTimer() {
    if (on) {
      cudaEventRecord(c->ev[2 * k + 1], c->stream);
      c->recorded[k] = true;
    }
  }
};

// A stage-boundary event inside a launch sequence that may be captured: a
// captured record becomes an event-record node of the graph.
void record_stage_event(cg_ctx* c, int i) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(c->stream, &cs);
  if (cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(c->ev[i], c->stream, cudaEventRecordExternal);
  else
    cudaEventRecord(c->ev[i], c->stream);
}

uint64_t mix_key(uint64_t h, uint64_t v) { return (h ^ (v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2))); }

// The launch parameters a graph's stages use: the context's, with the graph's
// own layout tile (the granularity of its tile map, shares and copy chunks:
// 4 KiB below 2^31 bases of reads, else 8 KiB, where the finer map costs the
// offsets stage more than it gives the spelling). Each spelling launch groups
// layout tiles into spans of emit_tile bytes, or of a size it chooses from the
// output when emit_tile is 0.
const cg::Tuning& gt(cg_graph* g) {
  g->tune = g->ctx->tune;
  g->tune.tile_bytes = g->layout_tile;
  return g->tune;
}

// Runs one stage's launches. With graphs on, the launches are captured once
// into a CUDA graph per (stage, key) and replayed with a single launch; the
// key covers every host-side value the launches bake in (buffers, sizes,
// tuning, timing marks).
template <class F>
cg_status run_stage(cg_graph* g, int slot, uint64_t key, F&& launch) {
  cg_ctx* c = g->ctx;
  if (!c->graphs) return launch();
  StageExec& e = g->execs[slot];
  key = mix_key(key, c->marks.on ? 1 : 2);
  key = mix_key(key, c->env.pdl ? 3 : 4);
  key = mix_key(mix_key(key, (uint64_t)(uintptr_t)g->s.part), (uint64_t)(uint32_t)g->s.part_p);
  if (e.exec && e.key == key) {
    c->launches += e.kernels;
    if (c->marks.on) c->marks.n = e.mark_end;
    CK(cudaGraphLaunch(e.exec, c->stream), "cudaGraphLaunch");
    return CG_OK;
  }
  if (e.exec) {
    cudaGraphExecDestroy(e.exec);
    e.exec = nullptr;
  }
  const unsigned long long l0 = c->launches;
  CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  cg_status st = launch();
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(c->stream, &graph);
  if (st != CG_OK) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return st;
  }
  if (ee != cudaSuccess) return cuda_fail(c, ee, "cudaStreamEndCapture");
  ee = cudaGraphInstantiate(&e.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ee != cudaSuccess) {
    e.exec = nullptr;
    return cuda_fail(c, ee, "cudaGraphInstantiate");
  }
  e.key = key;
  e.kernels = c->launches - l0;
  e.mark_end = c->marks.n;
  CK(cudaGraphLaunch(e.exec, c->stream), "cudaGraphLaunch");
  return CG_OK;
}

cg_status run_mask(cg_graph* g) {
  cg_ctx* c = g->ctx;
  if (c->marks.on) {                   // a new run: per-kernel marks start over
    c->marks.n = 0;
    cudaEventRecord(c->marks.ev[0], c->stream);
  }
  StageTimer tm(c, 0);
  cg_status st = run_stage(g, 0, 1, [&]() -> cg_status {
    CK(cg::launch_mask(g->g, g->s, c->env), "mask kernels");
    return CG_OK;
  });
  if (st != CG_OK) return st;
  g->stage = 1;
  return CG_OK;
}

cg_status run_chains(cg_graph* g) {
  cg_ctx* c = g->ctx;
  if (g->stage < 1) {
    cg_status st0 = run_mask(g);
    if (st0 != CG_OK) return st0;
  }
  StageTimer tm(c, 1);
  cg_status st = run_stage(g, 1, (uint64_t)gt(g).ruler_log2, [&]() -> cg_status {
    CK(cg::launch_chains(g->g, g->s, gt(g), c->env), "chain kernels");
    return CG_OK;
  });
  if (st != CG_OK) return st;
  g->stage = 2;
  return CG_OK;
}

// The mask and chain calls return nothing when asked for no outputs or
// counts; then, with graphs on and no per-kernel marks or per-stage events,
// their launches wait for the next call, so that a spelling into device
// buffers replays all four stages as one CUDA graph (each graph launch of its
// own costs the GPU a few microseconds between stages). flush() issues what
// waits; every call that uses the graph's device state does that first.
bool defer_ok(const cg_ctx* c) {
  return c->graphs && !c->marks.on && (!c->timing || c->timing_emit_only);
}

cg_status flush(cg_graph* g) {
  const int want = g->want;
  g->want = 0;
  if (want > g->stage) return want >= 2 ? run_chains(g) : run_mask(g);
  return CG_OK;
}

cg_status run_offsets(cg_graph* g) {
  cg_ctx* c = g->ctx;
  if (g->want) {
    cg_status st0 = flush(g);
    if (st0 != CG_OK) return st0;
  }
  if (g->stage < 2) {
    cg_status st0 = run_chains(g);
    if (st0 != CG_OK) return st0;
  }
  StageTimer tm(c, 2);
  cg_status st = run_stage(g, 2, (uint64_t)gt(g).tile_bytes, [&]() -> cg_status {
    CK(cg::launch_offsets(g->g, g->s, gt(g), c->env), "offset kernels");
    return CG_OK;
  });
  if (st != CG_OK) return st;
  g->stage = 3;
  return CG_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

// The graph the spelling kernels read: g itself, or for a batch with
// host-resident reads the gathered pieces (prepare_emit).
const cg::DevGraph& emit_graph(const cg_graph* g) { return g->host_batch ? g->g_emit : g->g; }

// For a batch with host-resident reads, after the offsets stage: the words of
// every piece, gathered from its graph's pinned host stream into one device
// buffer (at most total/16 + 3 W words), and the pieces' sources moved there.
// With gather_all false only the slots are laid out: the caller gathers the
// pieces range by range (gather_range) before spelling each range of tiles.
cg_status prepare_emit(cg_graph* g, bool gather_all = true) {
  if (!g->host_batch) return CG_OK;
  cg_ctx* c = g->ctx;
  cg_status st = wait_and_read(g);                  // the walk positions and bases of this layout
  if (st != CG_OK) return st;
  const long long W = c->h_ctr->n_walk, total = c->h_ctr->total_bases;
  if (!g->hb_slot) {
    const long long n = g->g.n > 0 ? g->g.n : 1;
    g->hb_state_cap = (n + 2047) / 2048 + 1;
    g->hb_slot = galloc<unsigned long long>(g, (size_t)n + 1, &st);
    g->hb_state = galloc<unsigned long long>(g, (size_t)g->hb_state_cap + 1, &st);
    if (st != CG_OK) return st;
  }
  const long long need = total / 16 + 3 * W + 16;
  if (g->hb_dst_words < need) {
    if (g->hb_dst) dfree(c, g->hb_dst);
    g->hb_dst = (uint32_t*)dalloc(c, (size_t)need * 4, &st);
    g->hb_dst_words = g->hb_dst ? need : 0;
    if (st != CG_OK) return st;
  }
  CK(cg::launch_gather_slots(g->s, W, g->hb_slot, g->hb_state, g->hb_state_cap, c->env), "gather slots");
  if (gather_all)
    CK(cg::launch_gather_pieces(g->s, g->batch_k, g->hb_PB, g->hb_base, g->hb_bytes, g->hb_slot, g->hb_dst,
                                g->hb_dst_words, W, c->env), "gather pieces");
  g->g_emit = g->g;
  g->g_emit.packed = reinterpret_cast<const uint8_t*>(g->hb_dst);
  g->g_emit.packed_bytes = 4 * g->hb_dst_words;
  g->g_emit.packed_readable = 4 * g->hb_dst_words;
  g->g_emit.packed_host = false;
  return CG_OK;
}

// The device address of pinned (page-locked, mapped) host memory, or nullptr
// for any other pointer: only such memory may be read or written by kernels.
void* pinned_device_alias(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer || !a.hostPointer) return nullptr;
  // the alias of p itself (p may lie inside a larger pinned allocation)
  return (char*)a.devicePointer + ((const char*)p - (const char*)a.hostPointer);
}

// Scratch, input checks and output bounds of a graph whose inputs are in place.
cg_status finish_load(cg_graph* g, uint32_t flags) {
  cg_ctx* c = g->ctx;
  cg::DevGraph& G = g->g;
  const int64_t n = G.n;
  cg_status st = CG_OK;
  // scratch
  cg::Scratch& S = g->s;
  const size_t N = (size_t)(n > 0 ? n : 1), N2 = 2 * N, NW = N / 32 + 2;
  S.branch = galloc<uint8_t>(g, N, &st);
  S.cand = galloc<int32_t>(g, N, &st);
  S.cidx = galloc<int32_t>(g, N, &st);
  S.lone = galloc<int32_t>(g, N, &st);
  S.hb_mask = galloc<unsigned>(g, NW, &st);
  S.hb = galloc<unsigned>(g, NW, &st);
  S.wp = galloc<unsigned>(g, NW, &st);
  S.succ = galloc<int4>(g, N, &st);
  S.sufin = galloc<int32_t>(g, N2, &st);
  if (G.pre) {
    S.preout = galloc<int32_t>(g, N2, &st);
    S.pfirst = galloc<int32_t>(g, N, &st);
  }
  S.rr = galloc<int2>(g, N2, &st);
  S.rlist = galloc<int32_t>(g, N2, &st);
  S.hlist = galloc<int32_t>(g, N2, &st);
  S.rec = galloc<int4>(g, N2, &st);
  for (int b = 0; b < 2; ++b) {
    S.pj[b] = galloc<int4>(g, N2, &st);
    S.c_ptr[b] = galloc<int32_t>(g, N2, &st);
    S.c_val[b] = galloc<long long>(g, N2, &st);
  }
  S.c_head = galloc<int32_t>(g, N2, &st);
  S.prd = galloc<int4>(g, N, &st);
  S.headq = galloc<int32_t>(g, N, &st);
  S.cyc = galloc<int32_t>(g, N, &st);
  S.qd = galloc<int32_t>(g, N, &st);
  S.cbase = galloc<unsigned long long>(g, N + 1, &st);
  S.wsrc = galloc<unsigned long long>(g, N, &st);
  S.wlen = galloc<int32_t>(g, N, &st);
  S.out_off = galloc<int64_t>(g, N + 1, &st);
  S.wfirst = galloc<int32_t>(g, N, &st);
  if (G.no_reads) S.wread = galloc<int32_t>(g, N, &st);
  S.contig_off = galloc<int64_t>(g, N + 1, &st);
  S.scan_tiles_cap = (int64_t)(N + 2047) / 2048 + 1;
  S.scan_state[0] = galloc<unsigned long long>(g, 3 * ((size_t)S.scan_tiles_cap + 1), &st);
  if (S.scan_state[0]) {
    S.scan_state[1] = S.scan_state[0] + (S.scan_tiles_cap + 1);
    S.scan_state[2] = S.scan_state[1] + (S.scan_tiles_cap + 1);
    // zeroed once; afterwards each offsets-stage scan zeroes the other's descriptors
    CK(cudaMemsetAsync(S.scan_state[0], 0, 3 * ((size_t)S.scan_tiles_cap + 1) * sizeof(unsigned long long),
                       c->stream), "clear scan descriptors");
  }
  S.ctr = galloc<cg::Counters>(g, 1, &st);
  S.tickets = galloc<unsigned long long>(g, cg::kTicketSets * cg::kTicketStride, &st);
  g->d_sum = galloc<unsigned long long>(g, 1, &st);
  S.derr = c->derr;
  if (st != CG_OK) return st;
  CK(cudaMemsetAsync(S.ctr, 0, sizeof(cg::Counters), c->stream), "clear counters");
  CK(cudaMemsetAsync(g->d_sum, 0, 8, c->stream), "clear sum");

  if (!(flags & CG_NO_VALIDATE) && n > 0) CK(cg::launch_validate(G, c->derr, c->env), "validation kernels");
  CK(cg::launch_sum_len(G, g->d_sum, c->env), "length sum");
  CK(cudaMemcpyAsync(c->h_u64, g->d_sum, 8, cudaMemcpyDeviceToHost, c->stream), "read sum");
  st = wait_and_read(g);
  if (st != CG_OK) return st;
  if (c->fault.hit("bad_graph")) return fail(c, CG_EGRAPH, "injected: invalid string graph");
  g->sum_len = (int64_t)*c->h_u64;
  g->layout_tile = g->sum_len < ((int64_t)1 << 31) ? 4096 : 8192;
  // the longest possible output is every read spelled whole, in tiles of at least 4 KiB
  S.tiles_cap = g->sum_len / 4096 + 2;
  S.tile_seg = galloc<int32_t>(g, (size_t)S.tiles_cap + 1, &st);
  return st;
}


}  // namespace

extern "C" {

const char* cg_status_str(cg_status s) {
  switch (s) {
    case CG_OK: return "CG_OK";
    case CG_EINVAL: return "CG_EINVAL";
    case CG_ENOMEM: return "CG_ENOMEM";
    case CG_ECUDA: return "CG_ECUDA";
    case CG_EGRAPH: return "CG_EGRAPH";
    case CG_ETIMEOUT: return "CG_ETIMEOUT";
    case CG_EBUSY: return "CG_EBUSY";
    case CG_EKERNEL: return "CG_EKERNEL";
  }
  return "CG_UNKNOWN";
}

cg_status cg_last_error(cg_ctx* c, char* buf, size_t buflen) {
  if (!c || !buf || buflen == 0) return CG_EINVAL;
  snprintf(buf, buflen, "%s", c->last_error.c_str());
  return CG_OK;
}

cg_status cg_create(cg_ctx** out, int device, uint64_t hbm_budget_bytes, void* cuda_stream) {
  if (!out) return CG_EINVAL;
  *out = nullptr;
  cg_ctx* c = new (std::nothrow) cg_ctx();
  if (!c) return CG_ENOMEM;
  c->device = device;
  c->budget = hbm_budget_bytes;
  c->fault.from_env();
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) { delete c; return CG_ECUDA; }
  if (cuda_stream) {
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return CG_ECUDA; }
    c->own_stream = true;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  c->env.stream = c->stream;
  c->env.num_sms = sms > 0 ? sms : 1;
  c->env.coop_blocks = cg::coop_blocks_for_grid_kernels(c->env.num_sms);
  c->env.pdl = true;
  c->env.pdl_first = false;
  {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&c->mempool, &props) != cudaSuccess) {
      cudaGetLastError();
      c->mempool = nullptr;
      cg_destroy(c);
      return CG_ECUDA;
    }
    uint64_t keep = c->budget ? c->budget : ~0ull;   // freed memory stays in the pool up to this much
    cudaMemPoolSetAttribute(c->mempool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  c->env.launches = &c->launches;
  c->env.marks = &c->marks;
  if (cudaMalloc(&c->derr, sizeof(cg::DevError)) != cudaSuccess ||
      cudaMallocHost(&c->h_err, sizeof(cg::DevError)) != cudaSuccess ||
      cudaMallocHost(&c->h_ctr, sizeof(cg::Counters)) != cudaSuccess ||
      cudaMallocHost(&c->h_u64, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    cg_destroy(c);
    return CG_ENOMEM;
  }
  cudaMemsetAsync(c->derr, 0, sizeof(cg::DevError), c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) { cudaGetLastError(); cg_destroy(c); return CG_ECUDA; }
  *out = c;
  return CG_OK;
}

cg_status cg_destroy(cg_ctx* c) {
  if (!c) return CG_EINVAL;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& kv : c->sizes) cudaFreeAsync(kv.first, c->stream);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->mempool) cudaMemPoolDestroy(c->mempool);
  if (c->derr) cudaFree(c->derr);
  if (c->h_err) cudaFreeHost(c->h_err);
  if (c->h_ctr) cudaFreeHost(c->h_ctr);
  if (c->h_u64) cudaFreeHost(c->h_u64);
  for (cudaEvent_t e : c->ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : c->marks.ev)
    if (e) cudaEventDestroy(e);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  if (c->copy_ev) cudaEventDestroy(c->copy_ev);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  cudaGetLastError();
  delete c;
  return CG_OK;
}

cg_status cg_set_tuning(cg_ctx* c, const cg_tuning* t) {
  if (!c || !t) return CG_EINVAL;
  cg::Tuning n = c->tune;
  if (t->ruler_log2 > 0) {
    if (t->ruler_log2 > 12) return fail(c, CG_EINVAL, "ruler_log2 must be in 1..12");
    n.ruler_log2 = t->ruler_log2;
  }
  if (t->tile_bytes > 0) {
    if (t->tile_bytes < 4096 || t->tile_bytes > 131072 || (t->tile_bytes & (t->tile_bytes - 1)))
      return fail(c, CG_EINVAL, "tile_bytes must be a power of two from 4096 to 131072");
    n.emit_tile = t->tile_bytes;
  }
  if (t->emit_blocks_per_sm > 0) {
    if (t->emit_blocks_per_sm > 16) return fail(c, CG_EINVAL, "emit_blocks_per_sm must be in 1..16");
    n.emit_blocks_per_sm = t->emit_blocks_per_sm;
  }
  if (t->emit_block_threads > 0) {
    if (t->emit_block_threads != 128 && t->emit_block_threads != 256 && t->emit_block_threads != 512)
      return fail(c, CG_EINVAL, "emit_block_threads must be 128, 256 or 512");
    n.emit_block_threads = t->emit_block_threads;
  }
  c->tune = n;
  return CG_OK;
}

cg_status cg_get_tuning(cg_ctx* c, cg_tuning* out) {
  if (!c || !out) return CG_EINVAL;
  out->ruler_log2 = c->tune.ruler_log2;
  out->tile_bytes = c->tune.emit_tile;
  out->emit_blocks_per_sm = c->tune.emit_blocks_per_sm;
  out->emit_block_threads = c->tune.emit_block_threads;
  return CG_OK;
}

cg_status cg_set_graphs(cg_ctx* c, int enable) {
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  c->graphs = enable != 0;
  return CG_OK;
}

cg_status cg_set_pdl(cg_ctx* c, int enable) {
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  c->env.pdl = enable != 0;
  return CG_OK;
}

cg_status cg_set_fault(cg_ctx* c, const char* spec) {
  if (!c) return CG_EINVAL;
  c->fault.set(spec);
  return CG_OK;
}

cg_status cg_set_host_direct(cg_ctx* c, int enable) {
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  c->host_direct = enable != 0;
  return CG_OK;
}

cg_status cg_set_timing(cg_ctx* c, int enable) {
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (enable && !c->ev[0]) {
    for (cudaEvent_t& e : c->ev) CK(cudaEventCreate(&e), "cudaEventCreate");
    for (cudaEvent_t& e : c->marks.ev) CK(cudaEventCreate(&e), "cudaEventCreate");
  }
  c->timing = enable != 0;
  c->timing_emit_only = enable == 3;
  c->marks.on = enable == 2;
  c->marks.n = 0;
  for (bool& r : c->recorded) r = false;
  return CG_OK;
}

cg_status cg_get_stats(cg_ctx* c, cg_stats* out) {
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (!out) return CG_EINVAL;
  out->kernels_launched = c->launches;
  for (int k = 0; k < 4; ++k) out->stage_ms[k] = 0.f;
  if (c->timing) {
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    for (int k = 0; k < 4; ++k)
      if (c->recorded[k]) CK(cudaEventElapsedTime(&out->stage_ms[k], c->ev[2 * k], c->ev[2 * k + 1]), "event time");
  }
  return CG_OK;
}

cg_status cg_kernel_time(cg_ctx* c, int k, const char** name, float* ms) {
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (!c->marks.on || k < 0 || k >= c->marks.n) return CG_EINVAL;
  CK(cudaStreamSynchronize(c->stream), "stream synchronize");
  if (name) *name = c->marks.name[k + 1];
  if (ms && cudaEventElapsedTime(ms, c->marks.ev[k], c->marks.ev[k + 1]) != cudaSuccess) {
    cudaGetLastError();                // a measurement gap is not a failure of the context
    *ms = -1.f;
  }
  return CG_OK;
}

static cg_status wait_and_read_ctx(cg_ctx* c) {
  cg_graph tmp;
  tmp.ctx = c;
  return wait_and_read(&tmp);
}

cg_status cg_sync(cg_ctx* c) {
  if (!c) return CG_EINVAL;
  if (c->sticky != CG_OK) return c->sticky;
  return wait_and_read_ctx(c);
}

cg_status cg_selftest_wait_timeout(cg_ctx* c, int32_t tiles) {
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (tiles < 2 || tiles > 4096) return fail(c, CG_EINVAL, "selftest: tiles must be in 2..4096");
  CK(cudaStreamSynchronize(c->stream), "stream synchronize");   // earlier work reports its own errors first
  st = wait_and_read_ctx(c);
  if (st != CG_OK) return st;
  unsigned long long* state = static_cast<unsigned long long*>(dalloc(c, (size_t)(tiles + 1) * 8, &st));
  if (!state) return st;
  CK(cudaMemsetAsync(state, 0, (size_t)(tiles + 1) * 8, c->stream), "clear descriptors");
  *c->h_u64 = 1;   // the first ticket handed out is 1: no block ever takes tile 0
  CK(cudaMemcpyAsync(state + tiles, c->h_u64, 8, cudaMemcpyHostToDevice, c->stream), "seed ticket");
  CK(cg::launch_selftest_wait(state, tiles, c->derr, c->env), "launch selftest scan");
  CK(cudaMemcpyAsync(c->h_err, c->derr, sizeof(cg::DevError), cudaMemcpyDeviceToHost, c->stream), "read error word");
  CK(cudaStreamSynchronize(c->stream), "stream synchronize");
  dfree(c, state);
  const cg::DevError e = *c->h_err;
  if (e.err == cg::DERR_TIMEOUT && e.where == cg::K_SELFTEST_WAIT)
    return fail(c, CG_ETIMEOUT, "device wait timed out in kernel %d at tile %lld (self-test)", e.where, e.index);
  return fail(c, CG_EKERNEL, "self-test: the withheld tile's wait did not run out (error %d, kernel %d)", e.err,
              e.where);
}

cg_status cg_free_graph(cg_graph* g) {
  if (!g) return CG_EINVAL;
  cg_ctx* c = g->ctx;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);   // buffers may still be in use by queued work
  for (StageExec& e : g->execs)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  for (void* p : g->owned) dfree(c, p);
  dfree(c, g->stage_bases);
  dfree(c, g->hb_dst);
  dfree(c, g->part_buf);
  delete g;
  return CG_OK;
}

cg_status cg_load_graph(cg_ctx* c, const cg_graph_desc* d, uint32_t flags, cg_graph** out) {
  Range range("cg.load_graph");
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (!d || !out) return fail(c, CG_EINVAL, "null argument");
  *out = nullptr;
  const int64_t n = d->n_reads, m = d->n_entries;
  if (n < 0 || n >= (1ll << 30)) return fail(c, CG_EINVAL, "n_reads out of range");
  if (m < 0 || m >= (1ll << 31)) return fail(c, CG_EINVAL, "n_entries out of range");
  if (d->row_ptr_bytes != 4 && d->row_ptr_bytes != 8) return fail(c, CG_EINVAL, "row_ptr_bytes must be 4 or 8");
  if (d->mem != CG_MEM_HOST && d->mem != CG_MEM_DEVICE) return fail(c, CG_EINVAL, "bad mem");
  const bool xdrop = d->pre && d->post;
  const bool no_reads = (flags & CG_NO_READS) != 0;
  if (no_reads && (d->packed || (flags & CG_HOST_READS)))
    return fail(c, CG_EINVAL, "CG_NO_READS takes no packed reads (packed_bytes gives the virtual stream's size)");
  if (!d->row_ptr || (m > 0 && (!d->col || !d->code || (!xdrop && !d->suf))) || (n > 0 && (!d->len || !d->off)) ||
      d->packed_bytes < 0 || (d->packed_bytes > 0 && !d->packed && !no_reads))
    return fail(c, CG_EINVAL, "missing input array");
  const bool borrow = (flags & CG_BORROW_DEVICE) != 0;
  if (borrow && d->mem != CG_MEM_DEVICE) return fail(c, CG_EINVAL, "CG_BORROW_DEVICE needs device inputs");
  const bool host_reads = (flags & CG_HOST_READS) != 0;
  const uint8_t* host_packed_dev = nullptr;      // device address of pinned host reads
  if (host_reads) {
    if (borrow || d->mem != CG_MEM_HOST) return fail(c, CG_EINVAL, "CG_HOST_READS needs host inputs");
    host_packed_dev = (const uint8_t*)pinned_device_alias(d->packed);
    if (d->packed_bytes > 0 && !host_packed_dev)
      return fail(c, CG_EINVAL, "CG_HOST_READS needs the packed reads in pinned host memory");
  }
  if (borrow && ((!no_reads && !aligned(d->packed, 16)) || !aligned(d->row_ptr, d->row_ptr_bytes) || !aligned(d->col, 4) ||
                 (!xdrop && !aligned(d->suf, 4)) || (xdrop && (!aligned(d->pre, 4) || !aligned(d->post, 4))) ||
                 !aligned(d->len, 4) || !aligned(d->off, 8)))
    return fail(c, CG_EINVAL, "borrowed device inputs are misaligned");

  cg_graph* g = new (std::nothrow) cg_graph();
  if (!g) return fail(c, CG_ENOMEM, "host allocation");
  g->ctx = c;
  auto bail = [&](cg_status s) {
    cg_free_graph(g);
    return s;
  };
  st = CG_OK;
  const cudaMemcpyKind kind = d->mem == CG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cg::DevGraph& G = g->g;
  G.n = n;
  G.m = m;
  G.rp64 = d->row_ptr_bytes == 8;
  G.min_chain = d->min_chain_reads <= 0 ? 2 : d->min_chain_reads;
  G.packed_bytes = d->packed_bytes;
  G.packed_readable = borrow || host_reads ? d->packed_bytes : d->packed_bytes + 16;   // owned copies: 16 zero bytes
  G.no_reads = no_reads;
  if (no_reads) G.packed_readable = 0;
  if (borrow) {
    G.row_ptr = d->row_ptr;
    G.col = d->col;
    G.code = d->code;
    G.suf = xdrop ? nullptr : d->suf;
    G.pre = xdrop ? d->pre : nullptr;
    G.post = xdrop ? d->post : nullptr;
    G.len = d->len;
    G.off = d->off;
    G.packed = d->packed;
  } else {
    auto copy_in = [&](const void* src, size_t bytes, size_t pad) -> const void* {
      void* p = dalloc(c, bytes + pad, &st);
      if (!p) return nullptr;
      g->owned.push_back(p);
      if (c->fault.hit("h2d")) {
        st = fail(c, CG_ECUDA, "injected: copy graph input failed");
        return nullptr;
      }
      if (bytes) {
        cudaError_t e = cudaMemcpyAsync(p, src, bytes, kind, c->stream);
        if (e != cudaSuccess) { st = cuda_fail(c, e, "copy graph input"); return nullptr; }
      }
      if (pad) cudaMemsetAsync((char*)p + bytes, 0, pad, c->stream);
      return p;
    };
    G.row_ptr = copy_in(d->row_ptr, (size_t)(n + 1) * d->row_ptr_bytes, 0);
    if (st == CG_OK) G.col = (const int32_t*)copy_in(d->col, (size_t)m * 4, 0);
    if (st == CG_OK) G.code = (const uint8_t*)copy_in(d->code, (size_t)m, 0);
    if (xdrop) {
      if (st == CG_OK) G.pre = (const int32_t*)copy_in(d->pre, (size_t)m * 4, 0);
      if (st == CG_OK) G.post = (const int32_t*)copy_in(d->post, (size_t)m * 4, 0);
    } else if (st == CG_OK) {
      G.suf = (const int32_t*)copy_in(d->suf, (size_t)m * 4, 0);
    }
    if (st == CG_OK) G.len = (const int32_t*)copy_in(d->len, (size_t)n * 4, 0);
    if (st == CG_OK) G.off = (const int64_t*)copy_in(d->off, (size_t)n * 8, 0);
    if (host_reads) {
      G.packed = host_packed_dev;
      G.packed_host = true;
    } else if (no_reads) {
      G.packed = nullptr;
    } else if (st == CG_OK) {
      G.packed = (const uint8_t*)copy_in(d->packed, (size_t)d->packed_bytes, 16);
    }
    if (st != CG_OK) return bail(st);
  }

  st = finish_load(g, flags);
  if (st != CG_OK) return bail(st);
  *out = g;
  return CG_OK;
}

cg_status cg_load_batch(cg_ctx* c, const cg_graph_desc* d, int k, uint32_t flags, cg_graph** out) {
  Range range("cg.load_batch");
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (!d || !out || k < 1) return fail(c, CG_EINVAL, "null argument or empty batch");
  *out = nullptr;
  if (flags & CG_BORROW_DEVICE) return fail(c, CG_EINVAL, "a batch is always copied into one union graph");
  if (flags & CG_NO_READS) return fail(c, CG_EINVAL, "a batch takes its graphs' reads");
  const bool host_reads = (flags & CG_HOST_READS) != 0;
  std::vector<const uint8_t*> alias(host_reads ? k : 0, nullptr);
  std::vector<int64_t> gbytes(host_reads ? k : 0, 0);
  if (host_reads) {
    for (int j = 0; j < k; ++j) {
      if (d[j].mem != CG_MEM_HOST) return fail(c, CG_EINVAL, "CG_HOST_READS needs host inputs");
      gbytes[j] = d[j].packed_bytes;
      if (d[j].packed_bytes == 0) continue;
      alias[j] = (const uint8_t*)pinned_device_alias(d[j].packed);
      if (!alias[j]) return fail(c, CG_EINVAL, "graph %d: CG_HOST_READS needs its reads in pinned host memory", j);
      if (!aligned(alias[j], 4)) return fail(c, CG_EINVAL, "graph %d: pinned reads must start 4-byte aligned", j);
    }
  }
  const int mem = d[0].mem, rpb = d[0].row_ptr_bytes, mcr = d[0].min_chain_reads;
  const bool xdrop = d[0].pre && d[0].post;
  std::vector<int64_t> R(k + 1, 0), E(k + 1, 0), PB(k + 1, 0), SR(k + 1, 0);
  for (int j = 0; j < k; ++j) {
    const cg_graph_desc& q = d[j];
    if (q.mem != mem || q.row_ptr_bytes != rpb || q.min_chain_reads != mcr || (q.pre && q.post) != xdrop)
      return fail(c, CG_EINVAL, "graph %d: mem, row_ptr_bytes, min_chain_reads and the overlap form must match", j);
    if ((rpb != 4 && rpb != 8) || (mem != CG_MEM_HOST && mem != CG_MEM_DEVICE)) return fail(c, CG_EINVAL, "bad desc");
    if (q.n_reads < 0 || q.n_entries < 0 || q.packed_bytes < 0 || !q.row_ptr ||
        (q.n_entries > 0 && (!q.col || !q.code || (!xdrop && !q.suf))) || (q.n_reads > 0 && (!q.len || !q.off)) ||
        (q.packed_bytes > 0 && !q.packed))
      return fail(c, CG_EINVAL, "graph %d: missing input array", j);
    R[j + 1] = R[j] + q.n_reads;
    E[j + 1] = E[j] + q.n_entries;
    PB[j + 1] = PB[j] + (q.packed_bytes + 15) / 16 * 16;   // each graph's bases start 16-byte aligned
    SR[j + 1] = SR[j] + q.n_reads + 1;
  }
  const int64_t n = R[k], m = E[k];
  if (n >= (1ll << 30) || m >= (1ll << 31)) return fail(c, CG_EINVAL, "batch too large");
  cg_graph* g = new (std::nothrow) cg_graph();
  if (!g) return fail(c, CG_ENOMEM, "host allocation");
  g->ctx = c;
  auto bail = [&](cg_status s2) {
    cg_free_graph(g);
    return s2;
  };
  const cudaMemcpyKind kind = mem == CG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cg::DevGraph& G = g->g;
  G.n = n;
  G.m = m;
  G.rp64 = 1;
  G.min_chain = mcr <= 0 ? 2 : mcr;
  G.packed_bytes = PB[k];
  G.packed_readable = PB[k] + 16;
  int64_t* rp = galloc<int64_t>(g, (size_t)n + 1, &st);
  int32_t* col = galloc<int32_t>(g, (size_t)(m > 0 ? m : 1), &st);
  uint8_t* code = galloc<uint8_t>(g, (size_t)(m > 0 ? m : 1), &st);
  int32_t* suf = xdrop ? nullptr : galloc<int32_t>(g, (size_t)(m > 0 ? m : 1), &st);
  int32_t* pre = xdrop ? galloc<int32_t>(g, (size_t)(m > 0 ? m : 1), &st) : nullptr;
  int32_t* post = xdrop ? galloc<int32_t>(g, (size_t)(m > 0 ? m : 1), &st) : nullptr;
  int32_t* len = galloc<int32_t>(g, (size_t)(n > 0 ? n : 1), &st);
  int64_t* off = galloc<int64_t>(g, (size_t)(n > 0 ? n : 1), &st);
  uint8_t* packed = host_reads ? nullptr : galloc<uint8_t>(g, (size_t)PB[k] + 16, &st);
  const uint8_t** hb_base = host_reads ? galloc<const uint8_t*>(g, (size_t)k, &st) : nullptr;
  int64_t* hb_bytes = host_reads ? galloc<int64_t>(g, (size_t)k, &st) : nullptr;
  void* stage_rp = dalloc(c, (size_t)SR[k] * rpb, &st);
  int64_t* tab = galloc<int64_t>(g, 4 * (size_t)(k + 1), &st);
  if (st != CG_OK) { dfree(c, stage_rp); return bail(st); }
  g->batch_k = k;
  g->batch_R = tab;
  if (!host_reads) CK(cudaMemsetAsync(packed, 0, (size_t)PB[k] + 16, c->stream), "clear packed");
  // Host inputs all in pinned memory: one kernel reads the graph arrays in place
  // (a copy call per graph and array costs a few microseconds of host time
  // each, which dominates a batch of hundreds of small graphs); the packed
  // reads, when copied, go by the copy engines, which move large arrays over
  // the host link faster than the kernel. Otherwise a copy per array.
  std::vector<cg::CopySeg> segs;
  bool in_place = mem == CG_MEM_HOST;
  for (int j = 0; j < k && in_place; ++j) {
    const cg_graph_desc& q = d[j];
    auto add = [&](void* dst, const void* src, long long bytes) {
      if (!in_place || bytes <= 0) return;
      const uint8_t* a = (const uint8_t*)pinned_device_alias(src);
      if (!a) { in_place = false; return; }
      const long long kPiece = 256 << 10;               // long arrays in pieces, to spread them over warps
      for (long long o = 0; o < bytes; o += kPiece)
        segs.push_back({a + o, (uint8_t*)dst + o, std::min(kPiece, bytes - o)});
    };
    add((char*)stage_rp + (size_t)SR[j] * rpb, q.row_ptr, (q.n_reads + 1) * (long long)rpb);
    add(col + E[j], q.col, q.n_entries * 4ll);
    add(code + E[j], q.code, q.n_entries);
    if (!xdrop) add(suf + E[j], q.suf, q.n_entries * 4ll);
    if (xdrop) add(pre + E[j], q.pre, q.n_entries * 4ll);
    if (xdrop) add(post + E[j], q.post, q.n_entries * 4ll);
    add(len + R[j], q.len, q.n_reads * 4ll);
    add(off + R[j], q.off, q.n_reads * 8ll);
  }
  cg::CopySeg* d_segs = nullptr;
  if (in_place) {
    cudaError_t e = cudaSuccess;
    if (!segs.empty()) {
      d_segs = (cg::CopySeg*)dalloc(c, segs.size() * sizeof(cg::CopySeg), &st);
      if (!d_segs) { dfree(c, stage_rp); return bail(st); }
      e = cudaMemcpyAsync(d_segs, segs.data(), segs.size() * sizeof(cg::CopySeg), cudaMemcpyHostToDevice, c->stream);
      if (e == cudaSuccess) e = cg::launch_batch_copy(d_segs, (int)segs.size(), c->env);
    }
    for (int j = 0; j < k && e == cudaSuccess && !host_reads; ++j)
      if (d[j].packed_bytes > 0)
        e = cudaMemcpyAsync(packed + PB[j], d[j].packed, (size_t)d[j].packed_bytes, kind, c->stream);
    if (e != cudaSuccess) {
      if (d_segs) dfree(c, d_segs);
      dfree(c, stage_rp);
      return bail(cuda_fail(c, e, "copy batch input"));
    }
  }
  for (int j = 0; j < k && !in_place; ++j) {
    const cg_graph_desc& q = d[j];
    auto cp = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
      return bytes ? cudaMemcpyAsync(dst, src, bytes, kind, c->stream) : cudaSuccess;
    };
    cudaError_t e = cp((char*)stage_rp + (size_t)SR[j] * rpb, q.row_ptr, (size_t)(q.n_reads + 1) * rpb);
    if (e == cudaSuccess) e = cp(col + E[j], q.col, (size_t)q.n_entries * 4);
    if (e == cudaSuccess) e = cp(code + E[j], q.code, (size_t)q.n_entries);
    if (e == cudaSuccess && !xdrop) e = cp(suf + E[j], q.suf, (size_t)q.n_entries * 4);
    if (e == cudaSuccess && xdrop) e = cp(pre + E[j], q.pre, (size_t)q.n_entries * 4);
    if (e == cudaSuccess && xdrop) e = cp(post + E[j], q.post, (size_t)q.n_entries * 4);
    if (e == cudaSuccess) e = cp(len + R[j], q.len, (size_t)q.n_reads * 4);
    if (e == cudaSuccess) e = cp(off + R[j], q.off, (size_t)q.n_reads * 8);
    if (e == cudaSuccess && !host_reads) e = cp(packed + PB[j], q.packed, (size_t)q.packed_bytes);
    if (e != cudaSuccess) { dfree(c, stage_rp); return bail(cuda_fail(c, e, "copy batch input")); }
  }
  std::vector<int64_t> host_tab;
  host_tab.insert(host_tab.end(), R.begin(), R.end());
  host_tab.insert(host_tab.end(), E.begin(), E.end());
  host_tab.insert(host_tab.end(), PB.begin(), PB.end());
  host_tab.insert(host_tab.end(), SR.begin(), SR.end());
  CK(cudaMemcpyAsync(tab, host_tab.data(), host_tab.size() * 8, cudaMemcpyHostToDevice, c->stream), "copy tables");
  if (host_reads) {
    CK(cudaMemcpyAsync(hb_base, alias.data(), (size_t)k * sizeof(void*), cudaMemcpyHostToDevice, c->stream),
       "copy read stream table");
    CK(cudaMemcpyAsync(hb_bytes, gbytes.data(), (size_t)k * 8, cudaMemcpyHostToDevice, c->stream),
       "copy read stream table");
  }
  CK(cg::launch_batch_fixup(k, tab, tab + (k + 1), tab + 2 * (k + 1), tab + 3 * (k + 1), stage_rp, rpb, rp, col, off,
                            n, m, c->env), "batch fixup");
  CK(cudaStreamSynchronize(c->stream), "stream synchronize");   // host_tab and segs are read by the copies above
  dfree(c, stage_rp);
  if (d_segs) dfree(c, d_segs);
  G.row_ptr = rp;
  G.col = col;
  G.code = code;
  G.suf = suf;
  G.pre = pre;
  G.post = post;
  G.len = len;
  G.off = off;
  G.packed = packed;
  if (host_reads) {
    g->host_batch = true;
    g->hb_base = hb_base;
    g->hb_bytes = hb_bytes;
    g->hb_PB = tab + 2 * (k + 1);
    G.packed_readable = 0;          // no union stream on the device: the spelling reads gathered pieces
  }
  st = finish_load(g, flags);
  if (st != CG_OK) return bail(st);
  *out = g;
  return CG_OK;
}

cg_status cg_batch_ranges(cg_graph* g, int64_t* first_contig, int64_t* first_base, int mem) {
  if (!g) return CG_EINVAL;
  cg_ctx* c = g->ctx;
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (g->batch_k < 1) return fail(c, CG_EINVAL, "not a batch");
  if (mem != CG_MEM_HOST && mem != CG_MEM_DEVICE) return fail(c, CG_EINVAL, "bad mem");
  if (g->stage < 3) {
    st = run_offsets(g);
    if (st != CG_OK) return st;
  }
  const int k = g->batch_k;
  if (mem == CG_MEM_DEVICE) {
    CK(cg::launch_batch_ranges(g->s, k, g->batch_R, g->g.n, first_contig, first_base, c->env), "batch ranges");
    return CG_OK;
  }
  int64_t* tmp = (int64_t*)dalloc(c, 16 * (size_t)(k + 1), &st);
  if (!tmp) return st;
  cudaError_t e = cg::launch_batch_ranges(g->s, k, g->batch_R, g->g.n, tmp, tmp + (k + 1), c->env);
  if (e == cudaSuccess && first_contig)
    e = cudaMemcpyAsync(first_contig, tmp, 8 * (size_t)(k + 1), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && first_base)
    e = cudaMemcpyAsync(first_base, tmp + (k + 1), 8 * (size_t)(k + 1), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dfree(c, tmp);
  if (e != cudaSuccess) return cuda_fail(c, e, "batch ranges");
  return wait_and_read(g);
}

cg_status cg_mask_branches(cg_graph* g, uint8_t* is_branch, int mem, int64_t* n_branch) {
  if (!g) return CG_EINVAL;
  cg_ctx* c = g->ctx;
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (mem != CG_MEM_HOST && mem != CG_MEM_DEVICE) return fail(c, CG_EINVAL, "bad mem");
  if (!is_branch && !n_branch && defer_ok(c)) {   // nothing to return: launched with the next call
    g->stage = 0;
    g->want = 1;
    return CG_OK;
  }
  g->want = 0;
  st = run_mask(g);
  if (st != CG_OK) return st;
  if (is_branch && g->g.n > 0)
    CK(cudaMemcpyAsync(is_branch, g->s.branch, (size_t)g->g.n,
                       mem == CG_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream),
       "copy is_branch");
  if (n_branch || (is_branch && mem == CG_MEM_HOST)) {
    st = wait_and_read(g);
    if (st != CG_OK) return st;
    if (n_branch) *n_branch = (int64_t)c->h_ctr->n_branch;
  }
  return CG_OK;
}

cg_status cg_chains(cg_graph* g, int32_t* chain_id, int32_t* rank, uint8_t* orient, int mem, int64_t* n_contigs,
                    int64_t* n_cycles) {
  if (!g) return CG_EINVAL;
  cg_ctx* c = g->ctx;
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (mem != CG_MEM_HOST && mem != CG_MEM_DEVICE) return fail(c, CG_EINVAL, "bad mem");
  if (!chain_id && !rank && !orient && !n_contigs && !n_cycles && defer_ok(c)) {
    if (g->stage > 1) g->stage = 1;        // nothing to return: launched with the next call
    g->want = 2;
    return CG_OK;
  }
  if (g->want) {
    st = flush(g);
    if (st != CG_OK) return st;
  }
  st = run_chains(g);
  if (st != CG_OK) return st;
  const int64_t n = g->g.n;
  const bool want_reads = chain_id || rank || orient;
  if (want_reads && n > 0) {
    if (mem == CG_MEM_DEVICE) {
      CK(cg::launch_export_reads(g->g, g->s, chain_id, rank, orient, c->env), "export reads");
    } else {
      if (!g->stage_reads) {
        g->stage_reads = dalloc(c, (size_t)n * 9, &st);
        if (!g->stage_reads) return st;
        g->owned.push_back(g->stage_reads);
      }
      int32_t* dc = (int32_t*)g->stage_reads;
      int32_t* dr = dc + n;
      uint8_t* dor = (uint8_t*)(dr + n);
      CK(cg::launch_export_reads(g->g, g->s, dc, dr, dor, c->env), "export reads");
      if (chain_id) CK(cudaMemcpyAsync(chain_id, dc, (size_t)n * 4, cudaMemcpyDeviceToHost, c->stream), "copy chain_id");
      if (rank) CK(cudaMemcpyAsync(rank, dr, (size_t)n * 4, cudaMemcpyDeviceToHost, c->stream), "copy rank");
      if (orient) CK(cudaMemcpyAsync(orient, dor, (size_t)n, cudaMemcpyDeviceToHost, c->stream), "copy orient");
    }
  }
  if (n_contigs || n_cycles || (want_reads && mem == CG_MEM_HOST)) {
    st = wait_and_read(g);
    if (st != CG_OK) return st;
    if (n_contigs) *n_contigs = (int64_t)c->h_ctr->n_lone + (int64_t)c->h_ctr->n_heads;
    if (n_cycles) *n_cycles = (int64_t)c->h_ctr->n_cycles;
  }
  return CG_OK;
}

cg_status cg_emit_contigs(cg_graph* g, int64_t* contig_off, int64_t contig_off_cap, uint8_t* bases,
                          int64_t bases_cap, int mem, int64_t* n_contigs, int64_t* total_bases) {
  if (!g) return CG_EINVAL;
  cg_ctx* c = g->ctx;
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (g->g.no_reads && bases)
    return fail(c, CG_EINVAL, "the graph was loaded without its reads: spell a share with cg_emit_share_received");
  if (mem != CG_MEM_HOST && mem != CG_MEM_DEVICE) return fail(c, CG_EINVAL, "bad mem");
  if ((bases && bases_cap < 0) || (contig_off && contig_off_cap < 1)) return fail(c, CG_EINVAL, "bad capacity");
  if (mem == CG_MEM_DEVICE && bases && !g->host_batch) {
    // the layout, the spelling and the offsets export replayed as one graph;
    // with the mask and chain launches too when both wait (a whole step in one)
    if (!aligned(bases, 16)) return fail(c, CG_EINVAL, "device bases buffer must be 16-byte aligned");
    const bool whole = g->want == 2 && g->stage == 0 && defer_ok(c);
    if (!whole) {
      if (g->want) {
        st = flush(g);
        if (st != CG_OK) return st;
      }
      if (g->stage < 2) {
        st = run_chains(g);
        if (st != CG_OK) return st;
      }
    }
    g->want = 0;
    const bool timing = c->timing != 0, stages = timing && !c->timing_emit_only;
    uint64_t key = mix_key(mix_key(mix_key(mix_key((uint64_t)(uintptr_t)bases, (uint64_t)bases_cap),
                                           (uint64_t)(uintptr_t)g->g.packed), (uint64_t)gt(g).tile_bytes),
                           (uint64_t)cg::emit_launch_key(gt(g)));
    key = mix_key(mix_key(mix_key(key, (uint64_t)(uintptr_t)contig_off), (uint64_t)contig_off_cap),
                  stages ? 3 : (timing ? 5 : 4));
    if (whole) key = mix_key(key, (uint64_t)gt(g).ruler_log2);
    // the caller's contig offsets come from the piece scan itself (no copy kernel)
    const bool fold_off = contig_off && g->g.n > 0;
    st = run_stage(g, whole ? 7 : 6, key, [&]() -> cg_status {
      if (whole) {
        CK(cg::launch_mask(g->g, g->s, c->env), "mask kernels");
        CK(cg::launch_chains(g->g, g->s, gt(g), c->env), "chain kernels");
      }
      if (stages) record_stage_event(c, 4);
      CK(cg::launch_offsets(g->g, g->s, gt(g), c->env, fold_off ? contig_off : nullptr,
                            fold_off ? contig_off_cap : 0), "offset kernels");
      if (stages) record_stage_event(c, 5);
      if (timing) record_stage_event(c, 6);
      cg::LaunchEnv env = c->env;
      env.pdl_first = !timing;           // no event node between these kernels and the ones before
      CK(cg::launch_emit(g->g, g->s, gt(g), bases, bases_cap, env), "emission kernel");
      if (timing) record_stage_event(c, 7);
      if (contig_off && !fold_off)
        CK(cg::launch_export_contig_off(g->s, contig_off, contig_off_cap, env), "export contig_off");
      return CG_OK;
    });
    if (st != CG_OK) return st;
    if (stages) c->recorded[2] = true;
    if (timing) c->recorded[3] = true;
    g->stage = 3;
    if (n_contigs || total_bases) {
      st = wait_and_read(g);
      if (st != CG_OK) return st;
    }
    if (n_contigs) *n_contigs = (int64_t)c->h_ctr->n_contigs;
    if (total_bases) *total_bases = c->h_ctr->total_bases;
    return CG_OK;
  }
  st = run_offsets(g);
  if (st != CG_OK) return st;
  // Large outputs into host memory are spelled and copied in chunks of tiles
  // (below); a batch with host-resident reads then gathers each chunk's
  // pieces just before spelling it, so that the gathers, which read the host
  // link, overlap the copies of earlier chunks, which write it.
  const int64_t kPipelineMin = 64ll << 20, kChunk = 128ll << 20;
  bool chunk_gather = false;
  if (bases) {
    if (g->host_batch && mem == CG_MEM_HOST) {
      st = wait_and_read(g);
      if (st != CG_OK) return st;
      chunk_gather = c->h_ctr->total_bases >= kPipelineMin;
    }
    st = prepare_emit(g, !chunk_gather);
    if (st != CG_OK) return st;
  }
  if (mem == CG_MEM_DEVICE) {
    if (bases) {
      if (!aligned(bases, 16)) return fail(c, CG_EINVAL, "device bases buffer must be 16-byte aligned");
      StageTimer tm(c, 3);
      uint64_t key = mix_key(mix_key(mix_key(mix_key((uint64_t)(uintptr_t)bases, (uint64_t)bases_cap),
                                             (uint64_t)(uintptr_t)emit_graph(g).packed), (uint64_t)gt(g).tile_bytes),
                             (uint64_t)cg::emit_launch_key(gt(g)));
      st = run_stage(g, 3, key, [&]() -> cg_status {
        CK(cg::launch_emit(emit_graph(g), g->s, gt(g), bases, bases_cap, c->env), "emission kernel");
        return CG_OK;
      });
      if (st != CG_OK) return st;
    }
    if (contig_off) {
      st = run_stage(g, 4, mix_key((uint64_t)(uintptr_t)contig_off, (uint64_t)contig_off_cap), [&]() -> cg_status {
        CK(cg::launch_export_contig_off(g->s, contig_off, contig_off_cap, c->env), "export contig_off");
        return CG_OK;
      });
      if (st != CG_OK) return st;
    }
    if (n_contigs || total_bases) {
      st = wait_and_read(g);
      if (st != CG_OK) return st;
    }
  } else {
    st = wait_and_read(g);
    if (st != CG_OK) return st;
    const int64_t total = c->h_ctr->total_bases, C = c->h_ctr->n_contigs;
    if (bases && bases_cap < total) return fail(c, CG_EINVAL, "bases capacity %lld < %lld", (long long)bases_cap, (long long)total);
    if (contig_off && contig_off_cap < C + 1) return fail(c, CG_EINVAL, "contig_off capacity too small");
    // Large outputs: spelled into HBM in chunks of tiles, each chunk copied to
    // the host by the copy engines while the next one is spelled (the host
    // link, not the spelling, bounds the step). Smaller ones, when pinned: the
    // kernel writes them over the host link in place; otherwise staged and
    // copied once.
    const bool pipelined = bases && total >= kPipelineMin;
    uint8_t* direct = c->host_direct && !pipelined ? (uint8_t*)pinned_device_alias(bases) : nullptr;
    if (direct && !aligned(direct, 16)) direct = nullptr;
    if (pipelined) {
      if (g->stage_bases_cap < total) {
        if (g->stage_bases) dfree(c, g->stage_bases);
        g->stage_bases = (uint8_t*)dalloc(c, (size_t)total, &st);
        if (!g->stage_bases) { g->stage_bases_cap = 0; return st; }
        g->stage_bases_cap = total;
      }
      if (!c->copy_stream) {
        CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking), "copy stream");
        CK(cudaEventCreateWithFlags(&c->copy_ev, cudaEventDisableTiming), "copy event");
      }
      StageTimer tm(c, 3);
      const int64_t tb = gt(g).tile_bytes;
      const int64_t tiles = (total + tb - 1) / tb, per = std::max<int64_t>(1, kChunk / tb);
      for (int64_t t0 = 0; t0 < tiles; t0 += per) {
        const int64_t t1 = std::min(tiles, t0 + per);
        const int64_t b0 = t0 * tb, b1 = std::min(total, t1 * tb);
        if (chunk_gather)
          CK(cg::launch_gather_pieces(g->s, g->batch_k, g->hb_PB, g->hb_base, g->hb_bytes, g->hb_slot, g->hb_dst,
                                      g->hb_dst_words, c->h_ctr->n_walk, c->env, t0, t1), "gather pieces");
        CK(cg::launch_emit(emit_graph(g), g->s, gt(g), g->stage_bases, g->stage_bases_cap, c->env, t0, t1),
           "emission kernel");
        CK(cudaEventRecord(c->copy_ev, c->stream), "chunk event");
        CK(cudaStreamWaitEvent(c->copy_stream, c->copy_ev, 0), "copy stream wait");
        CK(cudaMemcpyAsync(bases + b0, g->stage_bases + b0, (size_t)(b1 - b0), cudaMemcpyDeviceToHost,
                           c->copy_stream), "copy bases");
      }
      CK(cudaEventRecord(c->copy_ev, c->copy_stream), "copies done");
      CK(cudaStreamWaitEvent(c->stream, c->copy_ev, 0), "stream waits for the copies");
    } else if (bases && total > 0) {
      uint8_t* dst = direct;
      int64_t dcap = bases_cap;
      if (!dst) {
        if (g->stage_bases_cap < total) {
          if (g->stage_bases) dfree(c, g->stage_bases);
          g->stage_bases = (uint8_t*)dalloc(c, (size_t)total, &st);
          if (!g->stage_bases) { g->stage_bases_cap = 0; return st; }
          g->stage_bases_cap = total;
        }
        dst = g->stage_bases;
        dcap = g->stage_bases_cap;
      }
      {
        StageTimer tm(c, 3);
        uint64_t key = mix_key(mix_key(mix_key(mix_key((uint64_t)(uintptr_t)dst, (uint64_t)dcap),
                                           (uint64_t)(uintptr_t)emit_graph(g).packed),
                                       (uint64_t)gt(g).tile_bytes), (uint64_t)cg::emit_launch_key(gt(g)));
        st = run_stage(g, 3, key, [&]() -> cg_status {
          CK(cg::launch_emit(emit_graph(g), g->s, gt(g), dst, dcap, c->env), "emission kernel");
          return CG_OK;
        });
        if (st != CG_OK) return st;
      }
      if (!direct) CK(cudaMemcpyAsync(bases, dst, (size_t)total, cudaMemcpyDeviceToHost, c->stream), "copy bases");
    }
    if (contig_off)
      CK(cudaMemcpyAsync(contig_off, g->s.contig_off, (size_t)(C + 1) * 8, cudaMemcpyDeviceToHost, c->stream),
         "copy contig_off");
    if (bases || contig_off) {
      st = wait_and_read(g);
      if (st != CG_OK) return st;
    }
  }
  if (n_contigs) *n_contigs = (int64_t)c->h_ctr->n_contigs;
  if (total_bases) *total_bases = c->h_ctr->total_bases;
  return CG_OK;
}

cg_status cg_emit_part(cg_graph* g, const int32_t* part, int64_t part_cap, int32_t p, int64_t* contig_off,
                       int64_t contig_off_cap, uint8_t* bases, int64_t bases_cap, int mem, int64_t* n_contigs,
                       int64_t* total_bases) {
  if (!g) return CG_EINVAL;
  cg_ctx* c = g->ctx;
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (g->g.no_reads && bases)
    return fail(c, CG_EINVAL, "the graph was loaded without its reads: spell a share with cg_emit_share_received");
  if (mem != CG_MEM_HOST && mem != CG_MEM_DEVICE) return fail(c, CG_EINVAL, "bad mem");
  if (g->host_batch) return fail(c, CG_EINVAL, "cg_emit_part: not for a batch with host-resident reads");
  if (g->stage < 2) {                  // the contig count: lone reads and chain heads
    st = run_chains(g);
    if (st != CG_OK) return st;
  }
  st = wait_and_read(g);
  if (st != CG_OK) return st;
  const int64_t C = (int64_t)c->h_ctr->n_lone + (int64_t)c->h_ctr->n_heads;
  if (C > 0 && (!part || part_cap < C)) return fail(c, CG_EINVAL, "part capacity %lld < %lld", (long long)part_cap,
                                                    (long long)C);
  const int32_t* d_part = part;
  if (C > 0 && mem == CG_MEM_HOST) {
    if (g->part_buf_cap < C) {
      if (g->part_buf) dfree(c, g->part_buf);
      g->part_buf = (int32_t*)dalloc(c, (size_t)C * 4, &st);
      g->part_buf_cap = g->part_buf ? C : 0;
      if (!g->part_buf) return st;
    }
    CK(cudaMemcpyAsync(g->part_buf, part, (size_t)C * 4, cudaMemcpyHostToDevice, c->stream), "copy part");
    d_part = g->part_buf;
  }
  g->s.part = C > 0 ? d_part : nullptr;
  g->s.part_p = C > 0 ? p : 0;
  g->stage = 2;                        // the offsets stage runs again, on the part's layout
  st = cg_emit_contigs(g, contig_off, contig_off_cap, bases, bases_cap, mem, n_contigs, total_bases);
  g->s.part = nullptr;
  g->s.part_p = 0;
  g->stage = 2;                        // the layout on the device is the part's: a later call redoes it
  return st;
}

cg_status cg_emit_share(cg_graph* g, int32_t share, int32_t n_shares, int64_t* contig_off, int64_t contig_off_cap,
                        uint8_t* bases, int64_t bases_cap, int mem, int64_t* first_base, int64_t* n_bases) {
  if (!g) return CG_EINVAL;
  cg_ctx* c = g->ctx;
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (g->g.no_reads && bases)
    return fail(c, CG_EINVAL, "the graph was loaded without its reads: spell a share with cg_emit_share_received");
  if (mem != CG_MEM_HOST && mem != CG_MEM_DEVICE) return fail(c, CG_EINVAL, "bad mem");
  if (n_shares < 1 || share < 0 || share >= n_shares)
    return fail(c, CG_EINVAL, "share %d of %d shares", (int)share, (int)n_shares);
  if ((bases && bases_cap < 0) || (contig_off && contig_off_cap < 1)) return fail(c, CG_EINVAL, "bad capacity");
  st = run_offsets(g);
  if (st != CG_OK) return st;
  if (bases) {
    st = prepare_emit(g);
    if (st != CG_OK) return st;
  }
  // the share's stream range, from the stream's size (known on the host after a wait)
  const int64_t tb = gt(g).tile_bytes;
  auto range = [&](int64_t total, int64_t* fb, int64_t* nb) {
    const int64_t T = (total + tb - 1) / tb;
    const int64_t t0 = (int64_t)share * T / n_shares, t1 = (int64_t)(share + 1) * T / n_shares;
    *fb = t0 * tb;
    *nb = std::max<int64_t>(0, std::min(total, t1 * tb) - t0 * tb);
  };
  auto spell = [&](uint8_t* dst, int64_t cap) -> cg_status {
    StageTimer tm(c, 3);
    uint64_t key = mix_key(mix_key(mix_key(mix_key((uint64_t)(uintptr_t)dst, (uint64_t)cap),
                                           (uint64_t)(uintptr_t)emit_graph(g).packed), (uint64_t)tb),
                           (uint64_t)cg::emit_launch_key(gt(g)));
    key = mix_key(mix_key(key, (uint64_t)share), (uint64_t)n_shares);
    return run_stage(g, 3, key, [&]() -> cg_status {
      CK(cg::launch_emit(emit_graph(g), g->s, gt(g), dst, cap, c->env, 0, 1ll << 62, share, n_shares),
         "emission kernel (one share)");
      return CG_OK;
    });
  };
  int64_t fb = 0, nb = 0;
  if (mem == CG_MEM_DEVICE) {
    if (bases) {
      if (!aligned(bases, 16)) return fail(c, CG_EINVAL, "device bases buffer must be 16-byte aligned");
      st = spell(bases, bases_cap);
      if (st != CG_OK) return st;
    }
    if (contig_off) {
      st = run_stage(g, 4, mix_key((uint64_t)(uintptr_t)contig_off, (uint64_t)contig_off_cap), [&]() -> cg_status {
        CK(cg::launch_export_contig_off(g->s, contig_off, contig_off_cap, c->env), "export contig_off");
        return CG_OK;
      });
      if (st != CG_OK) return st;
    }
    if (first_base || n_bases) {
      st = wait_and_read(g);
      if (st != CG_OK) return st;
      range(c->h_ctr->total_bases, &fb, &nb);
    }
  } else {
    st = wait_and_read(g);
    if (st != CG_OK) return st;
    const int64_t C = c->h_ctr->n_contigs;
    range(c->h_ctr->total_bases, &fb, &nb);
    if (bases && bases_cap < nb) return fail(c, CG_EINVAL, "bases capacity %lld < %lld", (long long)bases_cap, (long long)nb);
    if (contig_off && contig_off_cap < C + 1) return fail(c, CG_EINVAL, "contig_off capacity too small");
    if (bases && nb > 0) {
      if (g->stage_bases_cap < nb) {
        if (g->stage_bases) dfree(c, g->stage_bases);
        g->stage_bases = (uint8_t*)dalloc(c, (size_t)nb, &st);
        if (!g->stage_bases) { g->stage_bases_cap = 0; return st; }
        g->stage_bases_cap = nb;
      }
      st = spell(g->stage_bases, g->stage_bases_cap);
      if (st != CG_OK) return st;
      CK(cudaMemcpyAsync(bases, g->stage_bases, (size_t)nb, cudaMemcpyDeviceToHost, c->stream), "copy bases");
    }
    if (contig_off)
      CK(cudaMemcpyAsync(contig_off, g->s.contig_off, (size_t)(C + 1) * 8, cudaMemcpyDeviceToHost, c->stream),
         "copy contig_off");
    if (bases || contig_off) {
      st = wait_and_read(g);
      if (st != CG_OK) return st;
    }
  }
  if (first_base) *first_base = fb;
  if (n_bases) *n_bases = nb;
  return CG_OK;
}

// ------------------------------------------------------------ read exchange
// Device state of one exchange call: the read bounds, the shares' walk
// ranges, the first pair of each share's range.
struct Xchg {
  cg::XchgArgs x{};
  std::vector<long long> range, pair0;   // host copies
  long long n_pairs = 0;
  void* mem[3] = {nullptr, nullptr, nullptr};
};

static void x_release(cg_ctx* c, Xchg& X) {
  for (void*& p : X.mem) {
    dfree(c, p);
    p = nullptr;
  }
}

// Checks the arguments, lays out the graph if needed and fills X (waits).
static cg_status x_prepare(cg_graph* g, int32_t n_shares, const int64_t* read_first, int32_t rank, Xchg& X) {
  cg_ctx* c = g->ctx;
  if (!g->g.no_reads) return fail(c, CG_EINVAL, "the read exchange is for graphs loaded with CG_NO_READS");
  if (n_shares < 1 || n_shares > CG_MAX_PARTS || rank < 0 || rank >= n_shares || !read_first)
    return fail(c, CG_EINVAL, "rank %d of %d shares", (int)rank, (int)n_shares);
  if (read_first[0] != 0 || read_first[n_shares] != g->g.n) return fail(c, CG_EINVAL, "read_first must run from 0 to n");
  for (int r = 0; r < n_shares; ++r)
    if (read_first[r + 1] < read_first[r]) return fail(c, CG_EINVAL, "read_first must not decrease");
  cg_status st = CG_OK;
  if (g->stage < 3) {                  // the layout of the last call stands unless a later step changed it
    st = run_offsets(g);
    if (st != CG_OK) return st;
  }
  const int N = n_shares;
  int64_t* rf = (int64_t*)dalloc(c, (size_t)(N + 1) * 8, &st);
  long long* range = st == CG_OK ? (long long*)dalloc(c, (size_t)2 * N * 8, &st) : nullptr;
  long long* pair0 = st == CG_OK ? (long long*)dalloc(c, (size_t)(N + 1) * 8, &st) : nullptr;
  X.mem[0] = rf;
  X.mem[1] = range;
  X.mem[2] = pair0;
  if (st != CG_OK) return st;
  CK(cudaMemcpyAsync(rf, read_first, (size_t)(N + 1) * 8, cudaMemcpyHostToDevice, c->stream), "copy read bounds");
  CK(cg::launch_x_ranges(g->s, N, gt(g).tile_bytes, range, c->env), "share ranges");
  X.range.assign((size_t)2 * N, 0);
  CK(cudaMemcpyAsync(X.range.data(), range, (size_t)2 * N * 8, cudaMemcpyDeviceToHost, c->stream), "read ranges");
  st = wait_and_read(g);
  if (st != CG_OK) return st;
  X.pair0.assign((size_t)N + 1, 0);
  for (int p = 0; p < N; ++p)
    X.pair0[p + 1] = X.pair0[p] + std::max(0ll, X.range[2 * p + 1] - X.range[2 * p] + 1);
  X.n_pairs = X.pair0[N];
  CK(cudaMemcpyAsync(pair0, X.pair0.data(), (size_t)(N + 1) * 8, cudaMemcpyHostToDevice, c->stream), "copy pairs");
  X.x.rf = rf;
  X.x.n_shares = N;
  X.x.rank = rank;
  X.x.range = range;
  X.x.pair0 = pair0;
  return CG_OK;
}

// Words sent to each share and received from each rank (host vectors; waits).
static cg_status x_sizes(cg_graph* g, Xchg& X, std::vector<unsigned long long>& send_w,
                         std::vector<unsigned long long>& recv_w) {
  cg_ctx* c = g->ctx;
  const int N = X.x.n_shares;
  cg_status st = CG_OK;
  unsigned long long* d = (unsigned long long*)dalloc(c, (size_t)2 * N * 8, &st);
  if (!d) return st;
  send_w.assign((size_t)N, 0);
  recv_w.assign((size_t)N, 0);
  cudaError_t e = cg::launch_x_sizes(g->s, X.x, d, d + N, X.n_pairs, c->env);
  if (e == cudaSuccess) e = cudaMemcpyAsync(send_w.data(), d, (size_t)N * 8, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(recv_w.data(), d + N, (size_t)N * 8, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) st = wait_and_read(g);
  dfree(c, d);
  if (e != cudaSuccess) return cuda_fail(c, e, "exchange sizes");
  return st;
}

// Per-owner exclusive scans over walk ranges: slot arrays of `count` entries.
static cg_status x_scan(cg_graph* g, Xchg& X, long long j0, long long count, int who, long long* slot) {
  cg_ctx* c = g->ctx;
  if (count <= 0) return CG_OK;
  cg_status st = CG_OK;
  const long long cap = (count + 2047) / 2048 + 1;
  unsigned long long* state = (unsigned long long*)dalloc(c, (size_t)(cap + 1) * 8, &st);
  if (!state) return st;
  cudaError_t e = cg::launch_x_scan(g->s, X.x, j0, count, who, slot, state, cap, c->env);
  dfree(c, state);                    // stream-ordered: freed after the scan
  if (e != cudaSuccess) return cuda_fail(c, e, "exchange scan");
  return CG_OK;
}

cg_status cg_exchange_sizes(cg_graph* g, int32_t n_shares, const int64_t* read_first, int32_t rank,
                            int64_t* send_bytes, int64_t* recv_bytes) {
  if (!g) return CG_EINVAL;
  cg_ctx* c = g->ctx;
  Range range("cg.exchange_sizes");
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  Xchg X;
  st = x_prepare(g, n_shares, read_first, rank, X);
  std::vector<unsigned long long> sw, rw;
  if (st == CG_OK) st = x_sizes(g, X, sw, rw);
  x_release(c, X);
  if (st != CG_OK) return st;
  for (int p = 0; p < n_shares; ++p) {
    if (send_bytes) send_bytes[p] = (int64_t)(4 * sw[p]);
    if (recv_bytes) recv_bytes[p] = (int64_t)(4 * rw[p]);
  }
  return CG_OK;
}

cg_status cg_exchange_pack(cg_graph* g, int32_t n_shares, const int64_t* read_first, int32_t rank,
                           const uint8_t* my_packed, int64_t my_packed_bytes, const int64_t* my_off, uint8_t* send_buf,
                           int64_t send_cap) {
  if (!g) return CG_EINVAL;
  cg_ctx* c = g->ctx;
  Range range("cg.exchange_pack");
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (my_packed_bytes < 0 || (my_packed_bytes > 0 && !my_packed) || send_cap < 0 || !aligned(send_buf, 4) ||
      !aligned(my_off, 8))
    return fail(c, CG_EINVAL, "bad exchange buffers");
  Xchg X;
  st = x_prepare(g, n_shares, read_first, rank, X);
  std::vector<unsigned long long> sw, rw;
  if (st == CG_OK) st = x_sizes(g, X, sw, rw);
  long long* seg = nullptr;
  long long* slot = nullptr;
  if (st == CG_OK) {
    std::vector<long long> seg_h((size_t)n_shares + 1, 0);
    for (int p = 0; p < n_shares; ++p) seg_h[p + 1] = seg_h[p] + (long long)sw[p];
    if (4 * seg_h[n_shares] > send_cap)
      st = fail(c, CG_EINVAL, "send capacity %lld < %lld", (long long)send_cap, 4 * seg_h[n_shares]);
    const long long my_reads = read_first[rank + 1] - read_first[rank];
    if (st == CG_OK && my_reads > 0 && !my_off) st = fail(c, CG_EINVAL, "my_off is required");
    if (st == CG_OK) seg = (long long*)dalloc(c, (size_t)(n_shares + 1) * 8, &st);
    if (st == CG_OK) slot = (long long*)dalloc(c, (size_t)std::max(1ll, X.n_pairs) * 8, &st);
    if (st == CG_OK && seg_h[n_shares] > 0) {
      cudaError_t e = cudaMemcpyAsync(seg, seg_h.data(), (size_t)(n_shares + 1) * 8, cudaMemcpyHostToDevice, c->stream);
      if (e != cudaSuccess) st = cuda_fail(c, e, "copy segments");
      if (st == CG_OK) {               // one scan over every share's pairs
        const long long cap = (X.n_pairs + 2047) / 2048 + 1;
        unsigned long long* state = (unsigned long long*)dalloc(c, (size_t)(cap + 1) * 8, &st);
        if (state) {
          e = cg::launch_x_scan_pairs(g->s, X.x, X.n_pairs, slot, state, cap, c->env);
          dfree(c, state);
          if (e != cudaSuccess) st = cuda_fail(c, e, "exchange scan");
        }
      }
      if (st == CG_OK) {
        e = cg::launch_x_pack(g->g, g->s, X.x, my_packed, my_packed_bytes, my_off, seg, slot,
                              reinterpret_cast<uint32_t*>(send_buf), X.n_pairs, c->env);
        if (e != cudaSuccess) st = cuda_fail(c, e, "exchange pack");
      }
      if (st == CG_OK) st = wait_and_read(g);
    }
  }
  dfree(c, seg);
  dfree(c, slot);
  x_release(c, X);
  return st;
}

cg_status cg_emit_share_received(cg_graph* g, int32_t n_shares, const int64_t* read_first, int32_t rank,
                                 const uint8_t* recv_buf, int64_t recv_bytes, int64_t* contig_off,
                                 int64_t contig_off_cap, uint8_t* bases, int64_t bases_cap, int64_t* first_base,
                                 int64_t* n_bases) {
  if (!g) return CG_EINVAL;
  cg_ctx* c = g->ctx;
  Range range("cg.emit_share_received");
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (recv_bytes < 0 || (recv_bytes > 0 && !recv_buf) || !aligned(recv_buf, 4) || (bases && !aligned(bases, 16)) ||
      (bases && bases_cap < 0) || (contig_off && contig_off_cap < 1))
    return fail(c, CG_EINVAL, "bad receive or output buffers");
  Xchg X;
  st = x_prepare(g, n_shares, read_first, rank, X);
  std::vector<unsigned long long> sw, rw;
  if (st == CG_OK) st = x_sizes(g, X, sw, rw);
  long long* seg = nullptr;
  long long* slot = nullptr;
  const long long j0 = X.range.empty() ? 0 : X.range[2 * rank];
  const long long count = st == CG_OK ? X.pair0[rank + 1] - X.pair0[rank] : 0;
  if (st == CG_OK) {
    std::vector<long long> seg_h((size_t)n_shares + 1, 0);
    for (int r = 0; r < n_shares; ++r) seg_h[r + 1] = seg_h[r] + (long long)rw[r];
    if (4 * seg_h[n_shares] != recv_bytes)
      st = fail(c, CG_EINVAL, "received %lld bytes, the layout needs %lld", (long long)recv_bytes, 4 * seg_h[n_shares]);
    if (st == CG_OK) seg = (long long*)dalloc(c, (size_t)(n_shares + 1) * 8, &st);
    if (st == CG_OK) slot = (long long*)dalloc(c, (size_t)std::max(1ll, count) * 8, &st);
    if (st == CG_OK) {
      cudaError_t e = cudaMemcpyAsync(seg, seg_h.data(), (size_t)(n_shares + 1) * 8, cudaMemcpyHostToDevice, c->stream);
      if (e != cudaSuccess) st = cuda_fail(c, e, "copy segments");
    }
    for (int r = 0; r < n_shares && st == CG_OK; ++r) st = x_scan(g, X, j0, count, r, slot);
    if (st == CG_OK && count > 0) {
      cudaError_t e = cg::launch_x_rewrite(g->s, X.x, seg, slot, c->env);
      if (e != cudaSuccess) st = cuda_fail(c, e, "exchange rewrite");
    }
  }
  if (st == CG_OK) {
    g->stage = 2;                       // the sources now point into recv_buf: a later call lays out again
    cg::DevGraph ge = g->g;
    ge.packed = recv_buf;
    ge.packed_bytes = recv_bytes;
    ge.packed_readable = recv_bytes;
    if (bases) {
      StageTimer tm(c, 3);
      cudaError_t e = cg::launch_emit(ge, g->s, gt(g), bases, bases_cap, c->env, 0, 1ll << 62, rank, n_shares);
      if (e != cudaSuccess) st = cuda_fail(c, e, "emission kernel (received share)");
    }
    if (st == CG_OK && contig_off) {
      cudaError_t e = cg::launch_export_contig_off(g->s, contig_off, contig_off_cap, c->env);
      if (e != cudaSuccess) st = cuda_fail(c, e, "export contig_off");
    }
    if (st == CG_OK) st = wait_and_read(g);
    if (st == CG_OK) {
      const int64_t tb = gt(g).tile_bytes, total = c->h_ctr->total_bases;
      const int64_t T = (total + tb - 1) / tb;
      const int64_t t0 = (int64_t)rank * T / n_shares, t1 = (int64_t)(rank + 1) * T / n_shares;
      if (first_base) *first_base = t0 * tb;
      if (n_bases) *n_bases = std::max<int64_t>(0, std::min(total, t1 * tb) - t0 * tb);
    }
  }
  dfree(c, seg);
  dfree(c, slot);
  x_release(c, X);
  return st;
}

cg_status cg_emit_contigs_2bit(cg_graph* g, int64_t* contig_off, int64_t contig_off_cap, uint8_t* packed_out,
                               int64_t packed_cap, int mem, int64_t* n_contigs, int64_t* total_bases) {
  if (!g) return CG_EINVAL;
  cg_ctx* c = g->ctx;
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (g->g.no_reads && packed_out)
    return fail(c, CG_EINVAL, "the graph was loaded without its reads: spell a share with cg_emit_share_received");
  if (mem != CG_MEM_HOST && mem != CG_MEM_DEVICE) return fail(c, CG_EINVAL, "bad mem");
  if ((packed_out && packed_cap < 0) || (contig_off && contig_off_cap < 1)) return fail(c, CG_EINVAL, "bad capacity");
  st = run_offsets(g);
  if (st != CG_OK) return st;
  if (packed_out) {
    st = prepare_emit(g);
    if (st != CG_OK) return st;
  }
  auto emit = [&](uint8_t* dst, int64_t cap) -> cg_status {
    StageTimer tm(c, 3);
    uint64_t key = mix_key(mix_key(mix_key(mix_key((uint64_t)(uintptr_t)dst, (uint64_t)cap),
                                           (uint64_t)(uintptr_t)emit_graph(g).packed), (uint64_t)gt(g).tile_bytes),
                           (uint64_t)cg::emit_launch_key(gt(g)));
    return run_stage(g, 5, key, [&]() -> cg_status {
      CK(cg::launch_emit2(emit_graph(g), g->s, gt(g), dst, cap, c->env), "2-bit emission kernel");
      return CG_OK;
    });
  };
  if (mem == CG_MEM_DEVICE) {
    if (packed_out) {
      if (!aligned(packed_out, 16)) return fail(c, CG_EINVAL, "device output buffer must be 16-byte aligned");
      st = emit(packed_out, packed_cap);
      if (st != CG_OK) return st;
    }
    if (contig_off) {
      st = run_stage(g, 4, mix_key((uint64_t)(uintptr_t)contig_off, (uint64_t)contig_off_cap), [&]() -> cg_status {
        CK(cg::launch_export_contig_off(g->s, contig_off, contig_off_cap, c->env), "export contig_off");
        return CG_OK;
      });
      if (st != CG_OK) return st;
    }
    if (n_contigs || total_bases) {
      st = wait_and_read(g);
      if (st != CG_OK) return st;
    }
  } else {
    st = wait_and_read(g);
    if (st != CG_OK) return st;
    const int64_t total = c->h_ctr->total_bases, C = c->h_ctr->n_contigs;
    const int64_t need = 16 * ((total + 63) / 64);
    if (packed_out && packed_cap < need)
      return fail(c, CG_EINVAL, "packed capacity %lld < %lld", (long long)packed_cap, (long long)need);
    if (contig_off && contig_off_cap < C + 1) return fail(c, CG_EINVAL, "contig_off capacity too small");
    // large outputs: spelled into HBM in chunks of tiles, each copied to the host
    // while the next one is spelled (as for the ASCII form)
    const int64_t kPipelineMin = 64ll << 20, kChunk = 128ll << 20;
    const bool pipelined = packed_out && need >= kPipelineMin;
    uint8_t* direct = c->host_direct && !pipelined ? (uint8_t*)pinned_device_alias(packed_out) : nullptr;
    if (direct && !aligned(direct, 16)) direct = nullptr;
    if (pipelined) {
      if (g->stage_bases_cap < need) {
        if (g->stage_bases) dfree(c, g->stage_bases);
        g->stage_bases = (uint8_t*)dalloc(c, (size_t)need, &st);
        if (!g->stage_bases) { g->stage_bases_cap = 0; return st; }
        g->stage_bases_cap = need;
      }
      if (!c->copy_stream) {
        CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking), "copy stream");
        CK(cudaEventCreateWithFlags(&c->copy_ev, cudaEventDisableTiming), "copy event");
      }
      StageTimer tm(c, 3);
      const int64_t tb = gt(g).tile_bytes, tile_out = tb / 4;   // a tile holds tb bases, tb / 4 bytes
      const int64_t tiles = (total + tb - 1) / tb, per = std::max<int64_t>(1, kChunk / tile_out);
      for (int64_t t0 = 0; t0 < tiles; t0 += per) {
        const int64_t t1 = std::min(tiles, t0 + per);
        const int64_t b0 = t0 * tile_out, b1 = std::min(need, t1 * tile_out);
        CK(cg::launch_emit2(emit_graph(g), g->s, gt(g), g->stage_bases, g->stage_bases_cap, c->env, t0, t1),
           "2-bit emission kernel");
        CK(cudaEventRecord(c->copy_ev, c->stream), "chunk event");
        CK(cudaStreamWaitEvent(c->copy_stream, c->copy_ev, 0), "copy stream wait");
        CK(cudaMemcpyAsync(packed_out + b0, g->stage_bases + b0, (size_t)(b1 - b0), cudaMemcpyDeviceToHost,
                           c->copy_stream), "copy packed");
      }
      CK(cudaEventRecord(c->copy_ev, c->copy_stream), "copies done");
      CK(cudaStreamWaitEvent(c->stream, c->copy_ev, 0), "stream waits for the copies");
    } else if (packed_out && need > 0) {
      if (direct) {
        st = emit(direct, packed_cap);
        if (st != CG_OK) return st;
      } else {
        if (g->stage_bases_cap < need) {
          if (g->stage_bases) dfree(c, g->stage_bases);
          g->stage_bases = (uint8_t*)dalloc(c, (size_t)need, &st);
          if (!g->stage_bases) { g->stage_bases_cap = 0; return st; }
          g->stage_bases_cap = need;
        }
        st = emit(g->stage_bases, g->stage_bases_cap);
        if (st != CG_OK) return st;
        CK(cudaMemcpyAsync(packed_out, g->stage_bases, (size_t)need, cudaMemcpyDeviceToHost, c->stream),
           "copy packed");
      }
    }
    if (contig_off)
      CK(cudaMemcpyAsync(contig_off, g->s.contig_off, (size_t)(C + 1) * 8, cudaMemcpyDeviceToHost, c->stream),
         "copy contig_off");
    if (packed_out || contig_off) {
      st = wait_and_read(g);
      if (st != CG_OK) return st;
    }
  }
  if (n_contigs) *n_contigs = (int64_t)c->h_ctr->n_contigs;
  if (total_bases) *total_bases = c->h_ctr->total_bases;
  return CG_OK;
}

cg_status cg_transitive_reduction(cg_ctx* c, const cg_graph_desc* d, int32_t fuzz, int64_t* row_ptr, int32_t* col,
                                  uint8_t* code, int32_t* suf, int64_t cap_entries, int mem, int64_t* n_entries) {
  Range range("cg.transitive_reduction");
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (!d) return fail(c, CG_EINVAL, "null argument");
  const int64_t n = d->n_reads, m = d->n_entries;
  if (n < 0 || n >= (1ll << 30) || m < 0 || m >= (1ll << 31)) return fail(c, CG_EINVAL, "sizes out of range");
  if (fuzz < 0) return fail(c, CG_EINVAL, "negative tolerance");
  if (mem != CG_MEM_HOST && mem != CG_MEM_DEVICE) return fail(c, CG_EINVAL, "bad mem");
  if (d->mem != CG_MEM_HOST && d->mem != CG_MEM_DEVICE) return fail(c, CG_EINVAL, "bad input mem");
  if (d->row_ptr_bytes != 4 && d->row_ptr_bytes != 8) return fail(c, CG_EINVAL, "row_ptr_bytes must be 4 or 8");
  if (d->pre || d->post) return fail(c, CG_EINVAL, "the reduction takes the suffix form");
  if (!d->row_ptr || (m > 0 && (!d->col || !d->code || !d->suf)) || (n > 0 && !d->len))
    return fail(c, CG_EINVAL, "missing input array");
  const bool want = row_ptr || col || code || suf;
  if (want && (!row_ptr || (cap_entries > 0 && (!col || !code || !suf)) || cap_entries < 0))
    return fail(c, CG_EINVAL, "outputs: row_ptr, col, code and suf together");
  // device inputs are read in place for the duration of the call; host inputs are copied
  std::vector<void*> tmp;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = dalloc(c, bytes > 0 ? bytes : 1, &st);
    if (p) tmp.push_back(p);
    return p;
  };
  auto done = [&](cg_status s2) {
    for (void* p : tmp) dfree(c, p);
    return s2;
  };
  auto in = [&](const void* src, size_t bytes) -> const void* {
    if (d->mem == CG_MEM_DEVICE) return src;
    void* p = alloc(bytes);
    if (p && bytes && cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
      st = cuda_fail(c, cudaGetLastError(), "copy overlap graph");
      return nullptr;
    }
    return p;
  };
  cg::DevGraph G{};
  G.n = n;
  G.m = m;
  G.rp64 = d->row_ptr_bytes == 8;
  G.min_chain = 2;
  G.row_ptr = in(d->row_ptr, (size_t)(n + 1) * d->row_ptr_bytes);
  G.col = (const int32_t*)in(d->col, (size_t)m * 4);
  G.code = (const uint8_t*)in(d->code, (size_t)m);
  G.suf = (const int32_t*)in(d->suf, (size_t)m * 4);
  G.len = (const int32_t*)in(d->len, (size_t)n * 4);
  cg::TrBuffers t{};
  t.row_of = (int32_t*)alloc((size_t)m * 4);
  t.trans = (uint8_t*)alloc((size_t)m);
  t.keep = (uint8_t*)alloc((size_t)m);
  t.row_cnt = (int32_t*)alloc((size_t)n * 4);
  t.out_rp = (int64_t*)alloc((size_t)(n + 1) * 8);
  t.total = (unsigned long long*)alloc(8);
  t.state_cap = (n + 2047) / 2048 + 1;
  t.state = (unsigned long long*)alloc((size_t)(t.state_cap + 1) * 8);
  t.derr = c->derr;
  if (st != CG_OK) return done(st);
  if (c->marks.on) {                   // per-kernel marks cover this call alone
    c->marks.n = 0;
    cudaEventRecord(c->marks.ev[0], c->stream);
  }
  // the rows (offsets, order), then the entries (columns, codes, suffixes,
  // mirrors), each waited for: the reduction indexes rows by column values
  cg_graph probe{};
  probe.ctx = c;
  cudaError_t e = cg::launch_transitive_check(G, c->derr, c->env);
  if (e != cudaSuccess) return done(cuda_fail(c, e, "row checks"));
  st = wait_and_read(&probe);
  if (st != CG_OK) return done(st);
  e = cg::launch_transitive_entries(G, t, c->env);
  if (e != cudaSuccess) return done(cuda_fail(c, e, "entry checks"));
  st = wait_and_read(&probe);
  if (st != CG_OK) return done(st);
  e = cg::launch_transitive(G, fuzz, t, c->env);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_u64, t.total, 8, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return done(cuda_fail(c, e, "transitive reduction kernels"));
  st = wait_and_read(&probe);
  if (st != CG_OK) return done(st);
  const int64_t total = (int64_t)*c->h_u64;
  if (n_entries) *n_entries = total;
  if (!want) return done(CG_OK);
  if (cap_entries < total) return done(fail(c, CG_EINVAL, "capacity %lld < %lld entries", (long long)cap_entries,
                                            (long long)total));
  int32_t* oc = col;
  uint8_t* ok = code;
  int32_t* os = suf;
  if (mem == CG_MEM_HOST) {
    oc = (int32_t*)alloc((size_t)total * 4);
    ok = (uint8_t*)alloc((size_t)total);
    os = (int32_t*)alloc((size_t)total * 4);
    if (st != CG_OK) return done(st);
  }
  e = cg::launch_transitive_scatter(G, t, oc, ok, os, c->env);
  const cudaMemcpyKind k = mem == CG_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (e == cudaSuccess) e = cudaMemcpyAsync(row_ptr, t.out_rp, (size_t)(n + 1) * 8, k, c->stream);
  if (mem == CG_MEM_HOST && total > 0) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(col, oc, (size_t)total * 4, k, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(code, ok, (size_t)total, k, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(suf, os, (size_t)total * 4, k, c->stream);
  }
  if (e != cudaSuccess) return done(cuda_fail(c, e, "write the reduced graph"));
  st = wait_and_read(&probe);
  return done(st);
}

static_assert(cg::kMaxParts == CG_MAX_PARTS, "part limit");

cg_status cg_partition_contigs(cg_graph* g, int32_t n_parts, int32_t weight, int32_t* part, int64_t part_cap,
                               int64_t* part_weight, int mem, int64_t* n_contigs) {
  Range range("cg.partition_contigs");
  if (!g) return CG_EINVAL;
  cg_ctx* c = g->ctx;
  cg_status st = check_ctx(c);
  if (st != CG_OK) return st;
  if (mem != CG_MEM_HOST && mem != CG_MEM_DEVICE) return fail(c, CG_EINVAL, "bad mem");
  if (n_parts < 1 || n_parts > CG_MAX_PARTS) return fail(c, CG_EINVAL, "n_parts %d not in [1, %d]", n_parts, CG_MAX_PARTS);
  if (weight != CG_WEIGHT_READS && weight != CG_WEIGHT_BASES) return fail(c, CG_EINVAL, "bad weight");
  if (!part_weight) return fail(c, CG_EINVAL, "part_weight is required");
  if (g->stage < 3) {
    st = run_offsets(g);
    if (st != CG_OK) return st;
  }
  st = wait_and_read(g);
  if (st != CG_OK) return st;
  const long long C = c->h_ctr->n_contigs;
  const long long max_w = weight == CG_WEIGHT_READS ? (long long)c->h_ctr->n_walk : (long long)c->h_ctr->total_bases;
  if (C > 0 && (!part || part_cap < C)) return fail(c, CG_EINVAL, "part capacity %lld < %lld", (long long)part_cap, C);
  // temporaries: the sort buffers, and staging for host outputs
  const size_t N = (size_t)(C > 0 ? C : 1);
  const long long tiles = (long long)(N + 2047) / 2048;
  cg::SortBuffers b{};
  b.tiles_cap = tiles;
  b.state_cap = (256 * tiles + 2047) / 2048 + 1;
  const size_t bytes[8] = {8 * N, 8 * N, 4 * N, 4 * N, 4 * 256 * (size_t)tiles, 8 * 256 * (size_t)tiles,
                           8 * ((size_t)b.state_cap + 1), mem == CG_MEM_HOST ? 4 * N + 8 * (size_t)n_parts : 0};
  void* p[8] = {};
  for (int k = 0; k < 8 && st == CG_OK; ++k)
    if (bytes[k]) p[k] = dalloc(c, bytes[k], &st);
  auto release = [&]() {
    for (int k = 0; k < 8; ++k) dfree(c, p[k]);
  };
  if (st != CG_OK) {
    release();
    return st;
  }
  b.key[0] = (unsigned long long*)p[0];
  b.key[1] = (unsigned long long*)p[1];
  b.val[0] = (int32_t*)p[2];
  b.val[1] = (int32_t*)p[3];
  b.hist = (unsigned*)p[4];
  b.base = (unsigned long long*)p[5];
  b.state = (unsigned long long*)p[6];
  int64_t* d_w = mem == CG_MEM_HOST ? (int64_t*)p[7] : part_weight;
  int32_t* d_part = mem == CG_MEM_HOST ? (int32_t*)((char*)p[7] + 8 * (size_t)n_parts) : part;
  if (c->marks.on) {                   // per-kernel marks cover the partition alone
    c->marks.n = 0;
    cudaEventRecord(c->marks.ev[0], c->stream);
  }
  cudaError_t e = cg::launch_partition(g->s, C, weight, max_w, n_parts, b, d_part, d_w, c->env);
  if (e == cudaSuccess && mem == CG_MEM_HOST) {
    e = cudaMemcpyAsync(part_weight, d_w, 8 * (size_t)n_parts, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && C > 0) e = cudaMemcpyAsync(part, d_part, 4 * (size_t)C, cudaMemcpyDeviceToHost, c->stream);
  }
  if (e == cudaSuccess) st = wait_and_read(g);
  release();
  if (e != cudaSuccess) return cuda_fail(c, e, "partition kernels");
  if (st != CG_OK) return st;
  if (n_contigs) *n_contigs = C;
  return CG_OK;
}

}  // extern "C"
