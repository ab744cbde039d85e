// cg_server.cu - the served form: a request loop over the library's batched
// path. Requests (one string graph each, host inputs) are admitted against a
// device-memory budget, grouped by continuous batching -- every admitted
// request waiting when a worker becomes free joins its batch -- and run as
// one union graph per batch. Several workers, each with its own context and
// stream, keep as many batches in flight, so that one batch's host-to-device
// copy or host-link reads overlap the others' kernels and copies back; each
// request's contigs are copied from the batch's device output straight into
// the request's result. Host code only.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "cg.h"
#include "cg_fault.h"
#include <nvtx3/nvToolsExt.h>

namespace {

using Clock = std::chrono::steady_clock;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t id = 0;
  cg_graph_desc desc{};
  uint64_t est_bytes = 0;
  int64_t t_submit = 0, t_start = 0, t_done = 0;
  int done = 0;
  cg_status status = CG_OK;
  int64_t n_contigs = 0, total_bases = 0;
  std::vector<int64_t> contig_off;
  std::vector<uint8_t> bases;
  int batch_size = 0;
};

}  // namespace

struct cg_server {
  int device = 0;
  cg_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> waiting;          // submitted, not yet admitted
  std::deque<Request*> admitted;         // within the budget, not yet taken by a worker
  std::map<uint64_t, Request*> all;
  uint64_t next_id = 1;
  uint64_t in_flight_bytes = 0;          // estimates of admitted, unfinished requests
  bool stopping = false;
  std::vector<std::thread> workers;
  cg::FaultPlan fault;                   // host-side fault injection (tests)
  std::vector<cg_ctx*> ctxs;             // one per worker (under mu: a worker may replace its own)
  std::vector<cudaStream_t> streams;
  cudaMemPool_t pool = nullptr;          // the workers' device output buffers (stream-ordered)
  uint64_t batches = 0, batched_requests = 0, contexts_replaced = 0;
  uint64_t retired_kernels = 0;          // kernels launched by replaced contexts
};

namespace {

// Device memory a request needs at most: its inputs, the library's scratch
// (about 400 bytes per read and 16 per CSR entry) and room for its output.
uint64_t estimate(const cg_graph_desc& d) {
  return (uint64_t)d.packed_bytes * 2 + 400ull * (uint64_t)d.n_reads + 16ull * (uint64_t)d.n_entries + (1ull << 20);
}

// Moves waiting requests into the admitted queue while the budget allows.
void admit_locked(cg_server* s) {
  while (!s->waiting.empty()) {
    Request* r = s->waiting.front();
    if (s->in_flight_bytes + r->est_bytes > s->opts.hbm_budget_bytes && s->in_flight_bytes > 0) break;
    s->waiting.pop_front();
    s->in_flight_bytes += r->est_bytes;
    s->admitted.push_back(r);
  }
}

// A worker's device output buffers, grown when a batch needs more. They come
// from the server's stream-ordered memory pool on the worker's stream, so
// growing them never calls cudaMalloc or cudaFree, which would synchronise
// the whole device and stall the other worker's batch.
struct WorkerBuffers {
  uint8_t* bases = nullptr;
  int64_t bases_cap = 0;
  int64_t* off = nullptr;
  int64_t off_cap = 0;
};

struct Worker {
  int index = 0;
  cg_ctx* ctx = nullptr;               // replaced after an error that leaves it refusing work
  cudaStream_t stream = nullptr;
  WorkerBuffers wb;
  unsigned long long kernels_seen = 0;   // kernels of the current context before its last batch
};

bool leaves_context_refusing(cg_status st) { return st == CG_ECUDA || st == CG_ETIMEOUT || st == CG_EKERNEL; }

cg_status grow(cg_server* s, Worker& w, int64_t total, int64_t contigs) {
  WorkerBuffers& wb = w.wb;
  if (total > wb.bases_cap) {
    if (wb.bases) cudaFreeAsync(wb.bases, w.stream);
    wb.bases = nullptr;
    const int64_t cap = total + total / 4 + 4096;
    if (cudaMallocFromPoolAsync((void**)&wb.bases, (size_t)cap, s->pool, w.stream) != cudaSuccess) {
      cudaGetLastError();
      wb.bases = nullptr;
      wb.bases_cap = 0;
      return CG_ENOMEM;
    }
    wb.bases_cap = cap;
  }
  if (contigs + 1 > wb.off_cap) {
    if (wb.off) cudaFreeAsync(wb.off, w.stream);
    wb.off = nullptr;
    const int64_t cap = contigs + contigs / 4 + 1024;
    if (cudaMallocFromPoolAsync((void**)&wb.off, (size_t)cap * 8, s->pool, w.stream) != cudaSuccess) {
      cudaGetLastError();
      wb.off = nullptr;
      wb.off_cap = 0;
      return CG_ENOMEM;
    }
    wb.off_cap = cap;
  }
  return CG_OK;
}

void release_buffers(Worker& w) {
  if (w.wb.bases) cudaFreeAsync(w.wb.bases, w.stream);
  if (w.wb.off) cudaFreeAsync(w.wb.off, w.stream);
  cudaStreamSynchronize(w.stream);
  w.wb = WorkerBuffers{};
}

// A context that returned CG_ECUDA, CG_ETIMEOUT or CG_EKERNEL refuses all
// further work; the worker destroys it and creates a fresh one on its stream
// (its device output buffers belong to the server's pool and stay).
void replace_context(cg_server* s, Worker& w) {
  cg_ctx* fresh = nullptr;
  if (cg_create(&fresh, s->device, s->opts.hbm_budget_bytes, w.stream) == CG_OK) cg_set_graphs(fresh, 0);
  else fresh = nullptr;
  cg_ctx* old = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    old = w.ctx;
    w.ctx = fresh;
    s->ctxs[(size_t)w.index] = fresh;
    s->contexts_replaced += 1;
    s->retired_kernels += w.kernels_seen;   // a refusing context no longer reports its count
    w.kernels_seen = 0;
  }
  if (old) cg_destroy(old);
}

// One union graph over `batch` on the worker's context: fills each request's
// contigs and counts (not its status). Returns the batch's status.
cg_status run_union(cg_server* s, Worker& w, std::vector<Request*>& batch) {
  if (!w.ctx) return CG_ECUDA;
  cg_ctx* ctx = w.ctx;
  const int k = (int)batch.size();
  std::vector<cg_graph_desc> descs(k);
  for (int j = 0; j < k; ++j) descs[j] = batch[j]->desc;
  {
    cg_stats stt{};
    if (cg_get_stats(ctx, &stt) == CG_OK) w.kernels_seen = stt.kernels_launched;
  }
  // requests whose reads are pinned host memory leave them there: the batch
  // gathers only the bases it spells over the host link; otherwise every
  // request's reads are copied
  cg_graph* g = nullptr;
  cg_status st = cg_load_batch(ctx, descs.data(), k, CG_HOST_READS, &g);
  if (st == CG_EINVAL) st = cg_load_batch(ctx, descs.data(), k, 0, &g);
  std::vector<int64_t> fc(k + 1), fb(k + 1);
  int64_t n_contigs = 0, total = 0;
  if (st == CG_OK) st = cg_mask_branches(g, nullptr, CG_MEM_DEVICE, nullptr);
  if (st == CG_OK) st = cg_chains(g, nullptr, nullptr, nullptr, CG_MEM_DEVICE, nullptr, nullptr);
  if (st == CG_OK) st = cg_emit_contigs(g, nullptr, 0, nullptr, 0, CG_MEM_DEVICE, &n_contigs, &total);
  if (st == CG_OK) st = grow(s, w, total, n_contigs);
  WorkerBuffers& wb = w.wb;
  if (st == CG_OK)
    st = cg_emit_contigs(g, wb.off, wb.off_cap, wb.bases, wb.bases_cap, CG_MEM_DEVICE, nullptr, nullptr);
  if (st == CG_OK) st = cg_batch_ranges(g, fc.data(), fb.data(), CG_MEM_HOST);   // waits for the stream
  if (st == CG_OK) {
    // each request's slice goes straight from device memory into its result
    for (int j = 0; j < k && st == CG_OK; ++j) {
      Request* r = batch[j];
      const int64_t c0 = fc[j], c1 = fc[j + 1], b0 = fb[j], b1 = fb[j + 1];
      r->n_contigs = c1 - c0;
      r->total_bases = b1 - b0;
      r->contig_off.resize((size_t)(c1 - c0) + 1);
      r->bases.resize((size_t)(b1 - b0));
      if (cudaMemcpyAsync(r->contig_off.data(), wb.off + c0, (size_t)(c1 - c0 + 1) * 8, cudaMemcpyDeviceToHost,
                          w.stream) != cudaSuccess ||
          (b1 > b0 && cudaMemcpyAsync(r->bases.data(), wb.bases + b0, (size_t)(b1 - b0), cudaMemcpyDeviceToHost,
                                      w.stream) != cudaSuccess))
        st = CG_ECUDA;
    }
    if (cudaStreamSynchronize(w.stream) != cudaSuccess) st = CG_ECUDA;
    for (int j = 0; j < k; ++j)
      for (int64_t& o : batch[j]->contig_off) o -= fb[j];
  }
  if (g) cg_free_graph(g);
  cudaGetLastError();
  if (st != CG_OK)
    for (Request* r : batch) {
      r->n_contigs = r->total_bases = 0;
      r->contig_off.clear();
      r->bases.clear();
    }
  return st;
}

void run_batch(cg_server* s, Worker& w, std::vector<Request*>& batch) {
  nvtxRangePushA("cg.server.batch");
  const int k = (int)batch.size();
  const int64_t t0 = now_ns();
  for (Request* r : batch) {
    r->t_start = t0;
    r->batch_size = k;
  }
  if (w.ctx && s->fault.hit("batch_timeout")) cg_set_fault(w.ctx, "timeout:1");   // injected: a device wait runs out
  std::vector<cg_status> sts((size_t)k, run_union(s, w, batch));
  const cg_status st = sts[0];
  if (leaves_context_refusing(st)) replace_context(s, w);
  if ((st == CG_EGRAPH || st == CG_EINVAL) && k > 1) {
    // One malformed request fails the whole union (its input checks, or its
    // sizes): run every member alone, so that only the bad ones report it.
    for (int j = 0; j < k; ++j) {
      std::vector<Request*> one{batch[(size_t)j]};
      batch[(size_t)j]->batch_size = 1;
      sts[(size_t)j] = run_union(s, w, one);
      if (leaves_context_refusing(sts[(size_t)j])) replace_context(s, w);
    }
  }
  const int64_t t1 = now_ns();
  std::lock_guard<std::mutex> lk(s->mu);
  for (int j = 0; j < k; ++j) {
    Request* r = batch[(size_t)j];
    r->status = sts[(size_t)j];
    r->t_done = t1;
    r->done = 1;
    s->in_flight_bytes -= r->est_bytes;
  }
  s->batches += 1;
  s->batched_requests += (uint64_t)k;
  admit_locked(s);
  s->cv_done.notify_all();
  s->cv_work.notify_all();
  nvtxRangePop();
}

void worker_main(cg_server* s, int index) {
  Worker w;
  w.index = index;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    w.ctx = s->ctxs[(size_t)index];
  }
  w.stream = s->streams[(size_t)index];
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Request*> batch;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stopping || !s->admitted.empty(); });
      if (s->admitted.empty() && s->stopping) break;
      while (!s->admitted.empty() && (int)batch.size() < s->opts.max_batch) {
        batch.push_back(s->admitted.front());
        s->admitted.pop_front();
      }
    }
    int stall_ms = 0;
    if (!batch.empty() && s->fault.hit("queue_stall", &stall_ms) && stall_ms > 0)
      std::this_thread::sleep_for(std::chrono::milliseconds(stall_ms));
    if (!batch.empty()) run_batch(s, w, batch);
  }
  release_buffers(w);
}

}  // namespace

extern "C" {

cg_status cg_server_start(int device, const cg_server_opts* opts, cg_server** out) {
  if (!opts || !out || opts->max_batch < 1 || opts->workers < 1 || opts->workers > 16 || opts->hbm_budget_bytes == 0)
    return CG_EINVAL;
  *out = nullptr;
  cg_server* s = new (std::nothrow) cg_server();
  if (!s) return CG_ENOMEM;
  s->device = device;
  s->opts = *opts;
  s->fault.from_env();
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return CG_ECUDA;
  }
  {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return CG_ECUDA;
    }
    uint64_t keep = ~0ull;   // freed buffers stay in the pool for the next batch
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  for (int w = 0; w < opts->workers; ++w) {
    cg_ctx* c = nullptr;
    cudaStream_t st_w = nullptr;
    cg_status st = cudaStreamCreateWithFlags(&st_w, cudaStreamNonBlocking) == cudaSuccess ? CG_OK : CG_ECUDA;
    if (st == CG_OK) st = cg_create(&c, device, opts->hbm_budget_bytes, st_w);
    if (st != CG_OK) {
      if (st_w) cudaStreamDestroy(st_w);
      for (cg_ctx* x : s->ctxs) cg_destroy(x);
      for (cudaStream_t y : s->streams) cudaStreamDestroy(y);
      cudaMemPoolDestroy(s->pool);
      delete s;
      return st;
    }
    s->streams.push_back(st_w);
    cg_set_graphs(c, 0);   // every batch is a new union graph: nothing to replay
    s->ctxs.push_back(c);
  }
  for (int w = 0; w < opts->workers; ++w) s->workers.emplace_back(worker_main, s, w);
  *out = s;
  return CG_OK;
}

cg_status cg_server_submit(cg_server* s, const cg_graph_desc* d, uint64_t* id) {
  if (!s || !d || !id) return CG_EINVAL;
  if (d->mem != CG_MEM_HOST) return CG_EINVAL;
  Request* r = new (std::nothrow) Request();
  if (!r) return CG_ENOMEM;
  r->desc = *d;
  r->est_bytes = estimate(*d);
  if (s->fault.hit("admit")) {
    delete r;
    return CG_EBUSY;                     // injected: admission refused
  }
  if (r->est_bytes > s->opts.hbm_budget_bytes) {
    delete r;
    return CG_EBUSY;                     // can never fit the budget
  }
  r->t_submit = now_ns();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping) {
    delete r;
    return CG_EINVAL;
  }
  r->id = s->next_id++;
  *id = r->id;
  s->all[r->id] = r;
  s->waiting.push_back(r);
  admit_locked(s);
  s->cv_work.notify_one();
  return CG_OK;
}

cg_status cg_server_poll(cg_server* s, uint64_t id, int* done) {
  if (!s || !done) return CG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return CG_EINVAL;
  *done = it->second->done;
  return CG_OK;
}

cg_status cg_server_wait(cg_server* s, uint64_t id, int64_t timeout_ms, cg_server_result* res) {
  if (!s || !res) return CG_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return CG_EINVAL;
  Request* r = it->second;
  const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 1ll << 40 : timeout_ms),
                                      [&] { return r->done != 0; });
  if (!ok) return CG_ETIMEOUT;
  res->status = r->status;
  res->n_contigs = r->n_contigs;
  res->total_bases = r->total_bases;
  res->contig_off = r->contig_off.data();
  res->bases = r->bases.data();
  res->t_submit_ns = r->t_submit;
  res->t_start_ns = r->t_start;
  res->t_done_ns = r->t_done;
  res->batch_size = r->batch_size;
  return CG_OK;
}

cg_status cg_server_release(cg_server* s, uint64_t id) {
  if (!s) return CG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end() || !it->second->done) return CG_EINVAL;
  delete it->second;
  s->all.erase(it);
  return CG_OK;
}

cg_status cg_server_stats(cg_server* s, uint64_t* batches, uint64_t* requests, uint64_t* in_flight_bytes) {
  if (!s) return CG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (batches) *batches = s->batches;
  if (requests) *requests = s->batched_requests;
  if (in_flight_bytes) *in_flight_bytes = s->in_flight_bytes;
  return CG_OK;
}

cg_status cg_server_kernels(cg_server* s, uint64_t* launched) {
  if (!s || !launched) return CG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  uint64_t n = s->retired_kernels;
  for (cg_ctx* c : s->ctxs) {
    cg_stats st{};
    if (c && cg_get_stats(c, &st) == CG_OK) n += st.kernels_launched;
  }
  *launched = n;
  return CG_OK;
}

cg_status cg_server_contexts_replaced(cg_server* s, uint64_t* replaced) {
  if (!s || !replaced) return CG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *replaced = s->contexts_replaced;
  return CG_OK;
}

cg_status cg_server_stop(cg_server* s) {
  if (!s) return CG_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (std::thread& t : s->workers) t.join();
  for (cg_ctx* c : s->ctxs)
    if (c) cg_destroy(c);
  for (cudaStream_t y : s->streams) cudaStreamDestroy(y);
  if (s->pool) cudaMemPoolDestroy(s->pool);
  for (auto& kv : s->all) delete kv.second;   // every request is in `all` until released; workers drained them
  delete s;
  return CG_OK;
}

}  // extern "C"
