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
