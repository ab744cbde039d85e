// cg_reduce.cu - TransitiveReduction (Alg. 1: S <- TransitiveReduction(R);
// Sec. 2) on sm_103a: the string graph of an overlap graph.
//
// An entry x = (u->w) is transitive when some read v gives a valid walk
// u -> v -> w that leaves u through x's end of u, passes through v (entered
// through one end, left through the other) and enters w through x's end of w,
// and whose suffixes add up to x's within a tolerance. A pair of reads keeps
// both entries only when neither is transitive.
//
// Rows hold a few entries and most reads none, so after one pass that writes
// every entry's row, the work takes one thread per entry: the entry (u->v)
// walks v's row and looks each w up in u's row (rows are sorted by column) by
// binary search; an entry is kept when neither it nor its mirror is
// transitive; per-row counts and a look-back scan give the new row offsets;
// every kept entry goes to its row's offset plus the kept entries before it.
#include <cuda_runtime.h>

#include "cg_internal.cuh"
#include "cg_lookback.cuh"

namespace cg {

namespace {

// Position of column w in the sorted row [a, b), or -1.
__device__ __forceinline__ int64_t find_col(const int32_t* col, int64_t a, int64_t b, int32_t w) {
  int64_t lo = a, hi = b;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(col + mid) < w) lo = mid + 1;
    else hi = mid;
  }
  return lo < b && __ldg(col + lo) == w ? lo : -1;
}

// Rows: offsets in [0, m] and increasing, columns strictly increasing (sorted,
// no repeated pair), every read at least one base long.
__global__ void k_tr_check(DevGraph g, DevError* e) {
  for (long long u = grid_tid(); u < g.n; u += grid_threads()) {
    const int64_t a = rowp(g, u), b = rowp(g, u + 1);
    if (a < 0 || b < a || b > g.m || g.len[u] < 1) {
      set_error(e, DERR_GRAPH, K_TRANSITIVE, u);
      continue;
    }
    for (int64_t x = a + 1; x < b; ++x)
      if (g.col[x] <= g.col[x - 1]) set_error(e, DERR_GRAPH, K_TRANSITIVE, x);
  }
  if (grid_tid() == 0 && (rowp(g, 0) != 0 || rowp(g, g.n) != g.m)) set_error(e, DERR_GRAPH, K_TRANSITIVE, -1);
}

// Row of every entry (one thread per row), so that the kernels below can
// take one thread per entry: rows hold few entries and most reads none.
__global__ void k_tr_rowof(DevGraph g, int32_t* row_of) {
  for (long long u = grid_tid(); u < g.n; u += grid_threads()) {
    const int64_t a = rowp(g, u), b = rowp(g, u + 1);
    for (int64_t x = a; x < b; ++x) row_of[x] = (int32_t)u;
  }
}

// Entries, once the rows are known sorted: column in range and not the row
// itself, code 0..3, suffix in [1, len-1], and exactly one mirror entry (found
// by binary search) with the swapped code.
__global__ void k_tr_entries(DevGraph g, const int32_t* row_of, DevError* e) {
  for (long long x = grid_tid(); x < g.m; x += grid_threads()) {
    const int32_t u = row_of[x], w = g.col[x];
    const int cd = g.code[x];
    if (w < 0 || w >= g.n || w == u || cd > 3) {
      set_error(e, DERR_GRAPH, K_TRANSITIVE, x);
      continue;
    }
    const int32_t sf = g.suf[x];
    if (sf < 1 || sf > g.len[w] - 1) set_error(e, DERR_GRAPH, K_TRANSITIVE, x);
    const int64_t y = find_col(g.col, rowp(g, w), rowp(g, w + 1), u);
    if (y < 0 || g.code[y] != (((cd & 1) << 1) | (cd >> 1))) set_error(e, DERR_GRAPH, K_TRANSITIVE, x);
  }
}

// One thread per entry y = (u->v): every walk u -> v -> w through v's row,
// each w looked up in u's sorted row; marks the transitive (u->w).
__global__ void __launch_bounds__(kBlock) k_tr_mark(DevGraph g, const int32_t* row_of, int fuzz, uint8_t* trans) {
  for (long long y = grid_tid(); y < g.m; y += grid_threads()) {
    const int32_t u = row_of[y], v = g.col[y];
    const int cy = g.code[y];
    const int32_t sy = g.suf[y];
    const int eu = cy & 1, ev_in = (cy >> 1) & 1;
    const int64_t a = rowp(g, u), b = rowp(g, u + 1);
    const int64_t va = rowp(g, v), vb = rowp(g, v + 1);
    for (int64_t z = va; z < vb; ++z) {
      const int cz = g.code[z];
      if ((cz & 1) != 1 - ev_in) continue;        // leave v through its other end
      const int32_t w = g.col[z];
      if (w == u) continue;
      const int64_t x = find_col(g.col, a, b, w);
      if (x < 0) continue;
      const int cx = g.code[x];
      if ((cx & 1) != eu || ((cx >> 1) & 1) != ((cz >> 1) & 1)) continue;   // the ends of x
      const long long d = (long long)sy + g.suf[z] - g.suf[x];
      if (d <= fuzz && d >= -fuzz) trans[x] = 1;
    }
  }
}

// One thread per entry: kept when neither it nor its mirror is transitive.
__global__ void k_tr_keep(DevGraph g, const int32_t* row_of, const uint8_t* trans, uint8_t* keep) {
  for (long long x = grid_tid(); x < g.m; x += grid_threads()) {
    const int32_t u = row_of[x], w = g.col[x];
    const int64_t y = find_col(g.col, rowp(g, w), rowp(g, w + 1), u);
    keep[x] = !trans[x] && !(y >= 0 && trans[y]);
  }
}

// One thread per row: its kept entries.
__global__ void k_tr_rowcnt(DevGraph g, const uint8_t* keep, int32_t* row_cnt) {
  for (long long u = grid_tid(); u < g.n; u += grid_threads()) {
    const int64_t a = rowp(g, u), b = rowp(g, u + 1);
    int cnt = 0;
    for (int64_t x = a; x < b; ++x) cnt += keep[x];
    row_cnt[u] = cnt;
  }
}

struct RowCntLoad {
  const int32_t* cnt;
  __device__ unsigned long long operator()(long long i) const { return (unsigned long long)cnt[i]; }
};
struct RowPtrStore {
  int64_t* rp;
  unsigned long long* total;
  __device__ void item(long long i, unsigned long long e) const { rp[i] = (int64_t)e; }
  __device__ void last(long long n, unsigned long long t) const {
    rp[n] = (int64_t)t;
    *total = t;
  }
};

// One thread per kept entry: its row's new offset plus the kept entries
// before it in the row (rows keep their order).
__global__ void k_tr_scatter(DevGraph g, const int32_t* row_of, const uint8_t* keep, const int64_t* out_rp,
                             int32_t* col, uint8_t* code, int32_t* suf) {
  for (long long x = grid_tid(); x < g.m; x += grid_threads()) {
    if (!keep[x]) continue;
    const int32_t u = row_of[x];
    int64_t o = out_rp[u];
    for (int64_t y = rowp(g, u); y < x; ++y) o += keep[y];
    col[o] = g.col[x];
    code[o] = g.code[x];
    suf[o] = g.suf[x];
  }
}

}  // namespace

cudaError_t launch_transitive_check(const DevGraph& g, DevError* derr, const LaunchEnv& env) {
  k_tr_check<<<grid_for(g.n, env), kBlock, 0, env.stream>>>(g, derr);
  mark(env, "k_tr_check");
  return cudaGetLastError();
}

cudaError_t launch_transitive_entries(const DevGraph& g, const TrBuffers& t, const LaunchEnv& env) {
  k_tr_rowof<<<grid_for(g.n, env), kBlock, 0, env.stream>>>(g, t.row_of);
  mark(env, "k_tr_rowof");
  k_tr_entries<<<grid_for(g.m, env), kBlock, 0, env.stream>>>(g, t.row_of, t.derr);
  mark(env, "k_tr_entries");
  return cudaGetLastError();
}

cudaError_t launch_transitive(const DevGraph& g, int fuzz, const TrBuffers& t, const LaunchEnv& env) {
  cudaMemsetAsync(t.trans, 0, (size_t)(g.m > 0 ? g.m : 1), env.stream);
  k_tr_mark<<<grid_for(g.m, env), kBlock, 0, env.stream>>>(g, t.row_of, fuzz, t.trans);
  mark(env, "k_tr_mark");
  k_tr_keep<<<grid_for(g.m, env), kBlock, 0, env.stream>>>(g, t.row_of, t.trans, t.keep);
  mark(env, "k_tr_keep");
  k_tr_rowcnt<<<grid_for(g.n, env), kBlock, 0, env.stream>>>(g, t.keep, t.row_cnt);
  mark(env, "k_tr_rowcnt");
  cudaMemsetAsync(t.state, 0, (size_t)(t.state_cap + 1) * sizeof(unsigned long long), env.stream);
  const long long tiles = (g.n + kTileItems - 1) / kTileItems;
  if (tiles > t.state_cap) return cudaErrorInvalidValue;
  if (g.n > 0) {
    k_scan<<<scan_grid(tiles, env), kBlock, 0, env.stream>>>(RowCntLoad{t.row_cnt}, RowPtrStore{t.out_rp, t.total}, g.n,
                                                       nullptr, t.state, t.state_cap, t.derr, K_TRANSITIVE);
    mark(env, "k_scan_rows");
  } else {
    cudaMemsetAsync(t.out_rp, 0, sizeof(int64_t), env.stream);
    cudaMemsetAsync(t.total, 0, sizeof(unsigned long long), env.stream);
  }
  return cudaGetLastError();
}

cudaError_t launch_transitive_scatter(const DevGraph& g, const TrBuffers& t, int32_t* col, uint8_t* code, int32_t* suf,
                                      const LaunchEnv& env) {
  k_tr_scatter<<<grid_for(g.m, env), kBlock, 0, env.stream>>>(g, t.row_of, t.keep, t.out_rp, col, code, suf);
  mark(env, "k_tr_scatter");
  return cudaGetLastError();
}

}  // namespace cg
