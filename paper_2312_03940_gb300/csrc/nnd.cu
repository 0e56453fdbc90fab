// NN-Descent graph index (Sec. 5.1, graph indices: the framework's
// PyNNDescent option with num_repeats; the steps follow NN-Descent, Dong et
// al., in a synchronous form so that the result does not depend on the
// order of the GPU's threads):
//   for each repeat: N(u) <- the K given ids sorted by (dis, id);
//     each round, from one snapshot of all lists:
//       R(x) <- the K smallest (D(q, x), q) among the q with x in N(q);
//       C(x) <- N(x) u R(x);
//       N'(u) <- the K smallest (dis, id) of N(u) u C(u) u (U_{p in C(u)} C(p)), minus u;
//     until no list changes or the round limit;
//   the repeats are merged (the K smallest of the union of their lists);
//   G(u) <- RobustPrune(u, N(u), alpha, R), then the reverse edges of all
//   points as one batch of the Vamana build (run_all_prune, build.cu).
//
// Kernels: one warp per point, on the beam-search building blocks
// (search_common.cuh): a width-K sorted beam of (dis, id) keys in shared
// memory, the seen-filter to skip repeated ids, canonical scoring of staged
// candidates and the merge that keeps the K smallest keys without repeats.
#include <string.h>

#include <algorithm>
#include <vector>

#include "dispatch.cuh"
#include "search_common.cuh"

namespace pecann {

struct NndArgs {
  SearchArgs a;          // rows, metric, Lw = K, stage, log2h, tag_bytes
  int K;
  const int32_t* N;      // n x K ids of the snapshot
  const float* Nd;       // n x K dis
  const int32_t* Rv;     // n x K reverse ids (-1 padded)
  int32_t* N2;           // n x K new ids
  float* N2d;
  int32_t* Rv_out;       // reverse-list kernel output
  const int32_t* init;   // init kernel: n x K ids
  unsigned long long* changes;
  // reverse lists
  int32_t* rcnt;         // n
  int32_t* rfill;        // n
  int32_t* roff;         // n
  int32_t* rcursor;
  uint64_t* rkeys;       // n x K (dis, source) keys grouped by target
  // merge of repeats
  const int32_t* reps;   // repeats x n x K ids
  const float* repsd;
  int repeats;
};

// Query row of point u in the lanes' chunk layout.
template <int W, int CPL>
__device__ __forceinline__ void nnd_query(const SearchArgs& a, int32_t u, int lane, uint4 (&qv)[CPL]) {
  load_row<W, CPL, false>(a.X + wide_mul(u, a.row_bytes), lane % W, a.C, qv);
}

// Put u into the empty seen-filter (an id the filter already holds is not
// admitted again).
__device__ __forceinline__ void filter_reset(const SearchArgs& a, WarpSmem& w, int32_t u, int lane) {
  const int H = 1 << a.log2h;
  for (int i = lane; i < H; i += 32) w.hash[i] = -1;
  __syncwarp();
  if (lane == 0) {
    if (a.tag_bytes == 1)
      reinterpret_cast<uint8_t*>(w.hash)[(uint32_t)u & ((4u << a.log2h) - 1)] = (uint8_t)((uint32_t)u >> (a.log2h + 2));
    else if (a.tag_bytes == 2)
      reinterpret_cast<uint16_t*>(w.hash)[(uint32_t)u & ((2u << a.log2h) - 1)] = (uint16_t)((uint32_t)u >> (a.log2h + 1));
    else
      w.hash[hash_slot(u, a.log2h)] = u;
  }
  __syncwarp();
}

// Admit the K ids of row[0..K) (K <= 64; -1 entries are padding).
__device__ __forceinline__ int admit_row(const SearchArgs& a, WarpSmem& w, const int32_t* row, int K, int32_t u,
                                         int nc, int lane, unsigned lt, bool* bad) {
  for (int b = 0; b < K; b += 32) {
    const int t = b + lane;
    const int32_t y = t < K ? __ldg(row + t) : -1;
    if (a.tag_bytes == 1)
      nc = admit<1>(a, w, y, u, nc, lt, bad);
    else if (a.tag_bytes == 2)
      nc = admit<2>(a, w, y, u, nc, lt, bad);
    else
      nc = admit<4>(a, w, y, u, nc, lt, bad);
  }
  __syncwarp();
  return nc;
}

__device__ __forceinline__ void write_list(const WarpSmem& w, int nb, int K, int32_t* ids, float* dis, int64_t u,
                                           int lane) {
  for (int t = lane; t < K; t += 32) {
    const uint64_t e = t < nb ? key_clean(w.beam[t]) : KEY_NONE;
    ids[u * K + t] = t < nb ? key_id(e) : -1;
    dis[u * K + t] = t < nb ? key_dis(e) : INFINITY;
  }
}

// N(u) <- the K given ids sorted by (dis, id).
template <int DT, int METRIC, int W, int CPL>
__global__ void __launch_bounds__(128) k_nnd_init(NndArgs r) {
  extern __shared__ __align__(16) uint8_t smem[];
  const SearchArgs& a = r.a;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpSmem w = carve(smem + (size_t)wib * a.warp_bytes, a);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; u < a.n; u += nw) {
    uint4 qv[CPL];
    nnd_query<W, CPL>(a, (int32_t)u, lane, qv);
    for (int t = lane; t < r.K; t += 32) {
      const int32_t y = __ldg(r.init + u * r.K + t);
      // out-of-range ids are reported and replaced by the point itself, whose
      // key is dropped below
      if ((uint32_t)y >= (uint32_t)a.n) set_error(a.err, ERR_BAD_ID);
      w.cids[t] = (uint32_t)y < (uint32_t)a.n ? y : (int32_t)u;
    }
    __syncwarp();
    const int m = eval_cands<DT, METRIC, W, CPL>(a, w, r.K, qv, lane);  // every key kept (m == K)
    for (int t = lane; t < m; t += 32)
      if (key_id(w.ckeys[t]) == (int32_t)u) w.ckeys[t] = KEY_NONE;
    __syncwarp();
    int nb = 0, cursor = 0;
    merge_cands(w, nb, r.K, m, cursor, lane);
    if (nb < r.K && lane == 0) set_error(a.err, ERR_BAD_ID);  // repeated or invalid initial ids
    write_list(w, nb, r.K, r.N2, r.N2d, u, lane);
    __syncwarp();
  }
}

// One synchronous round: N'(u) from the snapshot (N, Nd, Rv).
template <int DT, int METRIC, int W, int CPL>
__global__ void __launch_bounds__(128) k_nnd_round(NndArgs r) {
  extern __shared__ __align__(16) uint8_t smem[];
  const SearchArgs& a = r.a;
  const int K = r.K;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  WarpSmem w = carve(smem + (size_t)wib * a.warp_bytes, a);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; u < a.n; u += nw) {
    uint4 qv[CPL];
    nnd_query<W, CPL>(a, (int32_t)u, lane, qv);
    filter_reset(a, w, (int32_t)u, lane);
    bool bad = false;
    // the beam starts as N(u); its ids enter the filter
    // (a list shorter than K, after a reported bad initial list, ends in -1)
    int nb = 0;
    for (int b = 0; b < K; b += 32) {
      const int t = b + lane;
      const int32_t y = t < K ? __ldg(r.N + u * K + t) : -1;
      if (y >= 0) w.beam[t] = make_key(__ldg(r.Nd + u * K + t), y);
      nb += __popc(__ballot_sync(FULL, y >= 0));
    }
    __syncwarp();
    int nc = admit_row(a, w, r.N + u * K, K, (int32_t)u, 0, lane, lt, &bad);
    nc = 0;  // N(u) is already in the beam
    int cursor = 0;
    // R(u) directly, then C(p) for every p in C(u) = N(u) u R(u)
    nc = admit_row(a, w, r.Rv + u * K, K, (int32_t)u, nc, lane, lt, &bad);
    for (int s = 0; s < 2 * K; s++) {
      const int32_t p = s < K ? __ldg(r.N + u * K + s) : __ldg(r.Rv + u * K + (s - K));
      if (p < 0) continue;
      if (nc + 2 * K > a.stage) {
        eval_merge<DT, METRIC, W, CPL>(a, w, nc, qv, lane, nb, K, cursor);
        nc = 0;
      }
      nc = admit_row(a, w, r.N + (int64_t)p * K, K, (int32_t)u, nc, lane, lt, &bad);
      nc = admit_row(a, w, r.Rv + (int64_t)p * K, K, (int32_t)u, nc, lane, lt, &bad);
    }
    if (nc) {
      eval_merge<DT, METRIC, W, CPL>(a, w, nc, qv, lane, nb, K, cursor);
    }
    if (__any_sync(FULL, bad) && lane == 0) set_error(a.err, ERR_BAD_ID);
    write_list(w, nb, K, r.N2, r.N2d, u, lane);
    bool diff = false;
    for (int t = lane; t < K; t += 32) diff |= r.N2[u * K + t] != __ldg(r.N + u * K + t);
    if (__any_sync(FULL, diff) && lane == 0) atomicAdd(r.changes, 1ull);
    __syncwarp();
  }
}

// Reverse lists, step 1: incoming edges per target.
__global__ void k_nnd_rev_count(NndArgs r) {
  const int64_t total = r.a.n * (int64_t)r.K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    if (r.N[e] >= 0) atomicAdd(r.rcnt + r.N[e], 1);
}

// Step 2: a contiguous range of slots per target (the ranges' order is
// immaterial: every range is selected by key afterwards).
__global__ void k_nnd_rev_offsets(NndArgs r) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < r.a.n; x += (int64_t)gridDim.x * blockDim.x) {
    const int c = r.rcnt[x];
    r.roff[x] = c ? atomicAdd(r.rcursor, c) : 0;
  }
}

// Step 3: the (D(q, x), q) keys of the edges q -> x into x's range.
__global__ void k_nnd_rev_fill(NndArgs r) {
  const int64_t total = r.a.n * (int64_t)r.K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = r.N[e];
    if (x < 0) continue;
    const int32_t q = (int32_t)(e / r.K);
    r.rkeys[r.roff[x] + atomicAdd(r.rfill + x, 1)] = make_key(r.Nd[e], q);
  }
}

// Step 4, one warp per target: the K smallest keys of its range; the
// counters are cleared for the next round.
__global__ void __launch_bounds__(128) k_nnd_rev_select(NndArgs r) {
  extern __shared__ __align__(16) uint8_t smem[];
  const SearchArgs& a = r.a;
  const int K = r.K;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpSmem w = carve(smem + (size_t)wib * a.warp_bytes, a);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t x = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; x < a.n; x += nw) {
    const int c = r.rcnt[x];
    const uint64_t* seg = r.rkeys + r.roff[x];
    int nb = 0, cursor = 0;
    for (int c0 = 0; c0 < c; c0 += 64) {
      const int m = min(64, c - c0);
      for (int i = lane; i < m; i += 32) w.ckeys[i] = seg[c0 + i];
      __syncwarp();
      merge_cands(w, nb, K, m, cursor, lane);
    }
    for (int t = lane; t < K; t += 32) r.Rv_out[x * K + t] = t < nb ? key_id(key_clean(w.beam[t])) : -1;
    __syncwarp();
    if (lane == 0) {
      r.rcnt[x] = 0;
      r.rfill[x] = 0;
    }
  }
}

// The repeats merged: the K smallest of the union of their lists.
__global__ void __launch_bounds__(128) k_nnd_merge(NndArgs r) {
  extern __shared__ __align__(16) uint8_t smem[];
  const SearchArgs& a = r.a;
  const int K = r.K;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpSmem w = carve(smem + (size_t)wib * a.warp_bytes, a);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t nK = a.n * (int64_t)K;
  for (int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; u < a.n; u += nw) {
    int nb = 0, cursor = 0;
    for (int rp = 0; rp < r.repeats; rp++) {
      for (int t = lane; t < K; t += 32) {
        const int32_t y = r.reps[rp * nK + u * K + t];
        w.ckeys[t] = y >= 0 ? make_key(r.repsd[rp * nK + u * K + t], y) : KEY_NONE;
      }
      __syncwarp();
      merge_cands(w, nb, K, K, cursor, lane);
    }
    write_list(w, nb, K, r.N2, r.N2d, u, lane);
    __syncwarp();
  }
}

}  // namespace pecann

namespace pecann {

cudaError_t run_all_prune(const DataView& dv, int R, float alpha, const int32_t* ids, const float* dis, int K,
                          int32_t* G, void* ws, int* d_err, cudaStream_t st);
size_t all_prune_ws_bytes(int64_t n, int R);

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Seen-filter words per warp: 8 per candidate of a round (K + 4 K^2 ids at
// most), within 2^8 .. 2^12.
static int nnd_log2h(int K) {
  const int64_t want = 8 * ((int64_t)K + 4 * (int64_t)K * K) / 4;
  int l = 8;
  while (l < 12 && ((int64_t)1 << l) < want) l++;
  return l;
}

size_t nndescent_ws_bytes(int64_t n, int K, int repeats, int R) {
  const size_t nK = (size_t)n * K;
  return 4 * a256(nK * 4)                      // N, Nd, N2, N2d
         + a256(nK * 4)                        // Rv
         + 3 * a256((size_t)n * 4) + a256(64)  // reverse counts, fill, offsets, counters
         + a256(nK * 8)                        // reverse keys
         + 2 * a256(nK * 4 * repeats)          // each repeat's final lists (ids, dis)
         + all_prune_ws_bytes(n, R);
}

template <class KERN>
static cudaError_t launch_warps(KERN kern, const NndArgs& r, cudaStream_t st) {
  const int wpb = 4;
  const size_t smem = (size_t)wpb * r.a.warp_bytes;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((r.a.n + wpb - 1) / wpb, (int64_t)num_sms() * 16));
  kern<<<grid, wpb * 32, smem, st>>>(r);
  note_launch();
  return cudaGetLastError();
}

static unsigned egrid(int64_t m) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 16384)); }

// NN-Descent (see the top of this file). fv: FP32 or uint8 rows; init:
// repeats x n x K device ids; h_changes (host, repeats x rounds, may be
// NULL): the lists changed by each round (0 after convergence); knn_out
// (device n x K, may be NULL): the merged lists.
cudaError_t run_nndescent(const DataView& fv, int K, int repeats, const int32_t* init, int rounds, float alpha, int R,
                          int32_t* G, int32_t* knn_out, int64_t* h_changes, void* ws, int* d_err, cudaStream_t st) {
  const int64_t n = fv.n;
  const size_t nK = (size_t)n * K;
  uint8_t* w = (uint8_t*)ws;
  auto take = [&](size_t bytes) {
    uint8_t* r = w;
    w += a256(bytes);
    return r;
  };
  int32_t* N = (int32_t*)take(nK * 4);
  float* Nd = (float*)take(nK * 4);
  int32_t* N2 = (int32_t*)take(nK * 4);
  float* N2d = (float*)take(nK * 4);
  int32_t* Rv = (int32_t*)take(nK * 4);
  int32_t* rcnt = (int32_t*)take((size_t)n * 4);
  int32_t* rfill = (int32_t*)take((size_t)n * 4);
  int32_t* roff = (int32_t*)take((size_t)n * 4);
  unsigned long long* counters = (unsigned long long*)take(64);  // [0] changes, [1] reverse cursor
  uint64_t* rkeys = (uint64_t*)take(nK * 8);
  int32_t* reps = (int32_t*)take(nK * 4 * repeats);
  float* repsd = (float*)take(nK * 4 * repeats);
  void* prune_ws = take(all_prune_ws_bytes(n, R));

  NndArgs r;
  memset(&r, 0, sizeof(r));
  SearchArgs& a = r.a;
  a.X = fv.X;
  a.row_bytes = fv.row_bytes;
  a.n = n;
  a.C = fv.C;
  a.metric = fv.metric;
  a.Lw = K;
  a.stage = 2 * K + 64;
  a.log2h = nnd_log2h(K);
  const uint64_t top = (uint64_t)(n - 1);
  a.tag_bytes = (top >> (a.log2h + 2)) < 0xffu ? 1 : ((top >> (a.log2h + 1)) < 0xffffu ? 2 : 4);
  a.mode = MODE_KNN;
  a.warp_bytes = search_warp_bytes(a.Lw, a.log2h, a.stage, 0, false);
  a.err = d_err;
  r.K = K;
  r.changes = counters;
  r.rcnt = rcnt;
  r.rfill = rfill;
  r.roff = roff;
  r.rcursor = reinterpret_cast<int32_t*>(counters + 1);
  r.rkeys = rkeys;
  cudaError_t e;
  if ((e = cudaMemsetAsync(rcnt, 0, (size_t)n * 4, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(rfill, 0, (size_t)n * 4, st)) != cudaSuccess) return e;
  for (int rp = 0; rp < repeats; rp++) {
    // N(u) <- the given ids, sorted
    r.init = init + (size_t)rp * nK;
    r.N2 = N;
    r.N2d = Nd;
    set_where("nn-descent: initial lists");
    e = dispatch_layout(fv, [&](auto dt, auto met, auto wv, auto cpl) -> cudaError_t {
      return launch_warps(k_nnd_init<decltype(dt)::value, decltype(met)::value, decltype(wv)::value,
                                     decltype(cpl)::value>, r, st);
    });
    if (e != cudaSuccess) return e;
    for (int it = 0; it < rounds; it++) {
      // reverse lists of the snapshot
      r.N = N;
      r.Nd = Nd;
      r.Rv_out = Rv;
      if ((e = cudaMemsetAsync(counters, 0, 16, st)) != cudaSuccess) return e;
      set_where("nn-descent: reverse lists");
      k_nnd_rev_count<<<egrid((int64_t)nK), 256, 0, st>>>(r); note_launch();
      k_nnd_rev_offsets<<<egrid(n), 256, 0, st>>>(r); note_launch();
      k_nnd_rev_fill<<<egrid((int64_t)nK), 256, 0, st>>>(r); note_launch();
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = launch_warps(k_nnd_rev_select, r, st)) != cudaSuccess) return e;
      // the round
      r.Rv = Rv;
      r.N2 = N2;
      r.N2d = N2d;
      set_where("nn-descent: round");
      e = dispatch_layout(fv, [&](auto dt, auto met, auto wv, auto cpl) -> cudaError_t {
        return launch_warps(k_nnd_round<decltype(dt)::value, decltype(met)::value, decltype(wv)::value,
                                        decltype(cpl)::value>, r, st);
      });
      if (e != cudaSuccess) return e;
      unsigned long long ch = 0;
      if ((e = cudaMemcpyAsync(&ch, counters, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
      std::swap(N, N2);
      std::swap(Nd, N2d);
      if (h_changes) h_changes[(int64_t)rp * rounds + it] = (int64_t)ch;
      if (ch == 0) break;
    }
    if ((e = cudaMemcpyAsync(reps + rp * nK, N, nK * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(repsd + rp * nK, Nd, nK * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  }
  // the repeats merged
  r.reps = reps;
  r.repsd = repsd;
  r.repeats = repeats;
  r.N2 = N;
  r.N2d = Nd;
  set_where("nn-descent: merge");
  if ((e = launch_warps(k_nnd_merge, r, st)) != cudaSuccess) return e;
  if (knn_out && (e = cudaMemcpyAsync(knn_out, N, nK * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  // RobustPrune and reverse edges, all points as one batch
  return run_all_prune(fv, R, alpha, N, Nd, K, G, prune_ws, d_err, st);
}

}  // namespace pecann
