// Exact FP32 re-rank for reduced-precision traversal. The beam search walks
// BF16 rows; its candidates are re-scored here with the canonical FP32
// distance on the FP32 rows, so the k-NN lists, densities and dependent
// distances that leave the library are exact FP32 values for the points the
// traversal found.
#include "dispatch.cuh"
#include "search_common.cuh"

namespace pecann {

struct RerankArgs {
  SearchArgs a;          // FP32 rows, metric, k, outputs, density_fn
  const int32_t* cand;   // candidates, K per row
  const int32_t* cnt;    // valid candidates per row
  const int32_t* list;   // query ids of the rows (NULL: row = query id)
  int64_t rows;
  int K;
};

// One warp per row: score the candidates in chunks of `stage`, keep the k
// smallest exact keys in a sorted shared-memory beam (the merge of the
// search kernel), then write the k-NN list and the density.
template <int DT, int METRIC, int W, int CPL>
__global__ void __launch_bounds__(128) k_rerank_knn(RerankArgs r) {
  extern __shared__ __align__(16) uint8_t smem[];
  const SearchArgs& a = r.a;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpSmem w = carve(smem + (size_t)wib * a.warp_bytes, a);
  const int gl = lane % W;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; u < r.rows; u += nw) {
    const int c = min(r.cnt[u], r.K);
    if (c < 0) continue;  // handled elsewhere (a later pass or the exact SIMT kernels)
    const int64_t q = r.list ? (int64_t)r.list[u] : u;
    if (c < a.k) {
      if (lane == 0) a.fb_list[atomicAdd(a.fb_cnt, 1)] = (int32_t)q;
      continue;
    }
    uint4 qv[CPL];
    load_row<W, CPL, false>(a.X + q * a.row_bytes, gl, a.C, qv);
    int nb = 0, cursor = 0;
    for (int c0 = 0; c0 < c; c0 += a.stage) {
      const int nc = min(a.stage, c - c0);
      for (int i = lane; i < nc; i += 32) w.cids[i] = r.cand[u * r.K + c0 + i];
      __syncwarp();
      eval_merge<DT, METRIC, W, CPL>(a, w, nc, qv, lane, nb, a.k, cursor);
    }
    for (int t = lane; t < a.k; t += 32) {
      const uint64_t e = key_clean(w.beam[t]);
      a.out_ids[q * a.k + t] = key_id(e);
      a.out_dis[q * a.k + t] = out_dist(key_dis(e), a.metric);
    }
    __syncwarp();
    if (lane == 0) density_from_beam(w.beam, a.k, a.metric, a.density_fn, a.rho + q, a.rkey + q);
    __syncwarp();
  }
}

// One warp per listed query: the exact argmin of (dis, id) over its
// candidates (all of them rank above the query).
template <int DT, int METRIC, int W, int CPL>
__global__ void __launch_bounds__(128) k_rerank_dep(RerankArgs r) {
  extern __shared__ __align__(16) uint8_t smem[];
  const SearchArgs& a = r.a;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpSmem w = carve(smem + (size_t)wib * a.warp_bytes, a);
  const int gl = lane % W;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; u < r.rows; u += nw) {
    const int c = min(r.cnt[u], r.K);
    if (c <= 0) continue;  // none ranked above, or handled elsewhere (-1)
    const int32_t q = r.list[u];
    uint4 qv[CPL];
    load_row<W, CPL, false>(a.X + (int64_t)q * a.row_bytes, gl, a.C, qv);
    uint64_t best = KEY_NONE;
    for (int c0 = 0; c0 < c; c0 += a.stage) {
      const int nc = min(a.stage, c - c0);
      for (int i = lane; i < nc; i += 32) w.cids[i] = r.cand[u * r.K + c0 + i];
      __syncwarp();
      const int m = eval_cands<DT, METRIC, W, CPL>(a, w, nc, qv, lane);  // every key kept
      for (int i = lane; i < m; i += 32) best = w.ckeys[i] < best ? w.ckeys[i] : best;
      __syncwarp();
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      const uint64_t o = __shfl_xor_sync(FULL, best, off);
      best = o < best ? o : best;
    }
    if (lane == 0 && best != KEY_NONE) {
      a.lam[q] = key_id(best);
      a.delta[q] = out_dist(key_dis(best), a.metric);
    }
  }
}

template <class KERN>
static cudaError_t launch_rr(KERN kern, const RerankArgs& r, cudaStream_t st) {
  const int wpb = 4;
  const size_t smem = (size_t)wpb * r.a.warp_bytes;
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t want = (r.rows + wpb - 1) / wpb;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * 16));
  kern<<<grid, wpb * 32, smem, st>>>(r);
  note_launch();
  return cudaGetLastError();
}

static void fill_common(RerankArgs& r, const DataView& f32, int beam) {
  memset(&r, 0, sizeof(r));
  SearchArgs& a = r.a;
  a.X = f32.X;
  a.row_bytes = f32.row_bytes;
  a.n = f32.n;
  a.C = f32.C;
  a.metric = f32.metric;
  a.Lw = beam;
  a.stage = 64;
  a.log2h = 0;
  a.mode = MODE_KNN;
  a.warp_bytes = search_warp_bytes(beam, 0, a.stage, 0, false);
}

cudaError_t launch_rerank_knn(const DataView& f32, const int32_t* list, int64_t rows, const int32_t* cand,
                              const int32_t* cnt, int K, int k, int32_t* knn_ids, float* knn_dist, float* rho,
                              float* rkey, int density_fn, int32_t* fb_list, int32_t* fb_cnt, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  RerankArgs r;
  fill_common(r, f32, k);
  r.a.k = k;
  r.a.out_ids = knn_ids;
  r.a.out_dis = knn_dist;
  r.a.rho = rho;
  r.a.rkey = rkey;
  r.a.density_fn = density_fn;
  r.a.fb_list = fb_list;
  r.a.fb_cnt = fb_cnt;
  r.cand = cand;
  r.cnt = cnt;
  r.list = list;
  r.rows = rows;
  r.K = K;
  return dispatch_layout(f32, [&](auto dt, auto met, auto wv, auto cpl) -> cudaError_t {
    return launch_rr(k_rerank_knn<decltype(dt)::value, decltype(met)::value, decltype(wv)::value,
                                  decltype(cpl)::value>, r, st);
  });
}

cudaError_t launch_rerank_dep(const DataView& f32, const int32_t* list, int64_t m, const int32_t* cand,
                              const int32_t* cnt, int K, int32_t* lam, float* delta, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  RerankArgs r;
  fill_common(r, f32, 1);
  r.a.lam = lam;
  r.a.delta = delta;
  r.cand = cand;
  r.cnt = cnt;
  r.list = list;
  r.rows = m;
  r.K = K;
  return dispatch_layout(f32, [&](auto dt, auto met, auto wv, auto cpl) -> cudaError_t {
    return launch_rr(k_rerank_dep<decltype(dt)::value, decltype(met)::value, decltype(wv)::value,
                                  decltype(cpl)::value>, r, st);
  });
}

}  // namespace pecann
