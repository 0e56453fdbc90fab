// Greedy beam search (Algorithm 1), one query per warp.
//
// Per warp, in shared memory:
//   beam   Lw keys, sorted ascending by (dis, id); bit 31 marks "visited".
//          This is L of Algorithm 1 with its visited part: popping the
//          closest unvisited point is a scan for the first unflagged entry.
//   ckeys  candidate keys of the current expansion (staging)
//   ss     the surviving candidates, sorted
//   vis    (build searches) the vcap closest expanded points
//   hash   a direct-mapped filter of ids already evaluated. It may forget an
//          id (two ids sharing a slot); the only cost is a repeated distance,
//          because a repeated point is either already in the beam with the
//          identical key (dropped as a duplicate by the merge) or no better
//          than the beam's current worst entry (dropped by the filter) --
//          exactly what Algorithm 1 does with a point it adds again.
//   cids   candidate ids
//
// One expansion: pop p*, read its R out-neighbours (coalesced), drop the
// query, seen ids and -1 padding, compute the canonical distances of the
// rest (W lanes per row, several rows per warp pass, loads of all rows issued
// before any arithmetic), drop candidates no better than the current L-th
// entry (they would be pruned at once), and merge the survivors into the
// sorted beam in place. Algorithm 1's k closest points of (L u V) are the
// first k beam entries: a visited point that left L was worse than all L
// points kept at that moment, and the L-th entry only improves afterwards.
#include "search_kernel.cuh"

namespace pecann {

int search_warp_bytes(int Lw, int log2h, int stage, int vcap, bool build) {
  return search_warp_bytes_impl(Lw, log2h, stage, vcap, build);
}

bool pick_layout(int dtype, int metric, int d, Layout* out) {
  int epc = dtype == DT_F32 ? 4 : (dtype == DT_BF16 ? 8 : 16);
  if (d <= 0 || d % epc) return false;
  if (dtype != DT_F32 && dtype != DT_U8 && dtype != DT_BF16 && dtype != DT_FP8) return false;
  if (dtype == DT_U8 && (metric != MET_L2 || d > 256)) return false;
  int C = d / epc;
  if (dtype == DT_FP8) {
    // inner product only: the scale folds into the query (a_j = q_j s_j), so
    // a row costs one decode and one FMA per element; L2 would need s_j^2 per
    // element as a second operand
    if (metric != MET_IP) return false;
    if (C <= 8) *out = {8, 1};
    else if (C <= 16) *out = {16, 1};
    else if (C <= 32) *out = {32, 1};
    else if (C <= 64) *out = {32, 2};  // d <= 1024, the FP32 re-rank's limit
    else return false;
    return true;
  }
  if (dtype == DT_U8) {
    // integer sums are exact in any order; one 16-byte chunk per lane (a
    // 128-byte row takes 8 lanes) measured faster than two chunks per lane
    *out = {C <= 8 ? 8 : 16, 1};
    return true;
  }
  // FP32 / BF16: lane c of a 32-lane row owns chunk c (mod 32), as the
  // canonical summation order requires
  if (C <= 8) {
    *out = {8, 1};
  } else if (C <= 16) {
    *out = {16, 1};
  } else if (C <= 32) {
    *out = {32, 1};
  } else if (C <= 64) {
    *out = {32, 2};
  } else if (C <= 96) {
    *out = {32, 3};
  } else if (C <= 128) {
    *out = {32, 4};
  } else if (C <= 256) {
    *out = {32, 8};
  } else {
    return false;
  }
  return true;
}

cudaError_t launch_search_u8(const DataView& dv, const SearchArgs& a, const Layout& L, cudaStream_t st);
cudaError_t launch_search_f32_l2(const DataView& dv, const SearchArgs& a, const Layout& L, cudaStream_t st);
cudaError_t launch_search_f32_ip(const DataView& dv, const SearchArgs& a, const Layout& L, cudaStream_t st);
cudaError_t launch_search_bf16(const DataView& dv, const SearchArgs& a, const Layout& L, cudaStream_t st);
cudaError_t launch_search_batched(const DataView& dv, const SearchArgs& a, const Layout& L, cudaStream_t st);
cudaError_t launch_search_fp8(const DataView& dv, const SearchArgs& a, const Layout& L, cudaStream_t st);

cudaError_t launch_search(const DataView& dv, SearchArgs a, cudaStream_t st) {
  if (a.nq <= 0 && !a.nq_dev) return cudaSuccess;
  // the narrowest tags for which every id splits into slot bits and a tag
  // below the all-ones empty marker (8-bit: 4x the slots of whole ids in the
  // same bytes); in a batched launch a.n is the largest set
  const uint64_t top = (uint64_t)(a.n - 1);
  a.tag_bytes = (top >> (a.log2h + 2)) < 0xffu ? 1 : ((top >> (a.log2h + 1)) < 0xffffu ? 2 : 4);
  Layout L;
  if (!pick_layout(dv.dtype, dv.metric, dv.d, &L)) return cudaErrorNotSupported;
  if (a.sets) return launch_search_batched(dv, a, L, st);
  if (dv.dtype == DT_U8) return launch_search_u8(dv, a, L, st);
  if (dv.dtype == DT_BF16) return launch_search_bf16(dv, a, L, st);
  if (dv.dtype == DT_FP8) {
    if (a.sets || !dv.f32_rows || !dv.scale) return cudaErrorNotSupported;
    a.qrows = dv.f32_rows;
    a.scale = dv.scale;
    return launch_search_fp8(dv, a, L, st);
  }
  if (dv.dtype == DT_F32 && dv.metric == MET_L2) return launch_search_f32_l2(dv, a, L, st);
  if (dv.dtype == DT_F32 && dv.metric == MET_IP) return launch_search_f32_ip(dv, a, L, st);
  return cudaErrorNotSupported;
}

}  // namespace pecann

// ----------------------------------------------------------------- brute-force k-NN

namespace pecann {

struct BfKnnArgs {
  SearchArgs a;         // X, row_bytes, n, C, metric, k, outputs, density_fn, err
  const int32_t* list;  // queries
  const int32_t* cnt;   // number of queries in list (device)
  int64_t max_list;
};

// Exact k nearest points of each listed query over all other points, for the
// queries whose graph search returned fewer than k points (Sec. 4.1). The
// top-k is kept as a sorted beam of width k; every point is a candidate.
template <int DT, int METRIC, int W, int CPL>
__global__ void __launch_bounds__(128) k_bf_knn(BfKnnArgs b) {
  extern __shared__ __align__(16) uint8_t smem[];
  const SearchArgs& a = b.a;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpSmem w = carve(smem + (size_t)wib * a.warp_bytes, a);
  const int gl = lane % W;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t m = min((int64_t)*b.cnt, b.max_list);
  for (int64_t li = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; li < m; li += nwarps) {
    const int32_t q = b.list[li];
    uint4 qv[CPL];
    load_row<W, CPL, false>(a.X + (int64_t)q * a.row_bytes, gl, a.C, qv);
    int nb = 0, cursor = 0;
    for (int64_t j0 = 0; j0 < a.n; j0 += a.stage) {
      int nc = 0;
      for (int bb = 0; bb < a.stage; bb += 32) {
        int64_t j = j0 + bb + lane;
        bool take = j < a.n && j != q;
        unsigned mm = __ballot_sync(FULL, take);
        if (take) w.cids[nc + __popc(mm & lanemask_lt())] = (int32_t)j;
        nc += __popc(mm);
      }
      __syncwarp();
      if (nc) {
        eval_merge<DT, METRIC, W, CPL>(a, w, nc, qv, lane, nb, a.k, cursor);
      }
    }
    const int cnt = min(nb, a.k);
    for (int t = lane; t < a.k; t += 32) {
      int32_t id = -1;
      float dv = INFINITY;
      if (t < cnt) {
        uint64_t e = key_clean(w.beam[t]);
        id = key_id(e);
        dv = out_dist(key_dis(e), a.metric);
      }
      a.out_ids[(int64_t)q * a.k + t] = id;
      a.out_dis[(int64_t)q * a.k + t] = dv;
    }
    __syncwarp();
    if (lane == 0 && cnt == a.k) density_from_beam(w.beam, a.k, a.metric, a.density_fn, a.rho + q, a.rkey + q);
    __syncwarp();
  }
}

template <int DT, int METRIC, int W, int CPL>
static cudaError_t launch_bf_inst(const BfKnnArgs& b, cudaStream_t st) {
  auto kern = k_bf_knn<DT, METRIC, W, CPL>;
  const int wpb = 4;
  size_t smem = (size_t)wpb * b.a.warp_bytes;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = num_sms() * 2;
  kern<<<grid, wpb * 32, smem, st>>>(b); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bruteforce_knn(const DataView& dv, const int32_t* d_list, const int32_t* d_cnt,
                                  int64_t max_list, int k, int32_t* knn_ids, float* knn_dist,
                                  float* rho, float* rkey, int density_fn, int* err, cudaStream_t st) {
  Layout L;
  if (!pick_layout(dv.dtype, dv.metric, dv.d, &L)) return cudaErrorNotSupported;
  BfKnnArgs b;
  memset(&b, 0, sizeof(b));
  SearchArgs& a = b.a;
  a.X = dv.X;
  a.row_bytes = dv.row_bytes;
  a.n = dv.n;
  a.C = dv.C;
  a.metric = dv.metric;
  a.Lw = k;
  a.k = k;
  a.stage = 64;
  a.log2h = 0;
  a.mode = MODE_KNN;
  a.warp_bytes = search_warp_bytes(k, 0, a.stage, 0, false);
  a.out_ids = knn_ids;
  a.out_dis = knn_dist;
  a.rho = rho;
  a.rkey = rkey;
  a.density_fn = density_fn;
  a.err = err;
  b.list = d_list;
  b.cnt = d_cnt;
  b.max_list = max_list;
  if ((size_t)4 * a.warp_bytes > 227 * 1024) return cudaErrorInvalidConfiguration;
  return dispatch_layout(dv, [&](auto dt, auto met, auto wv, auto cpl) -> cudaError_t {
    return launch_bf_inst<decltype(dt)::value, decltype(met)::value, decltype(wv)::value, decltype(cpl)::value>(b, st);
  });
  return cudaErrorNotSupported;
}

}  // namespace pecann
