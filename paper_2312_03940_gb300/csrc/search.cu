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
#include "dispatch.cuh"
#include "search_common.cuh"

namespace pecann {

int search_warp_bytes(int Lw, int log2h, int stage, int vcap, bool build) {
  return search_warp_bytes_impl(Lw, log2h, stage, vcap, build);
}

template <int DT, int METRIC, int W, int CPL>
__global__ void __launch_bounds__(256, 5) k_search(SearchArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpSmem w = carve(smem + (size_t)wib * a.warp_bytes, a);
  const int H = 1 << a.log2h;
  const int gl = lane % W;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t qi = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; qi < a.nq; qi += nwarps) {
    const int32_t q = a.queries ? __ldg(a.queries + qi) : (int32_t)qi;
    if (q < 0 || q >= a.n) {
      if (lane == 0) set_error(a.err, ERR_BAD_ID);
      continue;
    }
    uint4 qv[CPL];
    load_row<W, CPL, false>(a.X + (int64_t)q * a.row_bytes, gl, a.C, qv);
    for (int i = lane; i < H; i += 32) w.hash[i] = -1;
    __syncwarp();
    if (lane == 0) {
      if (a.hash16)
        reinterpret_cast<uint16_t*>(w.hash)[(uint32_t)q & ((2u << a.log2h) - 1)] =
            (uint16_t)((uint32_t)q >> (a.log2h + 1));
      else
        w.hash[hash_slot(q, a.log2h)] = q;
    }
    __syncwarp();
    int nb = 0, cursor = 0, nv = 0;
    // L <- S. A query that is itself in S (always, for the k-NN and
    // dependent searches, whose S is {x_i}) is popped first: its out-list
    // joins L and the query stays out of the beam.
    // A start set larger than the staging area goes through the merge in
    // chunks; keeping the Lw closest of each merge leaves the Lw closest
    // points of S, which is what the first prune of Algorithm 1 keeps.
    bool q_in_s = a.S == nullptr;
    int nc = 0;
    int64_t evals = 0;
    for (int s0 = 0; a.S && s0 < a.nS; s0 += a.stage) {
      nc = gather_start(a, w, q, s0, lane, &q_in_s);
      if (nc) {
        eval_cands<DT, METRIC, W, CPL>(a, w, nc, qv, lane);
        merge_cands(w, nb, a.Lw, nc, cursor, lane);
        evals += nc;
      }
    }
    int64_t iters = 0;
    if (q_in_s) {
      nc = gather_out(a, w, q, q, lane);
      iters = 1;
      if (nc) {
        eval_cands<DT, METRIC, W, CPL>(a, w, nc, qv, lane);
        merge_cands(w, nb, a.Lw, nc, cursor, lane);
        evals += nc;
      }
    }
    for (;;) {
      // p* <- argmin over L \ V
      int next;
      int pos = find_unvisited(w.beam, nb, cursor, lane, &next);
      if (pos < 0) break;
      uint64_t e = w.beam[pos];
      // the runner-up is usually the next point popped: fetch its out-list early
      if (next >= 0 && lane < (a.R * 4 + 127) / 128)
        prefetch_l2(a.G + (int64_t)key_id(w.beam[next]) * a.R + lane * 32);
      __syncwarp();
      if (lane == 0) w.beam[pos] = e | VFLAG;  // V <- V u {p*}
      __syncwarp();
      cursor = pos + 1;
      const int32_t p = key_id(e);
      if (a.mode == MODE_BUILD) record_visit(w, nv, a.vcap, key_clean(e), lane);
      // L <- L u E_out(p*), keeping the Lw closest
      nc = gather_out(a, w, p, q, lane);
      if (nc) {
        eval_cands<DT, METRIC, W, CPL>(a, w, nc, qv, lane);
        merge_cands(w, nb, a.Lw, nc, cursor, lane);
        evals += nc;
      }
      if (++iters > a.n + 1) {
        if (lane == 0) set_error(a.err, ERR_NO_PROGRESS);
        break;
      }
    }
    if (a.work && lane == 0) {
      atomicAdd(a.work, (unsigned long long)iters);
      atomicAdd(a.work + 1, (unsigned long long)evals);
    }
    // ---- epilogues
    if (a.mode == MODE_RAW || a.mode == MODE_KNN) {
      const int cnt = min(nb, a.k);
      const int64_t row = a.mode == MODE_RAW ? qi : (int64_t)q;
      for (int t = lane; t < a.k; t += 32) {
        int32_t id = -1;
        float dv = INFINITY;
        if (t < cnt) {
          uint64_t e = key_clean(w.beam[t]);
          id = key_id(e);
          dv = key_dis(e);
          if (a.mode == MODE_KNN) dv = out_dist(dv, a.metric);
        }
        a.out_ids[row * a.k + t] = id;
        a.out_dis[row * a.k + t] = dv;
      }
      if (a.mode == MODE_RAW) {
        if (lane == 0) a.out_cnt[qi] = cnt;
      } else if (lane == 0) {
        if (cnt < a.k) {
          a.fb_list[atomicAdd(a.fb_cnt, 1)] = q;
        } else {
          density_from_beam(w.beam, a.k, a.metric, a.density_fn, a.rho + q, a.rkey + q);
        }
      }
    } else if (a.mode == MODE_DEPCAND) {
      // reduced-precision rounds: hand the first k returned points ranked
      // above q (in traversal order) to the exact re-rank
      int cnt = 0;
      for (int b = 0; b < nb && cnt < a.k; b += 32) {
        const int t = b + lane;
        bool ok = false;
        int32_t id = -1;
        if (t < nb) {
          id = key_id(key_clean(w.beam[t]));
          ok = ranks_above(a.rank_key, id, q);
        }
        const unsigned m = __ballot_sync(FULL, ok);
        const int pos = cnt + __popc(m & lanemask_lt());
        if (ok && pos < a.k) a.out_ids[qi * a.k + pos] = id;
        cnt += __popc(m);
      }
      if (lane == 0) a.out_cnt[qi] = min(cnt, a.k);
    } else if (a.mode == MODE_DEP) {
      // DPBruteForce over the returned points: the first one ranked above q
      for (int b = 0; b < nb; b += 32) {
        int t = b + lane;
        uint64_t e = 0;
        bool ok = false;
        if (t < nb) {
          e = key_clean(w.beam[t]);
          ok = ranks_above(a.rank_key, key_id(e), q);
        }
        unsigned m = __ballot_sync(FULL, ok);
        if (m) {
          if (lane == __ffs(m) - 1) {
            a.lam[q] = key_id(e);
            a.delta[q] = out_dist(key_dis(e), a.metric);
          }
          break;
        }
      }
    } else {
      const int m = min(nv, a.vcap);
      for (int t = lane; t < m; t += 32) {
        uint64_t e = w.vis[t];
        a.vis_ids[qi * a.vcap + t] = key_id(e);
        a.vis_dis[qi * a.vcap + t] = key_dis(e);
      }
      if (lane == 0) a.vis_cnt[qi] = m;
    }
    __syncwarp();
  }
}

// ----------------------------------------------------------------- layouts

bool pick_layout(int dtype, int metric, int d, Layout* out) {
  int epc = dtype == DT_F32 ? 4 : (dtype == DT_BF16 ? 8 : 16);
  if (d <= 0 || d % epc) return false;
  if (dtype == DT_U8 && (metric != MET_L2 || d > 256)) return false;
  if (dtype == DT_FP8) return false;  // FP8 traversal has no kernel in this build
  int C = d / epc;
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

template <int DT, int METRIC, int W, int CPL>
static cudaError_t launch_inst(const SearchArgs& a, cudaStream_t st) {
  auto kern = k_search<DT, METRIC, W, CPL>;
  int wpb = 8;
  while (wpb > 1 && (size_t)wpb * a.warp_bytes > 200 * 1024) wpb >>= 1;
  size_t smem = (size_t)wpb * a.warp_bytes;
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) {
    set_where("search: shared-memory attribute");
    return e;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem);
  if (e != cudaSuccess) {
    set_where("search: occupancy query");
    return e;
  }
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t want = (a.nq + wpb - 1) / wpb;
  int64_t cap = (int64_t)num_sms() * per_sm;
  int grid = (int)(want < cap ? want : cap);
  if (grid < 1) grid = 1;
  kern<<<grid, wpb * 32, smem, st>>>(a); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_search(const DataView& dv, SearchArgs a, cudaStream_t st) {
  if (a.nq <= 0) return cudaSuccess;
  // 16-bit tags when every id splits into slot bits and a tag below 0xffff
  // (0xffff marks an empty slot)
  a.hash16 = ((uint64_t)(a.n - 1) >> (a.log2h + 1)) < 0xffffu ? 1 : 0;
  return dispatch_layout(dv, [&](auto dt, auto met, auto wv, auto cpl) -> cudaError_t {
    return launch_inst<decltype(dt)::value, decltype(met)::value, decltype(wv)::value, decltype(cpl)::value>(a, st);
  });
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
        eval_cands<DT, METRIC, W, CPL>(a, w, nc, qv, lane);
        merge_cands(w, nb, a.k, nc, cursor, lane);
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
