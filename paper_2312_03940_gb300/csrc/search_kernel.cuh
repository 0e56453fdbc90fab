// The beam-search kernel template (Algorithm 1, one query per warp) and its
// launcher. Instantiated per dtype / metric in search_*.cu so that the
// instances compile in parallel.
#pragma once

#include <stdint.h>

#include "dispatch.cuh"
#include "search_common.cuh"

namespace pecann {

// Query side of an FP8 (inner product) row: lane gl's chunks c = gl + W t
// hold a_j = q_j * s_j for the 16 dimensions of row chunk c, from the FP32
// row of q and the per-dimension scales.
template <int W, int CPL>
__device__ __forceinline__ void load_query_fp8(const SearchArgs& a, int32_t q, int gl, uint4 (&qv)[4 * CPL]) {
  const float4* qr = reinterpret_cast<const float4*>(a.qrows) + wide_mul(q, (int64_t)a.C * 4);
  const float4* sc = reinterpret_cast<const float4*>(a.scale);
#pragma unroll
  for (int t = 0; t < CPL; t++) {
    const int c = gl + W * t;
#pragma unroll
    for (int u = 0; u < 4; u++) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (c < a.C) {
        const float4 x = __ldg(qr + 4 * c + u), s = __ldg(sc + 4 * c + u);
        v = make_float4(x.x * s.x, x.y * s.y, x.z * s.z, x.w * s.w);
      }
      qv[4 * t + u] = make_uint4(__float_as_uint(v.x), __float_as_uint(v.y), __float_as_uint(v.z),
                                 __float_as_uint(v.w));
    }
  }
}

template <int DT, int METRIC, int W, int CPL>
__device__ __forceinline__ void search_one(const SearchArgs& a, WarpSmem& w, int64_t qi, int32_t q, int lane) {
  const int H = 1 << a.log2h;
  const int gl = lane % W;
  if (q < 0 || q >= a.n) {
    if (lane == 0) set_error(a.err, ERR_BAD_ID);
    return;
  }
  uint4 qv[DT == DT_FP8 ? 4 * CPL : CPL];
  if constexpr (DT == DT_FP8) {
    load_query_fp8<W, CPL>(a, q, gl, qv);
  } else if constexpr (DT == DT_U8 && W == 4 && CPL == 2) {
    // the contiguous 32-byte lane chunks of the aligned 128-byte layout
    const uint4* qr = reinterpret_cast<const uint4*>(a.X + wide_mul(q, a.row_bytes)) + 2 * gl;
    qv[0] = ldg_l1(qr);
    qv[1] = ldg_l1(qr + 1);
  } else {
    load_row<W, CPL, false>(a.X + wide_mul(q, a.row_bytes), gl, a.C, qv);
  }
  for (int i = lane; i < H; i += 32) w.hash[i] = -1;
  __syncwarp();
  if (lane == 0) {
    if (a.tag_bytes == 1)
      reinterpret_cast<uint8_t*>(w.hash)[(uint32_t)q & ((4u << a.log2h) - 1)] =
          (uint8_t)((uint32_t)q >> (a.log2h + 2));
    else if (a.tag_bytes == 2)
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
  bool bad = false;  // an id >= n in S or an out-list (reported once below)
  const unsigned lt = lanemask_lt();
  int nc = 0;
  int64_t evals = 0;
  for (int s0 = 0; a.S && s0 < a.nS; s0 += a.stage) {
    nc = gather_start(a, w, q, s0, lane, lt, &bad, &q_in_s);
    if (nc) {
      eval_merge<DT, METRIC, W, CPL>(a, w, nc, qv, lane, nb, a.Lw, cursor);
      evals += nc;
    }
  }
  int64_t iters = 0;
  if (q_in_s) {
    nc = gather_out(a, w, q, q, lane, lt, &bad);
    iters = 1;
    if (nc) {
      eval_merge<DT, METRIC, W, CPL>(a, w, nc, qv, lane, nb, a.Lw, cursor);
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
      prefetch_l2(a.G + wide_mul(key_id(w.beam[next]), a.R) + lane * 32);
    __syncwarp();
    if (lane == 0) w.beam[pos] = e | VFLAG;  // V <- V u {p*}
    __syncwarp();
    cursor = pos + 1;
    const int32_t p = key_id(e);
    if (a.mode == MODE_BUILD) record_visit(w, nv, a.vcap, key_clean(e), lane);
    // L <- L u E_out(p*), keeping the Lw closest
    nc = gather_out(a, w, p, q, lane, lt, &bad);
    if (nc) {
      eval_merge<DT, METRIC, W, CPL>(a, w, nc, qv, lane, nb, a.Lw, cursor);
      evals += nc;
    }
    if (++iters > a.n + 1) {
      if (lane == 0) set_error(a.err, ERR_NO_PROGRESS);
      break;
    }
  }
  if (__any_sync(FULL, bad) && lane == 0) set_error(a.err, ERR_BAD_ID);
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
        a.fb_list[atomicAdd(a.fb_cnt, 1)] = (int32_t)(q + a.id_base);
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

// Point set of global id g: the last set whose base is <= g.
__device__ __forceinline__ int set_of(const int64_t* base, int n_sets, int64_t g) {
  int lo = 0, hi = n_sets - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Arguments of one set of a batched launch: its rows, graph and the slices
// of the concatenated outputs.
__device__ __forceinline__ void apply_set(SearchArgs& la, const SetDesc& d, int64_t base) {
  la.X = d.X;
  la.G = d.G;
  la.n = d.n;
  la.row_bytes = d.row_bytes;
  la.C = d.C;
  la.id_base = base;
  if (la.out_ids) la.out_ids += base * la.k;
  if (la.out_dis) la.out_dis += base * la.k;
  if (la.rho) la.rho += base;
  if (la.rkey) la.rkey += base;
  if (la.rank_key) la.rank_key += base;
  if (la.lam) la.lam += base;
  if (la.delta) la.delta += base;
}

// Resident 256-thread blocks per SM that the register allocation of an
// instance is sized for: wide query rows (FP8 with 2 chunks a lane, FP32 with
// 8, batched FP32 with 4 or more) and BF16 (its query is held unpacked) need
// more than 64 registers to stay free of spills; shared memory caps these at
// 2-4 blocks anyway. (Batched FP32 with 3 chunks a lane spills a few bytes at
// 4 blocks, which measured faster than 3 spill-free blocks.)
template <int DT, int CPL, bool BATCHED>
constexpr int search_min_blocks() {
  if ((DT == DT_FP8 && CPL >= 2) || CPL >= 8 || (BATCHED && CPL >= 4)) return 2;
  if (DT == DT_BF16) return 3;
  if (BATCHED || CPL >= 3 || DT == DT_U8 || DT == DT_FP8) return 4;
  return 5;
}

template <int DT, int METRIC, int W, int CPL, bool BATCHED>
__global__ void __launch_bounds__(256, search_min_blocks<DT, CPL, BATCHED>()) k_search(SearchArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpSmem w = carve(smem + (size_t)wib * a.warp_bytes, a);
  if (BATCHED) {
    // batched form: warps take global query slots from a device queue; a
    // slot names a point of one of the sets (concatenated id space)
    const int64_t nq = a.nq_dev ? (int64_t)*a.nq_dev : a.nq;
    for (;;) {
      unsigned long long g = 0;
      if (lane == 0) g = atomicAdd(a.queue, 1ull);
      g = __shfl_sync(FULL, g, 0);
      if ((int64_t)g >= nq) break;
      const int64_t gid = a.queries ? (int64_t)__ldg(a.queries + g) : (int64_t)g;
      const int s = set_of(a.set_base, a.n_sets, gid);
      if (a.set_active && !a.set_active[s]) continue;  // this set left the doubling rounds
      const int64_t base = a.set_base[s];
      SearchArgs la = a;
      apply_set(la, a.sets[s], base);
      search_one<DT, METRIC, W, CPL>(la, w, (int64_t)g, (int32_t)(gid - base), lane);
    }
    return;
  }
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t qi = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; qi < a.nq; qi += nwarps) {
    const int32_t q = a.queries ? __ldg(a.queries + qi) : (int32_t)qi;
    search_one<DT, METRIC, W, CPL>(a, w, qi, q, lane);
  }
}

// ----------------------------------------------------------------- layouts

template <int DT, int METRIC, int W, int CPL, bool BATCHED>
inline cudaError_t launch_inst(const SearchArgs& a, cudaStream_t st) {
  auto kern = k_search<DT, METRIC, W, CPL, BATCHED>;
  int wpb = (a.block_warps >= 1 && a.block_warps <= 8) ? a.block_warps : 8;
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
  // the batched form runs a persistent grid over its device queue
  int64_t want = BATCHED ? INT64_MAX : (a.nq + wpb - 1) / wpb;
  int64_t cap = (int64_t)num_sms() * per_sm;
  int grid = (int)(want < cap ? want : cap);
  if (grid < 1) grid = 1;
  kern<<<grid, wpb * 32, smem, st>>>(a); note_launch();
  return cudaGetLastError();
}

}  // namespace pecann
