// Vamana construction by batched insertion (Sec. 3.2, Sec. 4.1).
//
// Per batch (all steps on the GPU, no host synchronisation inside the loop):
//  1. beam search of every batch point from the start points on the graph
//     as it stood at the batch start (the search kernel in build mode keeps
//     the visit_cap closest expanded points V_p);
//  2. k_prune_new: out(p) <- RobustPrune(p, V_p u N_out(p), alpha, R), one
//     warp per point;
//  3. reverse edges: k_rev_count / k_rev_offsets / k_rev_fill group the new
//     edges p -> y by target y (an offset range per target, claimed with
//     atomics; the content of a range is sorted afterwards, so the result
//     does not depend on the order of the atomics), then k_rev_apply, one
//     warp per target, appends the new sources in id order when they fit and
//     otherwise re-prunes y over N_out(y) u the new sources.
//
// RobustPrune (the DiskANN rule): candidates sorted by (dis to p, id); the
// closest alive candidate p* joins the out-list, and every alive candidate p'
// with alpha^2 * dis(p*, p') <= dis(p, p') is dropped; stop at R.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "dispatch.cuh"
#include "internal.h"

namespace pecann {

constexpr int PRUNE_CAP = 2048;  // candidates staged in shared memory per warp

struct BuildArgs {
  const uint8_t* X;
  int64_t row_bytes;
  int64_t n;
  int C;
  int32_t* G;
  int R;
  float a2;  // alpha^2 in FP32
  // step 2
  const int32_t* batch;
  int64_t m;
  const int32_t* vis_ids;
  const float* vis_dis;
  const int32_t* vis_cnt;
  int vcap;
  int cap_new;  // staging entries for step 2 (power of 2)
  // step 3
  int32_t* cnt;
  int32_t* fillc;
  int32_t* off;
  int32_t* targets;
  int32_t* ntargets;
  int32_t* cursor;
  int32_t* src;
  int32_t* big;
  int32_t* nbig;
  uint64_t* big_keys;  // global staging for targets too large for shared memory
  int32_t* big_alive;
  int big_cap;         // power of 2
  int* err;
};

__device__ __forceinline__ int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Ascending sort of a[0..P) (P a power of 2) by one warp.
__device__ void warp_bitonic_sort(uint64_t* a, int P, int lane) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < P; i += 32) {
        int ixj = i ^ j;
        if (ixj > i) {
          uint64_t x = a[i], y = a[ixj];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[ixj] = x;
          }
        }
      }
      __syncwarp();
    }
  }
}

// Drop repeated keys from the sorted K[0..m) (and KEY_NONE padding) in place;
// returns the new count. A is scratch of m ints.
__device__ int warp_unique(uint64_t* K, int32_t* A, int m, int lane) {
  for (int i = lane; i < m; i += 32) A[i] = (K[i] != KEY_NONE) && (i == 0 || K[i] != K[i - 1]);
  __syncwarp();
  int out = 0;
  for (int b = 0; b < m; b += 32) {
    int i = b + lane;
    bool keep = i < m && A[i];
    uint64_t v = keep ? K[i] : 0;
    unsigned bm = __ballot_sync(FULL, keep);
    __syncwarp();
    if (keep) K[out + __popc(bm & lanemask_lt())] = v;
    out += __popc(bm);
    __syncwarp();
  }
  return out;
}

// RobustPrune over the sorted, unique candidate keys K[0..m) (dis to the
// pruned point, id). Writes the kept ids to out[0..deg) and returns deg.
template <int DT, int METRIC, int W, int CPL>
__device__ int robust_prune_warp(const BuildArgs& b, const uint64_t* K, int32_t* A, int m, int32_t* out,
                                 int lane) {
  constexpr int GR = 32 / W;
  const int g = lane / W, gl = lane % W;
  for (int i = lane; i < m; i += 32) A[i] = i;
  __syncwarp();
  int na = m, deg = 0;
  while (na > 0 && deg < b.R) {
    const int t = A[0];
    const int32_t ps = key_id(K[t]);
    if (lane == 0) out[deg] = ps;
    deg++;
    if (deg == b.R) break;
    uint4 pv[CPL];
    load_row<W, CPL, false>(b.X + (int64_t)ps * b.row_bytes, gl, b.C, pv);
    int keep_n = 0;
    for (int base = 1; base < na; base += GR) {
      const int idx = base + g;
      const int c = idx < na ? A[idx] : -1;
      uint4 r[CPL];
      if (c >= 0) {
        load_row<W, CPL, false>(b.X + (int64_t)key_id(K[c]) * b.row_bytes, gl, b.C, r);
      } else {
#pragma unroll
        for (int u = 0; u < CPL; u++) r[u] = make_uint4(0, 0, 0, 0);
      }
      float dv = group_dis<DT, METRIC, W, CPL>(pv, r);
      bool keep = c >= 0 && gl == 0 && !(__fmul_rn(b.a2, dv) <= key_dis(K[c]));
      unsigned bm = __ballot_sync(FULL, keep);
      __syncwarp();
      if (keep) A[keep_n + __popc(bm & lanemask_lt())] = c;
      keep_n += __popc(bm);
      __syncwarp();
    }
    na = keep_n;
  }
  __syncwarp();
  return deg;
}

// Keys (dis to the point whose row is in qv, id) of ids[0..m) into K.
template <int DT, int METRIC, int W, int CPL>
__device__ void keys_of(const BuildArgs& b, const uint4 (&qv)[CPL], const int32_t* ids, int m, uint64_t* K,
                        int lane) {
  constexpr int GR = 32 / W;
  const int g = lane / W, gl = lane % W;
  for (int base = 0; base < m; base += GR) {
    const int i = base + g;
    uint4 r[CPL];
    if (i < m) {
      load_row<W, CPL, false>(b.X + (int64_t)ids[i] * b.row_bytes, gl, b.C, r);
    } else {
#pragma unroll
      for (int u = 0; u < CPL; u++) r[u] = make_uint4(0, 0, 0, 0);
    }
    float dv = group_dis<DT, METRIC, W, CPL>(qv, r);
    if (gl == 0 && i < m) K[i] = make_key(dv, ids[i]);
  }
  __syncwarp();
}

__device__ __forceinline__ void write_row(int32_t* row, const int32_t* out, int deg, int R, int lane) {
  for (int j = lane; j < R; j += 32) row[j] = j < deg ? out[j] : -1;
  __syncwarp();
}

// Step 2: out(p) <- RobustPrune(p, V_p u N_out(p)) for every batch point.
// Shared memory per warp: K cap_new u64 | A cap_new i32 | ids R i32 | out R i32.
template <int DT, int METRIC, int W, int CPL>
__global__ void __launch_bounds__(128) k_prune_new(BuildArgs b) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const size_t per_warp = (size_t)b.cap_new * 12 + (size_t)b.R * 8;
  uint8_t* base = smem + wib * per_warp;
  uint64_t* K = (uint64_t*)base;
  int32_t* A = (int32_t*)(K + b.cap_new);
  int32_t* ids = A + b.cap_new;
  int32_t* out = ids + b.R;
  const int gl = lane % W;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; t < b.m; t += nw) {
    const int32_t p = b.batch[t];
    int32_t* row = b.G + (int64_t)p * b.R;
    const int nv = min(b.vis_cnt[t], b.vcap);
    for (int i = lane; i < nv; i += 32)
      K[i] = make_key(b.vis_dis[t * b.vcap + i], b.vis_ids[t * b.vcap + i]);
    // current out-neighbours of p (start points may already have some)
    int deg = 0;
    for (int j0 = 0; j0 < b.R; j0 += 32) {
      int j = j0 + lane;
      int32_t y = j < b.R ? row[j] : -1;
      bool ok = y >= 0 && y != p;
      unsigned bm = __ballot_sync(FULL, ok);
      if (ok) ids[deg + __popc(bm & lanemask_lt())] = y;
      deg += __popc(bm);
    }
    __syncwarp();
    uint4 pv[CPL];
    load_row<W, CPL, false>(b.X + (int64_t)p * b.row_bytes, gl, b.C, pv);
    keys_of<DT, METRIC, W, CPL>(b, pv, ids, deg, K + nv, lane);
    int m = nv + deg;
    int P = pow2_at_least(m < 1 ? 1 : m);
    for (int i = m + lane; i < P; i += 32) K[i] = KEY_NONE;
    __syncwarp();
    warp_bitonic_sort(K, P, lane);
    m = warp_unique(K, A, P, lane);
    int d2 = robust_prune_warp<DT, METRIC, W, CPL>(b, K, A, m, out, lane);
    write_row(row, out, d2, b.R, lane);
  }
}

// Step 3a: count the new edges per target; list each target once.
__global__ void k_rev_count(BuildArgs b) {
  const int64_t total = b.m * b.R;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t p = b.batch[e / b.R];
    int32_t y = b.G[(int64_t)p * b.R + e % b.R];
    if (y < 0) continue;
    if (atomicAdd(b.cnt + y, 1) == 0) b.targets[atomicAdd(b.ntargets, 1)] = y;
  }
}

// Step 3b: an offset range of cnt[y] source slots per target.
__global__ void k_rev_offsets(BuildArgs b) {
  const int64_t nt = *b.ntargets;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t y = b.targets[i];
    b.off[y] = atomicAdd(b.cursor, b.cnt[y]);
  }
}

// Step 3c: fill the ranges with the sources.
__global__ void k_rev_fill(BuildArgs b) {
  const int64_t total = b.m * b.R;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t p = b.batch[e / b.R];
    int32_t y = b.G[(int64_t)p * b.R + e % b.R];
    if (y < 0) continue;
    b.src[b.off[y] + atomicAdd(b.fillc + y, 1)] = p;
  }
}

// Step 3d for one target y, with staging K / A of capacity cap (power of 2).
template <int DT, int METRIC, int W, int CPL>
__device__ void rev_apply_one(const BuildArgs& b, int32_t y, uint64_t* K, int32_t* A, int32_t* rowbuf,
                              int32_t* out, int lane) {
  const int c = b.cnt[y];
  const int o = b.off[y];
  int32_t* row = b.G + (int64_t)y * b.R;
  // sources, ascending by id
  int P = pow2_at_least(c < 1 ? 1 : c);
  for (int i = lane; i < P; i += 32) K[i] = i < c ? (uint64_t)(uint32_t)b.src[o + i] : KEY_NONE;
  __syncwarp();
  warp_bitonic_sort(K, P, lane);
  int deg = 0;
  for (int j0 = 0; j0 < b.R; j0 += 32) {
    int j = j0 + lane;
    int32_t v = j < b.R ? row[j] : -1;
    bool ok = v >= 0;
    unsigned bm = __ballot_sync(FULL, ok);
    if (ok) rowbuf[deg + __popc(bm & lanemask_lt())] = v;
    deg += __popc(bm);
  }
  __syncwarp();
  // sources not already out-neighbours of y
  for (int i = lane; i < c; i += 32) {
    int32_t s = (int32_t)K[i];
    bool present = (i > 0 && K[i - 1] == K[i]);
    for (int j = 0; j < deg && !present; j++) present = rowbuf[j] == s;
    A[i] = present ? 0 : 1;
  }
  __syncwarp();
  int ni = 0;
  for (int b0 = 0; b0 < c; b0 += 32) {
    int i = b0 + lane;
    bool keep = i < c && A[i];
    int32_t s = keep ? (int32_t)K[i] : -1;
    unsigned bm = __ballot_sync(FULL, keep);
    __syncwarp();
    if (keep) A[ni + __popc(bm & lanemask_lt())] = s;  // A now holds the new ids
    ni += __popc(bm);
    __syncwarp();
  }
  if (deg + ni <= b.R) {
    for (int i = lane; i < ni; i += 32) row[deg + i] = A[i];
    __syncwarp();
  } else {
    // candidates N_out(y) u new sources, keyed by distance to y
    for (int i = lane; i < ni; i += 32) rowbuf[deg + i] = A[i];  // rowbuf has room: see callers
    __syncwarp();
    const int m = deg + ni;
    uint4 yv[CPL];
    load_row<W, CPL, false>(b.X + (int64_t)y * b.row_bytes, lane % W, b.C, yv);
    keys_of<DT, METRIC, W, CPL>(b, yv, rowbuf, m, K, lane);
    int P2 = pow2_at_least(m);
    for (int i = m + lane; i < P2; i += 32) K[i] = KEY_NONE;
    __syncwarp();
    warp_bitonic_sort(K, P2, lane);
    int mu = warp_unique(K, A, P2, lane);
    int d2 = robust_prune_warp<DT, METRIC, W, CPL>(b, K, A, mu, out, lane);
    write_row(row, out, d2, b.R, lane);
  }
  if (lane == 0) {
    b.cnt[y] = 0;
    b.fillc[y] = 0;
  }
  __syncwarp();
}

// Shared memory per warp: K PRUNE_CAP u64 | A PRUNE_CAP i32 | out R i32;
// rowbuf aliases the upper part of A? no: rowbuf gets its own PRUNE_CAP i32.
template <int DT, int METRIC, int W, int CPL>
__global__ void __launch_bounds__(128) k_rev_apply(BuildArgs b) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const size_t per_warp = (size_t)PRUNE_CAP * 16 + (size_t)b.R * 4;
  uint8_t* base = smem + wib * per_warp;
  uint64_t* K = (uint64_t*)base;
  int32_t* A = (int32_t*)(K + PRUNE_CAP);
  int32_t* rowbuf = A + PRUNE_CAP;
  int32_t* out = rowbuf + PRUNE_CAP;
  const int64_t nt = *b.ntargets;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; i < nt; i += nw) {
    const int32_t y = b.targets[i];
    if (b.cnt[y] + b.R > PRUNE_CAP) {
      if (lane == 0) b.big[atomicAdd(b.nbig, 1)] = y;
      continue;
    }
    rev_apply_one<DT, METRIC, W, CPL>(b, y, K, A, rowbuf, out, lane);
  }
}

// Targets with more new sources than shared memory holds: one warp per
// target with global staging (rare: a point that very many batch points
// link to).
template <int DT, int METRIC, int W, int CPL>
__global__ void __launch_bounds__(32) k_rev_apply_big(BuildArgs b) {
  __shared__ int32_t out[1024];
  const int lane = threadIdx.x & 31;
  const int64_t nb = *b.nbig;
  uint64_t* K = b.big_keys + (size_t)blockIdx.x * b.big_cap;
  int32_t* A = b.big_alive + (size_t)blockIdx.x * b.big_cap * 2;
  int32_t* rowbuf = A + b.big_cap;
  for (int64_t i = blockIdx.x; i < nb; i += gridDim.x)
    rev_apply_one<DT, METRIC, W, CPL>(b, b.big[i], K, A, rowbuf, out, lane);
}

__global__ void k_degree(int64_t n, int R, const int32_t* G, int32_t* deg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int d = 0;
    while (d < R && G[i * R + d] >= 0) d++;
    deg[i] = d;
  }
}

// ----------------------------------------------------------------- host side

static const int BIG_WARPS = 8;

size_t build_ws_bytes(int64_t n, const pecann_params& p, int64_t cap, int vcap) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t R = p.R;
  size_t big_cap = 1;
  while (big_cap < (size_t)(cap + R)) big_cap <<= 1;
  size_t b = 0;
  b += al((size_t)n * 4);                 // order (when generated)
  b += 3 * al((size_t)cap * vcap * 4);    // vis ids, dis (+ slack)
  b += al((size_t)cap * 4);               // vis cnt
  b += 3 * al((size_t)n * 4);             // cnt, fillc, off
  b += 3 * al((size_t)cap * R * 4);       // targets, src, big
  b += al(64);                            // counters
  b += al((size_t)BIG_WARPS * big_cap * 8);
  b += al((size_t)BIG_WARPS * big_cap * 8);
  return b;
}

static void splitmix_order(int64_t n, uint64_t seed, std::vector<int32_t>& perm) {
  // Fisher-Yates with SplitMix64 (Steele, Lea and Flood 2014) as the generator.
  perm.resize(n);
  for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
  uint64_t s = seed;
  for (int64_t i = n - 1; i > 0; i--) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    int64_t j = (int64_t)(z % (uint64_t)(i + 1));
    std::swap(perm[i], perm[j]);
  }
}

int64_t batch_cap_of(int64_t n, float frac) {
  int64_t cap = (int64_t)ceil((double)frac * (double)n);
  return cap < 1 ? 1 : cap;
}

// Steps 2 and 3 for the m points of b.batch, whose candidate lists are
// b.vis_ids / b.vis_dis / b.vis_cnt: prune each point's out-list, then apply
// the reverse edges grouped by target. b.cnt and b.fillc are zero on entry
// and on return.
static cudaError_t prune_reverse_batch(const DataView& dv, BuildArgs& b, int64_t m, int32_t* counters,
                                       cudaStream_t st) {
  const int R = b.R;
  const size_t new_smem_warp = (size_t)b.cap_new * 12 + (size_t)R * 8;
  const int new_wpb = new_smem_warp * 4 <= 200 * 1024 ? 4 : (new_smem_warp * 2 <= 200 * 1024 ? 2 : 1);
  const size_t rev_smem_warp = (size_t)PRUNE_CAP * 16 + (size_t)R * 4;
  const int rev_wpb = 2;
  const int sms = num_sms();
  return dispatch_layout(dv, [&](auto dt, auto met, auto wv, auto cpl) -> cudaError_t {
      constexpr int DT = decltype(dt)::value, MET = decltype(met)::value;
      constexpr int W = decltype(wv)::value, CPL = decltype(cpl)::value;
      auto kn = k_prune_new<DT, MET, W, CPL>;
      size_t sm = new_smem_warp * new_wpb;
      set_where("build: prune attribute");
      cudaError_t ee = cudaFuncSetAttribute(kn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (ee != cudaSuccess) return ee;
      set_where("build: prune launch");
      int64_t blocks = std::min<int64_t>((m + new_wpb - 1) / new_wpb, (int64_t)sms * 8);
      kn<<<(unsigned)blocks, new_wpb * 32, sm, st>>>(b); note_launch();
      if ((ee = cudaGetLastError()) != cudaSuccess) return ee;
      set_where("build: reverse-edge counters");
      if ((ee = cudaMemsetAsync(counters, 0, 64, st)) != cudaSuccess) return ee;
      int64_t edges = m * R;
      unsigned eb = (unsigned)std::min<int64_t>((edges + 255) / 256, (int64_t)sms * 16);
      set_where("build: reverse-edge count");
      k_rev_count<<<eb, 256, 0, st>>>(b); note_launch();
      if ((ee = cudaGetLastError()) != cudaSuccess) return ee;
      set_where("build: reverse-edge offsets");
      k_rev_offsets<<<eb, 256, 0, st>>>(b); note_launch();
      if ((ee = cudaGetLastError()) != cudaSuccess) return ee;
      set_where("build: reverse-edge fill");
      k_rev_fill<<<eb, 256, 0, st>>>(b); note_launch();
      if ((ee = cudaGetLastError()) != cudaSuccess) return ee;
      auto ka = k_rev_apply<DT, MET, W, CPL>;
      size_t sm2 = rev_smem_warp * rev_wpb;
      set_where("build: reverse-edge apply");
      if ((ee = cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2)) != cudaSuccess)
        return ee;
      unsigned ab = (unsigned)std::min<int64_t>((edges + rev_wpb - 1) / rev_wpb, (int64_t)sms * 8);
      ka<<<ab, rev_wpb * 32, sm2, st>>>(b); note_launch();
      k_rev_apply_big<DT, MET, W, CPL><<<BIG_WARPS, 32, 0, st>>>(b); note_launch();
      return cudaGetLastError();
    });
}

__global__ void k_iota_fill(int64_t n, int32_t* iota, int32_t* cnt, int32_t k) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    iota[i] = (int32_t)i;
    if (cnt) cnt[i] = k;
  }
}

static size_t pow2_size(size_t x) {
  size_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

size_t all_prune_ws_bytes(int64_t n, int R) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t big_cap = pow2_size((size_t)n + R);
  return 5 * al((size_t)n * 4) + 3 * al((size_t)n * R * 4) + al(64) + 2 * al((size_t)BIG_WARPS * big_cap * 8);
}

// Steps 2 and 3 of a batch that holds every point, from given candidate
// lists (ids / dis: n x K, sorted by (dis, id), unique) on an empty graph:
// G(p) <- RobustPrune(p, list(p), alpha, R), then the reverse edges of all
// points grouped by target. Used by graph indices built without searches.
cudaError_t run_all_prune(const DataView& dv, int R, float alpha, const int32_t* ids, const float* dis, int K,
                          int32_t* G, void* ws, int* d_err, cudaStream_t st) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int64_t n = dv.n;
  const size_t big_cap = pow2_size((size_t)n + R);
  uint8_t* w = (uint8_t*)ws;
  auto take = [&](size_t bytes) {
    uint8_t* r = w;
    w += al(bytes);
    return r;
  };
  int32_t* iota = (int32_t*)take((size_t)n * 4);
  int32_t* vis_cnt = (int32_t*)take((size_t)n * 4);
  int32_t* cnt = (int32_t*)take((size_t)n * 4);
  int32_t* fillc = (int32_t*)take((size_t)n * 4);
  int32_t* off = (int32_t*)take((size_t)n * 4);
  int32_t* targets = (int32_t*)take((size_t)n * R * 4);
  int32_t* src = (int32_t*)take((size_t)n * R * 4);
  int32_t* big = (int32_t*)take((size_t)n * R * 4);
  int32_t* counters = (int32_t*)take(64);
  uint64_t* big_keys = (uint64_t*)take((size_t)BIG_WARPS * big_cap * 8);
  int32_t* big_alive = (int32_t*)take((size_t)BIG_WARPS * big_cap * 8);
  cudaError_t e;
  set_where("graph prune: clear");
  if ((e = cudaMemsetAsync(G, 0xff, (size_t)n * R * 4, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(cnt, 0, (size_t)n * 4, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(fillc, 0, (size_t)n * 4, st)) != cudaSuccess) return e;
  k_iota_fill<<<(unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8), 256, 0, st>>>(n, iota, vis_cnt,
                                                                                                      K);
  note_launch();
  BuildArgs b;
  memset(&b, 0, sizeof(b));
  b.X = dv.X;
  b.row_bytes = dv.row_bytes;
  b.n = n;
  b.C = dv.C;
  b.G = G;
  b.R = R;
  b.a2 = alpha * alpha;
  b.batch = iota;
  b.m = n;
  b.vis_ids = ids;
  b.vis_dis = dis;
  b.vis_cnt = vis_cnt;
  b.vcap = K;
  b.cap_new = (int)pow2_size((size_t)K + R);
  b.cnt = cnt;
  b.fillc = fillc;
  b.off = off;
  b.targets = targets;
  b.ntargets = counters;
  b.cursor = counters + 1;
  b.nbig = counters + 2;
  b.src = src;
  b.big = big;
  b.big_keys = big_keys;
  b.big_alive = big_alive;
  b.big_cap = (int)big_cap;
  b.err = d_err;
  return prune_reverse_batch(dv, b, n, counters, st);
}

// Step 2 alone for every point, from given candidate lists (ids / dis: n x
// K, any order, repeats allowed; cnt: valid entries per point) on an empty
// graph: G(p) <- RobustPrune(p, list(p), alpha, R). No reverse edges. ws:
// prune_lists_ws_bytes(n) bytes.
size_t prune_lists_ws_bytes(int64_t n) { return ((size_t)n * 4 + 255) & ~(size_t)255; }

cudaError_t run_prune_lists(const DataView& dv, int R, float alpha, const int32_t* ids, const float* dis,
                            const int32_t* cnt, int K, int32_t* G, void* ws, int* d_err, cudaStream_t st) {
  const int64_t n = dv.n;
  int32_t* iota = (int32_t*)ws;
  cudaError_t e;
  set_where("graph prune: clear");
  if ((e = cudaMemsetAsync(G, 0xff, (size_t)n * R * 4, st)) != cudaSuccess) return e;
  k_iota_fill<<<(unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8), 256, 0, st>>>(n, iota, nullptr,
                                                                                                      0);
  note_launch();
  BuildArgs b;
  memset(&b, 0, sizeof(b));
  b.X = dv.X;
  b.row_bytes = dv.row_bytes;
  b.n = n;
  b.C = dv.C;
  b.G = G;
  b.R = R;
  b.a2 = alpha * alpha;
  b.batch = iota;
  b.m = n;
  b.vis_ids = ids;
  b.vis_dis = dis;
  b.vis_cnt = cnt;
  b.vcap = K;
  b.cap_new = (int)pow2_size((size_t)K + R);
  b.err = d_err;
  const size_t new_smem_warp = (size_t)b.cap_new * 12 + (size_t)R * 8;
  const int wpb = new_smem_warp * 4 <= 200 * 1024 ? 4 : (new_smem_warp * 2 <= 200 * 1024 ? 2 : 1);
  return dispatch_layout(dv, [&](auto dt, auto met, auto wv, auto cpl) -> cudaError_t {
    auto kn = k_prune_new<decltype(dt)::value, decltype(met)::value, decltype(wv)::value, decltype(cpl)::value>;
    const size_t sm = new_smem_warp * wpb;
    set_where("graph prune: attribute");
    cudaError_t ee = cudaFuncSetAttribute(kn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (ee != cudaSuccess) return ee;
    set_where("graph prune: launch");
    const int64_t blocks = std::min<int64_t>((n + wpb - 1) / wpb, (int64_t)num_sms() * 8);
    kn<<<(unsigned)blocks, wpb * 32, sm, st>>>(b);
    note_launch();
    return cudaGetLastError();
  });
}

cudaError_t run_build(const DataView& dv, const pecann_params& p, const int32_t* d_order, int32_t* G,
                      int32_t* d_degree, void* ws, int* d_err, int log2h, cudaStream_t st) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int64_t n = dv.n;
  const int R = p.R;
  const int vcap = p.visit_cap > 0 ? p.visit_cap : 2 * p.L_build;
  const int64_t cap = batch_cap_of(n, p.batch_frac);
  size_t big_cap = 1;
  while (big_cap < (size_t)(cap + R)) big_cap <<= 1;
  uint8_t* w = (uint8_t*)ws;
  auto take = [&](size_t bytes) {
    uint8_t* r = w;
    w += al(bytes);
    return r;
  };
  int32_t* order = (int32_t*)take((size_t)n * 4);
  int32_t* vis_ids = (int32_t*)take((size_t)cap * vcap * 4);
  float* vis_dis = (float*)take((size_t)cap * vcap * 4);
  take((size_t)cap * vcap * 4);
  int32_t* vis_cnt = (int32_t*)take((size_t)cap * 4);
  int32_t* cnt = (int32_t*)take((size_t)n * 4);
  int32_t* fillc = (int32_t*)take((size_t)n * 4);
  int32_t* off = (int32_t*)take((size_t)n * 4);
  int32_t* targets = (int32_t*)take((size_t)cap * R * 4);
  int32_t* src = (int32_t*)take((size_t)cap * R * 4);
  int32_t* big = (int32_t*)take((size_t)cap * R * 4);
  int32_t* counters = (int32_t*)take(64);
  uint64_t* big_keys = (uint64_t*)take((size_t)BIG_WARPS * big_cap * 8);
  int32_t* big_alive = (int32_t*)take((size_t)BIG_WARPS * big_cap * 8);
  cudaError_t e;
  if (!d_order) {
    std::vector<int32_t> perm;
    splitmix_order(n, p.seed, perm);
    if ((e = cudaMemcpyAsync(order, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    d_order = order;
  }
  set_where("build: clear graph and counters");
  if ((e = cudaMemsetAsync(G, 0xff, (size_t)n * R * 4, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(cnt, 0, (size_t)n * 4, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(fillc, 0, (size_t)n * 4, st)) != cudaSuccess) return e;

  BuildArgs b;
  memset(&b, 0, sizeof(b));
  b.X = dv.X;
  b.row_bytes = dv.row_bytes;
  b.n = n;
  b.C = dv.C;
  b.G = G;
  b.R = R;
  b.a2 = p.alpha * p.alpha;
  b.vis_ids = vis_ids;
  b.vis_dis = vis_dis;
  b.vis_cnt = vis_cnt;
  b.vcap = vcap;
  int cap_new = 1;
  while (cap_new < vcap + R) cap_new <<= 1;
  b.cap_new = cap_new;
  b.cnt = cnt;
  b.fillc = fillc;
  b.off = off;
  b.targets = targets;
  b.ntargets = counters;
  b.cursor = counters + 1;
  b.nbig = counters + 2;
  b.src = src;
  b.big = big;
  b.big_keys = big_keys;
  b.big_alive = big_alive;
  b.big_cap = (int)big_cap;
  b.err = d_err;

  SearchArgs a;
  memset(&a, 0, sizeof(a));
  a.X = dv.X;
  a.row_bytes = dv.row_bytes;
  a.n = n;
  a.C = dv.C;
  a.G = G;
  a.R = R;
  a.S = d_order;
  a.nS = p.n_start;
  a.Lw = p.L_build;
  a.log2h = log2h;
  a.stage = (std::max(R, 64) + 31) & ~31;
  a.vcap = vcap;
  a.mode = MODE_BUILD;
  a.metric = dv.metric;
  a.block_warps = p.block_warps;
  a.warp_bytes = search_warp_bytes(a.Lw, a.log2h, a.stage, a.vcap, true);
  a.vis_ids = vis_ids;
  a.vis_dis = vis_dis;
  a.vis_cnt = vis_cnt;
  a.err = d_err;

  const int sms = num_sms();
  const int passes = p.build_passes == 2 ? 2 : 1;

  for (int pass = 0; pass < passes; pass++) {
  // two passes: the first prunes with alpha = 1, the second with alpha
  b.a2 = (passes == 2 && pass == 0) ? 1.0f : p.alpha * p.alpha;
  int64_t pos = 0, bsz = 1;
  while (pos < n) {
    int64_t m = std::min(std::min(bsz, cap), n - pos);
    a.queries = d_order + pos;
    a.nq = m;
    set_where("build: batch search");
    if ((e = launch_search(dv, a, st)) != cudaSuccess) return e;
    b.batch = d_order + pos;
    b.m = m;
    e = prune_reverse_batch(dv, b, m, counters, st);
    if (e != cudaSuccess) return e;
    pos += m;
    bsz = std::min(2 * bsz, cap);  // doubling stops at the cap (no overflow)
  }
  }
  if (d_degree) {
    k_degree<<<(unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8), 256, 0, st>>>(n, R, G, d_degree); note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  set_where("build: final synchronize");
  return cudaStreamSynchronize(st);
}

}  // namespace pecann
