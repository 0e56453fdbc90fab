// Dependent points (Algorithm 3) outside the beam search itself: round 0
// over the k-NN lists, the global maximum, compaction of the unfinished
// points, the exact brute-force tail, and the normalised density pass.
#include "common.cuh"
#include "dispatch.cuh"
#include "internal.h"

namespace pecann {

// Rank key of a point as one integer: larger = ranked higher (key
// descending, then id ascending).
__device__ __forceinline__ unsigned long long rank64(const float* rk, int32_t i) {
  return ((unsigned long long)f2ord(__ldg(rk + i)) << 32) | (0xffffffffu - (uint32_t)i);
}

// Round 0: lambda_i <- DPBruteForce(x_i, N_i), N_i sorted by (dis, id), so
// the first point of N_i ranked above x_i is the closest one.
__global__ void k_dep_round0(int64_t n, int k, const int32_t* knn_ids, const float* knn_dist,
                             const float* rk, int32_t* lam, float* delta) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t best = -1;
    float bd = INFINITY;
    for (int t = 0; t < k; t++) {
      int32_t j = knn_ids[i * k + t];
      if (j >= 0 && ranks_above(rk, j, (int32_t)i)) {
        best = j;
        bd = knn_dist[i * k + t];
        break;
      }
    }
    lam[i] = best;
    delta[i] = bd;
  }
}

// The point of maximum rank (it has no dependent point).
__global__ void k_rank_max(int64_t n, const float* rk, unsigned long long* out) {
  unsigned long long best = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long v = rank64(rk, (int32_t)i);
    best = v > best ? v : best;
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    unsigned long long o = __shfl_xor_sync(FULL, best, off);
    best = o > best ? o : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

// P_unfinished <- par-filter(src, lambda_i = none), the maximum excluded.
// src == NULL means all points 0..m-1.
__global__ void k_compact_unfinished(const int32_t* src, int64_t m, const int32_t* lam,
                                     const unsigned long long* gmax, int32_t* dst, int32_t* cnt) {
  const int32_t top = (int32_t)(0xffffffffu - (uint32_t)(*gmax & 0xffffffffu));
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < m;
       u += (int64_t)gridDim.x * blockDim.x) {
    int32_t i = src ? src[u] : (int32_t)u;
    bool keep = lam[i] < 0 && i != top;
    unsigned bm = __ballot_sync(FULL, keep);
    int base = 0;
    if ((threadIdx.x & 31) == 0 && bm) base = atomicAdd(cnt, __popc(bm));
    base = __shfl_sync(FULL, base, 0);
    if (keep) dst[base + __popc(bm & lanemask_lt())] = i;
  }
}

// Exact tail: lambda_i <- DPBruteForce(x_i, P) for the listed points. Block b
// scans points [b*chunk, (b+1)*chunk) against the listed queries, TAIL_QT at
// a time: the query rows are staged in shared memory, each group of W lanes
// holds one point row in registers and scores it against every staged query,
// so a point row is read once per TAIL_QT queries. The smallest (dis, id) key
// among points ranked above each query is kept in shared memory and merged
// into best[u] with one atomicMin per (block, query).
static const int DEP_TAIL_QT = 32;

template <int DT, int METRIC, int W, int CPL>
__global__ void __launch_bounds__(256) k_dep_bf(const uint8_t* X, int64_t row_bytes, int64_t n, int C,
                                                 const int32_t* list, int64_t m, const float* rk,
                                                 int64_t chunk, unsigned long long* best) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ unsigned long long tile_best[DEP_TAIL_QT];
  __shared__ int32_t tile_q[DEP_TAIL_QT];
  __shared__ float tile_rk[DEP_TAIL_QT];
  constexpr int GR = 32 / W;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int g = lane / W, gl = lane % W;
  const int64_t j0 = (int64_t)blockIdx.x * chunk;
  const int64_t j1 = min(n, j0 + chunk);
  uint4* qrows = reinterpret_cast<uint4*>(smem);  // DEP_TAIL_QT rows of C chunks
  for (int64_t ub = 0; ub < m; ub += DEP_TAIL_QT) {
    const int nq = (int)(m - ub < DEP_TAIL_QT ? m - ub : DEP_TAIL_QT);
    for (int i = threadIdx.x; i < nq * C; i += blockDim.x) {
      const int qq = i / C, c = i % C;
      qrows[qq * C + c] = __ldg(reinterpret_cast<const uint4*>(X + (int64_t)list[ub + qq] * row_bytes) + c);
    }
    if (threadIdx.x < DEP_TAIL_QT) {
      tile_best[threadIdx.x] = KEY_NONE;
      if (threadIdx.x < nq) {
        const int32_t q = list[ub + threadIdx.x];
        tile_q[threadIdx.x] = q;
        tile_rk[threadIdx.x] = __ldg(rk + q);
      }
    }
    __syncthreads();
    for (int64_t jb = j0 + (int64_t)wib * GR; jb < j1; jb += (int64_t)nw * GR) {
      const int64_t j = jb + g;
      uint4 r[CPL];
      float rkj = 0.0f;
      if (j < j1) {
        load_row<W, CPL, false>(X + j * row_bytes, gl, C, r);
        rkj = __ldg(rk + j);
      } else {
#pragma unroll
        for (int t = 0; t < CPL; t++) r[t] = make_uint4(0, 0, 0, 0);
      }
      for (int qq = 0; qq < nq; qq++) {
        uint4 qv[CPL];
#pragma unroll
        for (int t = 0; t < CPL; t++) {
          const int ch = gl + W * t;
          qv[t] = ch < C ? qrows[qq * C + ch] : make_uint4(0, 0, 0, 0);
        }
        const float dv = group_dis<DT, METRIC, W, CPL>(qv, r);
        const int32_t q = tile_q[qq];
        const float rkq = tile_rk[qq];
        // j ranks above q: larger key, or equal key and smaller id
        if (gl == 0 && j < j1 && j != q && (rkj > rkq || (rkj == rkq && j < q))) {
          const unsigned long long kk = make_key(dv, (int32_t)j);
          if (kk < tile_best[qq]) atomicMin(tile_best + qq, kk);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < nq && tile_best[threadIdx.x] != KEY_NONE) atomicMin(best + ub + threadIdx.x, tile_best[threadIdx.x]);
    __syncthreads();
  }
}

// DPBruteForce for uint8 rows of at most 8 16-byte chunks (d <= 128): one
// point per thread with its row in registers, scored against a tile of up to
// DEP_TAIL_QT queries broadcast from shared memory (integer distances: any
// summation order is exact). A thread keeps its best key per query; warp
// minima (two 32-bit reductions: distance bits, then id), a shared-memory
// minimum and one atomicMin per query and block combine them.
__global__ void __launch_bounds__(256) k_dep_bf_u8(const uint8_t* X, int64_t row_bytes, int64_t n, int C,
                                                   const int32_t* list, int64_t m, const float* rk,
                                                   int64_t chunk, unsigned long long* best) {
  constexpr int CM = 8;
  __shared__ uint4 qrows[DEP_TAIL_QT * CM];
  __shared__ unsigned long long tile_best[DEP_TAIL_QT];
  __shared__ int32_t tile_q[DEP_TAIL_QT];
  __shared__ float tile_rk[DEP_TAIL_QT];
  const int lane = threadIdx.x & 31;
  const int64_t j0 = (int64_t)blockIdx.x * chunk;
  const int64_t j1 = min(n, j0 + chunk);
  for (int64_t ub = 0; ub < m; ub += DEP_TAIL_QT) {
    const int nq = (int)(m - ub < DEP_TAIL_QT ? m - ub : DEP_TAIL_QT);
    for (int i = threadIdx.x; i < DEP_TAIL_QT * CM; i += blockDim.x) {
      const int qq = i / CM, c = i % CM;
      qrows[i] = (qq < nq && c < C)
                     ? __ldg(reinterpret_cast<const uint4*>(X + (int64_t)list[ub + qq] * row_bytes) + c)
                     : make_uint4(0, 0, 0, 0);
    }
    if (threadIdx.x < DEP_TAIL_QT) {
      tile_best[threadIdx.x] = KEY_NONE;
      const bool live = threadIdx.x < nq;
      tile_q[threadIdx.x] = live ? list[ub + threadIdx.x] : -1;
      tile_rk[threadIdx.x] = live ? __ldg(rk + list[ub + threadIdx.x]) : 0.0f;
    }
    __syncthreads();
    unsigned long long bq[DEP_TAIL_QT];
#pragma unroll
    for (int qq = 0; qq < DEP_TAIL_QT; qq++) bq[qq] = KEY_NONE;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
      const uint4* rp = reinterpret_cast<const uint4*>(X + j * row_bytes);
      uint4 r[CM];
#pragma unroll
      for (int c = 0; c < CM; c++) r[c] = c < C ? __ldg(rp + c) : make_uint4(0, 0, 0, 0);
      const float rkj = __ldg(rk + j);
#pragma unroll
      for (int qq = 0; qq < DEP_TAIL_QT; qq++) {
        if (qq < nq) {
          unsigned acc = 0;
#pragma unroll
          for (int c = 0; c < CM; c++) {
            const uint4 qv = qrows[qq * CM + c];
            const unsigned a0 = __vabsdiffu4(qv.x, r[c].x), a1 = __vabsdiffu4(qv.y, r[c].y);
            const unsigned a2 = __vabsdiffu4(qv.z, r[c].z), a3 = __vabsdiffu4(qv.w, r[c].w);
            acc = __dp4a(a0, a0, acc);
            acc = __dp4a(a1, a1, acc);
            acc = __dp4a(a2, a2, acc);
            acc = __dp4a(a3, a3, acc);
          }
          const int32_t q = tile_q[qq];
          const float rkq = tile_rk[qq];
          // j ranks above q: larger key, or equal key and smaller id
          if (j != q && (rkj > rkq || (rkj == rkq && j < q))) {
            const unsigned long long kk = make_key((float)acc, (int32_t)j);
            bq[qq] = kk < bq[qq] ? kk : bq[qq];
          }
        }
      }
    }
#pragma unroll
    for (int qq = 0; qq < DEP_TAIL_QT; qq++) {
      if (qq < nq) {
        const uint32_t hi = (uint32_t)(bq[qq] >> 32);
        const uint32_t mh = __reduce_min_sync(FULL, hi);
        const uint32_t ml = __reduce_min_sync(FULL, hi == mh ? (uint32_t)bq[qq] : 0xffffffffu);
        if (lane == 0 && mh != 0xffffffffu) atomicMin(tile_best + qq, ((unsigned long long)mh << 32) | ml);
      }
    }
    __syncthreads();
    if (threadIdx.x < nq && tile_best[threadIdx.x] != KEY_NONE) atomicMin(best + ub + threadIdx.x, tile_best[threadIdx.x]);
    __syncthreads();
  }
}

__global__ void k_fill_u64(unsigned long long* p, int64_t m, unsigned long long v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void k_dep_bf_finish(const int32_t* list, int64_t m, const unsigned long long* best,
                                int metric, int32_t* lam, float* delta) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < m;
       u += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long kk = best[u];
    if (kk == KEY_NONE) continue;
    int32_t q = list[u];
    lam[q] = key_id(kk);
    delta[q] = out_dist(key_dis(kk), metric);
  }
}

template <int DT, int METRIC, int W, int CPL>
static cudaError_t launch_dep_bf_inst(const DataView& dv, const int32_t* list, int64_t m,
                                      const float* rk, unsigned long long* best, cudaStream_t st) {
  // chunk: enough blocks to fill the GPU, rows of a chunk stay in L1/L2
  int64_t blocks_target = (int64_t)num_sms() * 4;
  int64_t chunk = (dv.n + blocks_target - 1) / blocks_target;
  if (chunk < 256) chunk = 256;
  int64_t grid = (dv.n + chunk - 1) / chunk;
  const size_t smem = (size_t)DEP_TAIL_QT * dv.C * 16;
  auto kern = k_dep_bf<DT, METRIC, W, CPL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)grid, 256, smem, st>>>(dv.X, dv.row_bytes, dv.n, dv.C, list, m, rk, chunk, best);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_dep_bruteforce(const DataView& dv, const int32_t* d_list, int64_t m,
                                  const float* rank_key, unsigned long long* best, int32_t* lam,
                                  float* delta, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  Layout L;
  if (!pick_layout(dv.dtype, dv.metric, dv.d, &L)) return cudaErrorNotSupported;
  k_fill_u64<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(best, m, KEY_NONE); note_launch();
  cudaError_t e;
  if (dv.dtype == DT_U8 && dv.C <= 8) {
    // one point per thread: about two blocks per SM fit its registers
    const int64_t blocks_target = (int64_t)num_sms() * 2;
    int64_t chunk = (dv.n + blocks_target - 1) / blocks_target;
    if (chunk < 256) chunk = 256;
    const int64_t grid = (dv.n + chunk - 1) / chunk;
    k_dep_bf_u8<<<(unsigned)grid, 256, 0, st>>>(dv.X, dv.row_bytes, dv.n, dv.C, d_list, m, rank_key, chunk, best);
    note_launch();
    e = cudaGetLastError();
  } else {
    e = dispatch_layout(dv, [&](auto dt, auto met, auto wv, auto cpl) -> cudaError_t {
      return launch_dep_bf_inst<decltype(dt)::value, decltype(met)::value, decltype(wv)::value,
                                decltype(cpl)::value>(dv, d_list, m, rank_key, best, st);
    });
  }
  if (e != cudaSuccess) return e;
  k_dep_bf_finish<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(d_list, m, best, dv.metric, lam, delta); note_launch();
  return cudaGetLastError();
}

// rho'_i = rho_i k / sum_{j in N_i} rho_j (Sec. 4.2), from a copy of the raw
// densities; the normalised value is also the rank key.
__global__ void k_normalize_density(int64_t n, int k, const int32_t* knn_ids, const float* raw, float* rho,
                                    float* rk) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int t = 0; t < k; t++) s = __fadd_rn(s, raw[knn_ids[i * k + t]]);
    float r = __fdiv_rn(__fmul_rn(raw[i], (float)k), s);
    rho[i] = r;
    rk[i] = r;
  }
}

}  // namespace pecann
