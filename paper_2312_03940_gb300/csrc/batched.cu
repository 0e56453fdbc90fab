// Batched form: many independent FP32 point sets (uneven sizes, dimensions
// up to the largest set's) run through the whole path -- k-NN + density,
// dependent points (round 0, doubling rounds, brute-force tail) and clusters
// -- with one launch per step for all sets.
//
// Points of all sets share one global id space (set s owns ids base[s] ..
// base[s+1]-1); outputs are concatenated in that order and hold local ids.
// The k-NN pass and every doubling round are single persistent launches in
// which warps take work from a device queue (an atomic slot counter) and map
// a slot to its set by binary search over base[]. Every count that steers the
// work (unfinished points per set, which sets still double) stays on the
// device; the launch sequence depends only on the host-side set sizes, so a
// whole pecann_run_batched call can be captured into a CUDA graph.
//
// The per-set rules are those of the single-set calls: each set has its own
// maximum-rank point, its own "more than dep_threshold unfinished" test, its
// own brute-force tail over its own points and its own n_clusters centers.
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "search_kernel.cuh"

namespace pecann {

cudaError_t launch_search(const DataView& dv, SearchArgs a, cudaStream_t st);
__global__ void k_jump(int64_t n, int32_t* parent);
__global__ void k_center_keys(int64_t n, const float* rho, const float* delta, float rho_min,
                              unsigned long long* keys, unsigned long long* nonnoise);
__global__ void k_fill_u64(unsigned long long* p, int64_t m, unsigned long long v);

static const int MAX_SETS = 4096;
static const int64_t TAIL_CHUNK = 2048;  // points per block of the brute-force tail

// Device table written by pecann_batch_prepare (at the start of the
// workspace, after the 256-byte header).
struct BatchTable {
  SetDesc sets[MAX_SETS];
  int64_t base[MAX_SETS + 1];        // first global id of each set
  int64_t chunk_base[MAX_SETS + 1];  // first tail block of each set
  int32_t ncl[MAX_SETS];             // centers per set (product center)
  int32_t cnt[MAX_SETS];             // unfinished points per set (device-maintained)
  int32_t active[MAX_SETS];          // set still in the doubling rounds
  int32_t gofs[MAX_SETS + 1];        // tail: start of each set in the grouped list
  int32_t gcur[MAX_SETS];            // tail: scatter cursors
  unsigned long long gmax[MAX_SETS]; // rank of the maximum point per set
  unsigned long long thr[MAX_SETS];  // product-center threshold key per set
  int32_t all_centers[MAX_SETS];     // fewer candidates than n_clusters
  int32_t total[4];                  // [0] unfinished (current list), [1] next list
  unsigned long long queue[4];       // work-queue counters
};

__device__ __forceinline__ int b_set_of(const BatchTable* t, int n_sets, int64_t g) {
  return set_of(t->base, n_sets, g);
}

__device__ __forceinline__ unsigned long long b_rank64(const float* rk, int64_t g, int32_t local) {
  return ((unsigned long long)f2ord(__ldg(rk + g)) << 32) | (0xffffffffu - (uint32_t)local);
}

// the maximum-rank point of every set
__global__ void k_b_rank_max(BatchTable* t, int n_sets, int64_t N, const float* rk) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
    const int s = b_set_of(t, n_sets, g);
    atomicMax(t->gmax + s, b_rank64(rk, g, (int32_t)(g - t->base[s])));
  }
}

// round 0: the first point of N_i ranked above x_i (local ids, set-local keys)
__global__ void k_b_round0(const BatchTable* t, int n_sets, int64_t N, int k, const int32_t* knn_ids,
                           const float* knn_dist, const float* rk, int32_t* lam, float* delta) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
    const int s = b_set_of(t, n_sets, g);
    const int64_t off = t->base[s];
    const int32_t i = (int32_t)(g - off);
    int32_t best = -1;
    float bd = INFINITY;
    for (int j = 0; j < k; j++) {
      const int32_t y = knn_ids[g * k + j];
      if (y >= 0 && ranks_above(rk + off, y, i)) {
        best = y;
        bd = knn_dist[g * k + j];
        break;
      }
    }
    lam[g] = best;
    delta[g] = bd;
  }
}

// unfinished points of src (all points when src is NULL), the maximum of
// each set excluded; per-set counts are accumulated in t->cnt
__global__ void k_b_compact(BatchTable* t, int n_sets, const int32_t* src, const int32_t* m_dev, int64_t m_all,
                            const int32_t* lam, int32_t* dst, int32_t* dst_cnt) {
  const int64_t m = src ? (int64_t)*m_dev : m_all;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < m; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = src ? src[u] : u;
    const int s = b_set_of(t, n_sets, g);
    const int32_t local = (int32_t)(g - t->base[s]);
    const int32_t top = (int32_t)(0xffffffffu - (uint32_t)(t->gmax[s] & 0xffffffffu));
    if (lam[g] < 0 && local != top) {
      dst[atomicAdd(dst_cnt, 1)] = (int32_t)g;
      atomicAdd(t->cnt + s, 1);
    }
  }
}

// which sets keep doubling: still active and more than `threshold` unfinished
__global__ void k_b_active(BatchTable* t, int n_sets, int threshold, int first) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sets; s += gridDim.x * blockDim.x)
    t->active[s] = (first || t->active[s]) && t->cnt[s] > threshold;
}

// tail: group the remaining points by set (counts already in t->cnt)
__global__ void k_b_group_offsets(BatchTable* t, int n_sets) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int32_t acc = 0;
    for (int s = 0; s < n_sets; s++) {
      t->gofs[s] = acc;
      t->gcur[s] = acc;
      acc += t->cnt[s];
    }
    t->gofs[n_sets] = acc;
  }
}

__global__ void k_b_group_scatter(BatchTable* t, int n_sets, const int32_t* src, const int32_t* m_dev,
                                  int32_t* grouped) {
  const int64_t m = *m_dev;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < m; u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = src[u];
    const int s = b_set_of(t, n_sets, g);
    grouped[atomicAdd(t->gcur + s, 1)] = g;
  }
}

// brute-force tail: block b scans TAIL_CHUNK points of one set against the
// remaining points of that set, 32 queries at a time: the query rows sit in
// shared memory, each warp keeps one point row in registers and scores it
// against all 32 queries (canonical FP32 distance, W = 32 lanes, CPL chunks
// per lane), so a point row is read once per 32 queries
static const int TAIL_QT = 32;

template <int METRIC, int CPL>
__global__ void __launch_bounds__(256) k_b_dep_bf(const BatchTable* t, int n_sets, const int32_t* grouped,
                                                   const float* rk, unsigned long long* best) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ unsigned long long tile_best[TAIL_QT];
  __shared__ int32_t tile_q[TAIL_QT];
  __shared__ float tile_rk[TAIL_QT];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int s = set_of(t->chunk_base, n_sets, (int64_t)blockIdx.x);
  const SetDesc d = t->sets[s];
  const int64_t off = t->base[s];
  const int64_t j0 = ((int64_t)blockIdx.x - t->chunk_base[s]) * TAIL_CHUNK;
  const int64_t j1 = min(d.n, j0 + TAIL_CHUNK);
  const int u0 = t->gofs[s], u1 = t->gofs[s + 1];
  uint4* qrows = reinterpret_cast<uint4*>(smem);  // TAIL_QT rows of d.C chunks
  const float* rks = rk + off;
  for (int ub = u0; ub < u1; ub += TAIL_QT) {
    const int nq = min(TAIL_QT, u1 - ub);
    for (int i = threadIdx.x; i < nq * d.C; i += blockDim.x) {
      const int qq = i / d.C, c = i % d.C;
      const int32_t q = (int32_t)(grouped[ub + qq] - off);
      qrows[qq * d.C + c] = __ldg(reinterpret_cast<const uint4*>(d.X + (int64_t)q * d.row_bytes) + c);
    }
    if (threadIdx.x < TAIL_QT) {
      tile_best[threadIdx.x] = KEY_NONE;
      if (threadIdx.x < nq) {
        const int32_t q = (int32_t)(grouped[ub + threadIdx.x] - off);
        tile_q[threadIdx.x] = q;
        tile_rk[threadIdx.x] = __ldg(rks + q);
      }
    }
    __syncthreads();
    for (int64_t j = j0 + wib; j < j1; j += nw) {
      uint4 r[CPL];
      load_row<32, CPL, false>(d.X + j * d.row_bytes, lane, d.C, r);
      const float rkj = __ldg(rks + j);
      for (int qq = 0; qq < nq; qq++) {
        uint4 qv[CPL];
#pragma unroll
        for (int c = 0; c < CPL; c++) {
          const int ch = lane + 32 * c;
          qv[c] = ch < d.C ? qrows[qq * d.C + ch] : make_uint4(0, 0, 0, 0);
        }
        const float dv = group_dis<DT_F32, METRIC, 32, CPL>(qv, r);
        const int32_t q = tile_q[qq];
        const float rkq = tile_rk[qq];
        // j ranks above q: larger key, or equal key and smaller id
        if (lane == 0 && j != q && (rkj > rkq || (rkj == rkq && j < q))) {
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

__global__ void k_b_bf_finish(const BatchTable* t, const int32_t* grouped, int n_sets,
                              const unsigned long long* best, int metric, int32_t* lam, float* delta) {
  const int64_t m = t->gofs[n_sets];
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < m; u += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long kk = best[u];
    if (kk == KEY_NONE) continue;
    const int32_t g = grouped[u];
    lam[g] = key_id(kk);
    delta[g] = out_dist(key_dis(kk), metric);
  }
}

// product center per set: radix select of the ncl[s]-th largest key, 8 bits
// at a time, one block per set
__global__ void __launch_bounds__(256) k_b_select(BatchTable* t, int n_sets, const unsigned long long* keys) {
  __shared__ unsigned hist[256];
  __shared__ unsigned long long prefix, mask;
  __shared__ long long remaining;
  __shared__ unsigned long long nonnoise;
  const int s = blockIdx.x;
  if (s >= n_sets) return;
  const int64_t off = t->base[s], n = t->sets[s].n;
  if (threadIdx.x == 0) {
    prefix = 0;
    mask = 0;
    remaining = t->ncl[s];
    nonnoise = 0;
  }
  __syncthreads();
  unsigned long long c = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) c += keys[off + i] != 0;
  atomicAdd(&nonnoise, c);
  __syncthreads();
  if ((long long)nonnoise <= remaining) {
    if (threadIdx.x == 0) {
      t->all_centers[s] = 1;
      t->thr[s] = 1;
    }
    return;
  }
  for (int pass = 0; pass < 8; pass++) {
    const int shift = 56 - 8 * pass;
    hist[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const unsigned long long kk = keys[off + i];
      if (kk != 0 && (kk & mask) == prefix) atomicAdd(hist + ((kk >> shift) & 255), 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long acc = 0;
      for (int dg = 255; dg >= 0; dg--) {
        if (acc + hist[dg] >= remaining) {
          prefix |= (unsigned long long)dg << shift;
          mask |= 255ull << shift;
          remaining -= acc;
          break;
        }
        acc += hist[dg];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    t->all_centers[s] = 0;
    t->thr[s] = prefix;
  }
}

// union-find forest over global ids (parent of a non-root = its dependent point)
__global__ void k_b_parent(const BatchTable* t, int n_sets, int64_t N, const float* rho, const float* delta,
                           const int32_t* lam, int center_fn, float rho_min, float delta_min,
                           const unsigned long long* keys, int32_t* parent) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
    const int s = b_set_of(t, n_sets, g);
    const bool noise = rho[g] < rho_min;
    bool center;
    if (center_fn == PECANN_CENTER_THRESHOLD) {
      center = !noise && delta[g] > delta_min;
    } else {
      const unsigned long long kk = keys[g];
      center = kk != 0 && (t->all_centers[s] || kk >= t->thr[s]);
    }
    const int32_t l = lam[g];
    parent[g] = (noise || center || l < 0) ? (int32_t)g : (int32_t)(t->base[s] + l);
  }
}

__global__ void k_b_local_labels(const BatchTable* t, int n_sets, int64_t N, int32_t* labels) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
    const int s = b_set_of(t, n_sets, g);
    labels[g] -= (int32_t)t->base[s];
  }
}

}  // namespace pecann

namespace pecann {

// exact k-NN fallback of the batched form: one warp per listed global id,
// all points of its set are candidates (the merge keeps the k smallest)
template <int METRIC, int CPL>
__global__ void __launch_bounds__(128) k_b_bf_knn(SearchArgs a, const BatchTable* t, int n_sets,
                                                  const int32_t* list, const int32_t* cnt) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpSmem w = carve(smem + (size_t)wib * a.warp_bytes, a);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t m = *cnt;
  for (int64_t li = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; li < m; li += nw) {
    const int64_t g = list[li];
    const int s = set_of(t->base, n_sets, g);
    const SetDesc d = t->sets[s];
    const int64_t off = t->base[s];
    const int32_t q = (int32_t)(g - off);
    SearchArgs la = a;
    la.X = d.X;
    la.n = d.n;
    la.row_bytes = d.row_bytes;
    la.C = d.C;
    uint4 qv[CPL];
    load_row<32, CPL, false>(d.X + (int64_t)q * d.row_bytes, lane, d.C, qv);
    int nb = 0, cursor = 0;
    for (int64_t j0 = 0; j0 < d.n; j0 += la.stage) {
      int nc = 0;
      for (int bb = 0; bb < la.stage; bb += 32) {
        const int64_t j = j0 + bb + lane;
        const bool take = j < d.n && j != q;
        const unsigned mm = __ballot_sync(FULL, take);
        if (take) w.cids[nc + __popc(mm & lanemask_lt())] = (int32_t)j;
        nc += __popc(mm);
      }
      __syncwarp();
      if (nc) {
        eval_merge<DT_F32, METRIC, 32, CPL>(la, w, nc, qv, lane, nb, a.k, cursor);
      }
    }
    const int c = min(nb, a.k);
    for (int tt = lane; tt < a.k; tt += 32) {
      int32_t id = -1;
      float dv = INFINITY;
      if (tt < c) {
        const uint64_t e = key_clean(w.beam[tt]);
        id = key_id(e);
        dv = out_dist(key_dis(e), a.metric);
      }
      a.out_ids[g * a.k + tt] = id;
      a.out_dis[g * a.k + tt] = dv;
    }
    __syncwarp();
    if (lane == 0 && c == a.k) density_from_beam(w.beam, a.k, a.metric, a.density_fn, a.rho + g, a.rkey + g);
    __syncwarp();
  }
}

// ----------------------------------------------------------------- host side

struct HostPlan {
  int S;
  int64_t N, maxn;
  int maxd, metric;
  int64_t tail_blocks;
  std::vector<int64_t> base, chunk_base;
};

static size_t alb(size_t x) { return (x + 255) & ~(size_t)255; }
static const size_t BHDR = 256;

static pecann_status make_plan(int32_t S, const pecann_dataset* sets, HostPlan* hp) {
  if (S < 1 || S > MAX_SETS || !sets) {
    set_last_error("n_sets must be in 1..4096");
    return PECANN_EINVAL;
  }
  hp->S = S;
  hp->N = 0;
  hp->maxn = 0;
  hp->maxd = 0;
  hp->metric = sets[0].metric;
  hp->base.assign(S + 1, 0);
  hp->chunk_base.assign(S + 1, 0);
  for (int s = 0; s < S; s++) {
    const pecann_dataset& d = sets[s];
    if (!d.data || d.dtype != DT_F32 || d.metric != hp->metric || d.n < 2 || d.d <= 0 || d.d % 4 ||
        d.d > 1024 || (((uintptr_t)d.data) & 15)) {
      set_last_error("batched sets must be FP32, one metric, 16-byte aligned rows, d a multiple of 4 up to 1024, n >= 2");
      return PECANN_EINVAL;
    }
    hp->base[s + 1] = hp->base[s] + d.n;
    hp->chunk_base[s + 1] = hp->chunk_base[s] + (d.n + TAIL_CHUNK - 1) / TAIL_CHUNK;
    hp->maxn = std::max<int64_t>(hp->maxn, d.n);
    hp->maxd = std::max(hp->maxd, d.d);
  }
  hp->N = hp->base[S];
  hp->tail_blocks = hp->chunk_base[S];
  if (hp->N >= ((int64_t)1 << 31)) {
    set_last_error("the sets hold 2^31 points or more");
    return PECANN_EINVAL;
  }
  return PECANN_OK;
}

static size_t batch_ws_bytes(const HostPlan& hp) {
  return BHDR + alb(sizeof(BatchTable)) + 3 * alb((size_t)hp.N * 4) + alb((size_t)hp.N * 8) +
         alb((size_t)hp.N * 4) + alb((size_t)hp.N * 8) + 256;
}

struct BatchWs {
  int* err;
  BatchTable* t;
  int32_t *U0, *U1, *grouped, *fb;
  unsigned long long *best, *keys, *nonnoise;
};

static BatchWs carve_batch(void* ws, const HostPlan& hp) {
  BatchWs b;
  uint8_t* p = (uint8_t*)ws;
  b.err = (int*)p;
  p += BHDR;
  b.t = (BatchTable*)p;
  p += alb(sizeof(BatchTable));
  b.U0 = (int32_t*)p;
  p += alb((size_t)hp.N * 4);
  b.U1 = (int32_t*)p;
  p += alb((size_t)hp.N * 4);
  b.grouped = (int32_t*)p;
  p += alb((size_t)hp.N * 4);
  b.best = (unsigned long long*)p;
  p += alb((size_t)hp.N * 8);
  b.fb = (int32_t*)p;
  p += alb((size_t)hp.N * 4);
  b.keys = (unsigned long long*)p;
  p += alb((size_t)hp.N * 8);
  b.nonnoise = (unsigned long long*)p;
  return b;
}

static int cpl_of(int d) {
  const int C = d / 4;
  return C <= 32 ? 1 : (C <= 64 ? 2 : (C <= 96 ? 3 : (C <= 128 ? 4 : 8)));
}

template <class F>
static cudaError_t dispatch_metric_cpl(int metric, int cpl, F&& f) {
  auto go = [&](auto met) -> cudaError_t {
    if (cpl == 1) return f(met, IC<1>{});
    if (cpl == 2) return f(met, IC<2>{});
    if (cpl == 3) return f(met, IC<3>{});
    if (cpl == 4) return f(met, IC<4>{});
    return f(met, IC<8>{});
  };
  if (metric == MET_IP) return go(IC<MET_IP>{});
  return go(IC<MET_L2>{});
}

}  // namespace pecann

using namespace pecann;

extern "C" pecann_status pecann_batch_workspace_size(int32_t n_sets, const pecann_dataset* sets,
                                                     const pecann_params* p, size_t* bytes) {
  if (!p || !bytes) return set_last_error("NULL argument"), PECANN_EINVAL;
  HostPlan hp;
  pecann_status s = make_plan(n_sets, sets, &hp);
  if (s) return s;
  *bytes = batch_ws_bytes(hp);
  return PECANN_OK;
}

extern "C" pecann_status pecann_batch_prepare(int32_t n_sets, const pecann_dataset* sets, const int32_t* d_graphs,
                                              const int32_t* h_n_clusters, const pecann_params* p, void* ws,
                                              size_t ws_bytes, void* stream) {
  if (!p || !d_graphs || !ws) return set_last_error("NULL argument"), PECANN_EINVAL;
  HostPlan hp;
  pecann_status s = make_plan(n_sets, sets, &hp);
  if (s) return s;
  if (ws_bytes < batch_ws_bytes(hp)) return set_last_error("workspace too small"), PECANN_ENOMEM;
  if (p->R < 1 || p->R > 256) return set_last_error("R must be in 1..256"), PECANN_EINVAL;
  std::vector<uint8_t> host(sizeof(BatchTable), 0);
  BatchTable* t = (BatchTable*)host.data();
  for (int i = 0; i < n_sets; i++) {
    t->sets[i].X = (const uint8_t*)sets[i].data;
    t->sets[i].G = d_graphs + hp.base[i] * p->R;
    t->sets[i].n = sets[i].n;
    t->sets[i].row_bytes = (int64_t)sets[i].d * 4;
    t->sets[i].C = sets[i].d / 4;
    t->ncl[i] = h_n_clusters ? h_n_clusters[i] : p->n_clusters;
  }
  for (int i = 0; i <= n_sets; i++) {
    t->base[i] = hp.base[i];
    t->chunk_base[i] = hp.chunk_base[i];
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync((uint8_t*)ws + BHDR, host.data(), sizeof(BatchTable), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_last_error(std::string("batch prepare: ") + cudaGetErrorString(e));
    return PECANN_ECUDA;
  }
  return PECANN_OK;
}

extern "C" pecann_status pecann_run_batched(int32_t n_sets, const pecann_dataset* sets, const pecann_params* p,
                                            int32_t* d_knn_ids, float* d_knn_dist, float* d_density,
                                            float* d_rank_key, int32_t* d_dep, float* d_dep_dist,
                                            int32_t* d_labels, void* ws, size_t ws_bytes, void* stream) {
  if (!p || !d_knn_ids || !d_knn_dist || !d_density || !d_rank_key || !d_dep || !d_dep_dist || !d_labels || !ws)
    return set_last_error("NULL argument"), PECANN_EINVAL;
  HostPlan hp;
  pecann_status s = make_plan(n_sets, sets, &hp);
  if (s) return s;
  if (ws_bytes < batch_ws_bytes(hp)) return set_last_error("workspace too small"), PECANN_ENOMEM;
  int64_t minn = hp.maxn;
  for (int i = 0; i < n_sets; i++) minn = std::min<int64_t>(minn, sets[i].n);
  if (p->k < 1 || p->k >= minn || p->k > 1024 || p->L_search < p->k || p->L_search > 8192 || p->L_dep < 1 ||
      p->max_dep_beam < 1 || p->max_dep_beam > 8192 || p->density < 0 || p->density > 3 ||
      p->normalize_density || (p->center != PECANN_CENTER_THRESHOLD && p->center != PECANN_CENTER_PRODUCT))
    return set_last_error("batched: k, L_search, L_dep, max_dep_beam, density or center out of range "
                          "(normalised density is not offered in batched form)"),
           PECANN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  BatchWs b = carve_batch(ws, hp);
  BatchTable* t = b.t;
  const int S = n_sets;
  const int64_t N = hp.N;
  const unsigned blocks = (unsigned)std::min<int64_t>((N + 255) / 256, (int64_t)num_sms() * 8);
  const unsigned sblocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((S + 255) / 256, 64));
  auto fail = [&](cudaError_t e, const char* what) -> pecann_status {
    if (e == cudaSuccess) return PECANN_OK;
    set_last_error(std::string("batched ") + what + ": " + cudaGetErrorString(e));
    return e == cudaErrorNotSupported ? PECANN_EUNSUPPORTED : PECANN_ECUDA;
  };
  // dynamic part of the table and the header start from zero
  const size_t dyn = offsetof(BatchTable, cnt);
  cudaError_t e = cudaMemsetAsync(b.err, 0, BHDR, st);
  if (e == cudaSuccess) e = cudaMemsetAsync((uint8_t*)t + dyn, 0, sizeof(BatchTable) - dyn, st);
  if ((s = fail(e, "reset"))) return s;

  DataView dv;
  dv.X = (const uint8_t*)sets[0].data;
  dv.n = hp.maxn;
  dv.d = hp.maxd;
  dv.dtype = DT_F32;
  dv.metric = hp.metric;
  dv.row_bytes = (int64_t)hp.maxd * 4;
  dv.C = hp.maxd / 4;
  int slots = p->hash_slots > 0 ? p->hash_slots : std::max(512, std::min(8 * p->L_search, 16384));
  int log2h = 0;
  while ((1 << log2h) < slots) log2h++;

  // ---- 1. k-NN + density of every point of every set (one persistent launch)
  SearchArgs a;
  memset(&a, 0, sizeof(a));
  a.X = dv.X;
  a.row_bytes = dv.row_bytes;
  a.n = hp.maxn;
  a.C = dv.C;
  a.R = p->R;
  a.nq = N;
  a.Lw = p->L_search;
  a.log2h = log2h;
  a.stage = (std::max(p->R, 64) + 31) & ~31;
  a.mode = MODE_KNN;
  a.metric = hp.metric;
  a.block_warps = p->block_warps;
  a.warp_bytes = search_warp_bytes(a.Lw, a.log2h, a.stage, 0, false);
  a.k = p->k;
  a.out_ids = d_knn_ids;
  a.out_dis = d_knn_dist;
  a.rho = d_density;
  a.rkey = d_rank_key;
  a.density_fn = p->density;
  a.fb_list = b.fb;
  a.fb_cnt = &t->total[2];
  a.err = b.err;
  a.sets = t->sets;
  a.set_base = t->base;
  a.n_sets = S;
  a.queue = &t->queue[0];
  if ((s = fail(launch_search(dv, a, st), "k-NN search"))) return s;
  // exact k-NN where a search returned fewer than k points
  {
    SearchArgs f = a;
    f.Lw = p->k;
    f.stage = 64;
    f.log2h = 0;
    f.warp_bytes = search_warp_bytes(p->k, 0, 64, 0, false);
    const size_t smem = (size_t)4 * f.warp_bytes;
    e = dispatch_metric_cpl(hp.metric, cpl_of(hp.maxd), [&](auto met, auto cpl) -> cudaError_t {
      auto kern = k_b_bf_knn<decltype(met)::value, decltype(cpl)::value>;
      cudaError_t ee = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (ee != cudaSuccess) return ee;
      kern<<<num_sms() * 2, 128, smem, st>>>(f, t, S, b.fb, &t->total[2]);
      note_launch();
      return cudaGetLastError();
    });
    if ((s = fail(e, "k-NN fallback"))) return s;
  }

  // ---- 2. dependent points: maxima, round 0, unfinished points
  k_b_rank_max<<<blocks, 256, 0, st>>>(t, S, N, d_rank_key);
  note_launch();
  k_b_round0<<<blocks, 256, 0, st>>>(t, S, N, p->k, d_knn_ids, d_knn_dist, d_rank_key, d_dep, d_dep_dist);
  note_launch();
  int32_t *U0 = b.U0, *U1 = b.U1;
  k_b_compact<<<blocks, 256, 0, st>>>(t, S, nullptr, nullptr, N, d_dep, U0, &t->total[0]);
  note_launch();
  if ((s = fail(cudaGetLastError(), "round 0"))) return s;
  // doubling rounds: a fixed sequence; each set takes part while it has more
  // than dep_threshold unfinished points
  int64_t kdep = p->L_dep;
  for (int r = 0; r < p->max_dep_rounds && kdep <= p->max_dep_beam; r++, kdep *= 2) {
    k_b_active<<<sblocks, 256, 0, st>>>(t, S, p->dep_threshold, r == 0);
    note_launch();
    e = cudaMemsetAsync(&t->queue[1], 0, 8, st);
    if ((s = fail(e, "queue reset"))) return s;
    SearchArgs dq = a;
    dq.mode = MODE_DEP;
    dq.queries = U0;
    dq.nq_dev = &t->total[0];
    dq.queue = &t->queue[1];
    dq.set_active = t->active;
    dq.Lw = (int)kdep;
    int sl = p->hash_slots > 0 ? p->hash_slots : std::max(512, std::min((int)(8 * kdep), 16384));
    dq.log2h = 0;
    while ((1 << dq.log2h) < sl) dq.log2h++;
    dq.warp_bytes = search_warp_bytes(dq.Lw, dq.log2h, dq.stage, 0, false);
    dq.rank_key = d_rank_key;
    dq.lam = d_dep;
    dq.delta = d_dep_dist;
    dq.out_ids = nullptr;
    dq.out_dis = nullptr;
    dq.rho = nullptr;
    dq.rkey = nullptr;
    if ((s = fail(launch_search(dv, dq, st), "dependent round"))) return s;
    e = cudaMemsetAsync(t->cnt, 0, sizeof(int32_t) * S, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(&t->total[1], 0, 4, st);
    if ((s = fail(e, "counter reset"))) return s;
    k_b_compact<<<blocks, 256, 0, st>>>(t, S, U0, &t->total[0], 0, d_dep, U1, &t->total[1]);
    note_launch();
    e = cudaMemcpyAsync(&t->total[0], &t->total[1], 4, cudaMemcpyDeviceToDevice, st);
    if ((s = fail(e, "compaction"))) return s;
    std::swap(U0, U1);
  }
  // ---- 3. the rest: exact brute force within each set
  k_b_group_offsets<<<1, 32, 0, st>>>(t, S);
  note_launch();
  k_b_group_scatter<<<blocks, 256, 0, st>>>(t, S, U0, &t->total[0], b.grouped);
  note_launch();
  k_fill_u64<<<blocks, 256, 0, st>>>(b.best, N, KEY_NONE);
  note_launch();
  {
    const size_t smem = (size_t)TAIL_QT * (hp.maxd / 4) * 16;
    e = dispatch_metric_cpl(hp.metric, cpl_of(hp.maxd), [&](auto met, auto cpl) -> cudaError_t {
      auto kern = k_b_dep_bf<decltype(met)::value, decltype(cpl)::value>;
      cudaError_t ee = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (ee != cudaSuccess) return ee;
      kern<<<(unsigned)hp.tail_blocks, 256, smem, st>>>(t, S, b.grouped, d_rank_key, b.best);
      note_launch();
      return cudaGetLastError();
    });
    if ((s = fail(e, "brute-force tail"))) return s;
  }
  k_b_bf_finish<<<blocks, 256, 0, st>>>(t, b.grouped, S, b.best, hp.metric, d_dep, d_dep_dist);
  note_launch();
  // ---- 4. clusters per set
  if (p->center == PECANN_CENTER_PRODUCT) {
    k_center_keys<<<blocks, 256, 0, st>>>(N, d_density, d_dep_dist, p->rho_min, b.keys, b.nonnoise);
    note_launch();
    k_b_select<<<S, 256, 0, st>>>(t, S, b.keys);
    note_launch();
  }
  k_b_parent<<<blocks, 256, 0, st>>>(t, S, N, d_density, d_dep_dist, d_dep, p->center, p->rho_min, p->delta_min,
                                     b.keys, d_labels);
  note_launch();
  int sweeps = 1;
  while (((int64_t)1 << sweeps) < hp.maxn) sweeps++;
  for (int it = 0; it <= sweeps; it++) {
    k_jump<<<blocks, 256, 0, st>>>(N, d_labels);
    note_launch();
  }
  k_b_local_labels<<<blocks, 256, 0, st>>>(t, S, N, d_labels);
  note_launch();
  return fail(cudaGetLastError(), "clusters");
}
