// HCNNG graph index (Sec. 5.1, graph indices: the framework's HCNNG option,
// repeated num_repeats times and pruned with alpha; the paper names the method
// without its steps). Deterministic form of Munoz et al.'s construction:
//   for each repeat t, split the points hierarchically: a node [b, b + m) of
//   the current order with more than leaf_size points draws two pivots
//   p1 != p2 from its points (SplitMix64 keyed by (seed, t, b, m), below);
//   points with dis(x, p1) <= dis(x, p2) go left, the rest right, each side
//   keeping its order (a split that leaves a side empty cuts the node at
//   ceil(m / 2)). The order starts as 0..n-1, so a node lists its points in
//   ascending id;
//   in every leaf, a minimum spanning forest with degrees bounded by mst_deg:
//   the leaf's pairs in (dis, smaller id, larger id) order, each taken when
//   it joins two components and both ends are below the bound;
//   C(u) = u's neighbours in the forests of all repeats;
//   G(u) = RobustPrune(u, C(u), alpha, R) (the build's prune step, no
//   reverse edges).
//
// GPU form: the splits run level by level over all nodes of a level at once
// (pivot draws, one warp per point for its two pivot distances, a prefix sum
// of the "right" flags over the order, a stable scatter per node); the leaf
// forests take one CTA per leaf (pair distances by warps, a bitonic sort of
// the pair keys in shared memory, then Kruskal's scan by one thread with a
// union-find in shared memory).
#include <string.h>

#include <algorithm>
#include <vector>

#include "dispatch.cuh"
#include "search_common.cuh"

namespace pecann {

constexpr int HC_THREADS = 512;
constexpr int HC_SCAN = 1024;     // elements per block of the prefix sum

// SplitMix64 (Steele, Lea and Flood 2014): the output for state x.
__host__ __device__ __forceinline__ uint64_t hc_sm64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Draw j of node [b, b + m) of tree t: v = S(seed + t), v = S(v + b),
// v = S(v + m), draw = S(v + j).
__host__ __device__ __forceinline__ uint64_t hc_draw(uint64_t seed, int t, int64_t b, int64_t m, int j) {
  uint64_t v = hc_sm64(seed + (uint64_t)t);
  v = hc_sm64(v + (uint64_t)b);
  v = hc_sm64(v + (uint64_t)m);
  return hc_sm64(v + (uint64_t)j);
}

struct HcArgs {
  SearchArgs a;            // rows, row_bytes, n, C (the scoring of eval_cands)
  uint64_t seed;
  int t;
  int leaf;
  int mst_deg;
  // splits
  const int32_t* order;    // current order
  int32_t* order2;         // next order
  int32_t* node_of;        // per position: its active node, -1 in a leaf
  const int64_t* nb;       // active nodes: begin, size
  const int64_t* nm;
  int64_t nn;
  int32_t* piv;            // 2 per active node
  int32_t* flag;           // per position: 1 = right
  int32_t* pref;           // n + 1: exclusive prefix sum of flag
  int32_t* bsum;           // per scan block
  int64_t nblocks;
  int32_t* lsize;          // per active node: left size
  int32_t* degen;          // per active node: the split left a side empty
  int64_t* next_b;         // active nodes of the next level
  int64_t* next_m;
  int64_t* leaf_b;         // leaves
  int64_t* leaf_m;
  unsigned long long* counters;  // [0] next active nodes, [1] leaves
  // leaf forests
  int64_t nleaves;
  int32_t* cand;           // n x cap neighbour ids
  float* cand_dis;
  int32_t* ncand;
  int cap;
};

__global__ void k_hc_pivots(HcArgs h) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < h.nn; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = h.nb[k], m = h.nm[k];
    const int64_t i1 = (int64_t)(hc_draw(h.seed, h.t, b, m, 0) % (uint64_t)m);
    int64_t i2 = (int64_t)(hc_draw(h.seed, h.t, b, m, 1) % (uint64_t)(m - 1));
    if (i2 >= i1) i2++;
    h.piv[2 * k] = h.order[b + i1];
    h.piv[2 * k + 1] = h.order[b + i2];
  }
}

// node_of[i] = k for the positions of active node k (one block per node).
__global__ void k_hc_node_of(HcArgs h) {
  for (int64_t k = blockIdx.x; k < h.nn; k += gridDim.x) {
    const int64_t b = h.nb[k], m = h.nm[k];
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) h.node_of[b + i] = (int32_t)k;
  }
}

// flag[i] = 1 when the point at position i is closer to its node's second
// pivot (dis(x, p1) > dis(x, p2)); one warp per position.
template <int DT, int METRIC, int W, int CPL>
__global__ void __launch_bounds__(128) k_hc_side(HcArgs h) {
  __shared__ uint64_t ckeys[4][32];
  __shared__ int32_t cids[4][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpSmem w;
  memset(&w, 0, sizeof(w));
  w.ckeys = ckeys[wib];
  w.cids = cids[wib];
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; i < h.a.n; i += nw) {
    const int32_t k = h.node_of[i];
    if (k < 0) {
      if (lane == 0) h.flag[i] = 0;
      continue;
    }
    const int32_t x = h.order[i], p1 = h.piv[2 * k], p2 = h.piv[2 * k + 1];
    uint4 qv[CPL];
    load_row<W, CPL, false>(h.a.X + wide_mul(x, h.a.row_bytes), lane % W, h.a.C, qv);
    if (lane == 0) {
      w.cids[0] = p1;
      w.cids[1] = p2;
    }
    __syncwarp();
    eval_cands<DT, METRIC, W, CPL>(h.a, w, 2, qv, lane);  // both keys kept
    if (lane == 0) {
      const uint64_t k0 = w.ckeys[0], k1 = w.ckeys[1];
      const float d1 = key_id(k0) == p1 ? key_dis(k0) : key_dis(k1);
      const float d2 = key_id(k0) == p1 ? key_dis(k1) : key_dis(k0);
      h.flag[i] = d1 <= d2 ? 0 : 1;
    }
    __syncwarp();
  }
}

// Exclusive prefix sum of flag[0..n) into pref[0..n], in blocks of HC_SCAN.
__device__ __forceinline__ int32_t hc_block_scan(int32_t v, int32_t* wsum, int32_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int32_t s = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(FULL, s, o);
      if (lane >= o) s += y;
    }
    wsum[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  const int32_t r = x - v + (wid > 0 ? wsum[wid - 1] : 0);
  if (total) *total = wsum[(blockDim.x >> 5) - 1];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(HC_SCAN) k_hc_scan_local(HcArgs h) {
  __shared__ int32_t wsum[32];
  __shared__ int32_t tot;
  for (int64_t blk = blockIdx.x; blk < h.nblocks; blk += gridDim.x) {
    const int64_t i = blk * HC_SCAN + threadIdx.x;
    const int32_t v = i < h.a.n ? h.flag[i] : 0;
    const int32_t r = hc_block_scan(v, wsum, threadIdx.x == 0 ? &tot : nullptr);
    if (i < h.a.n) h.pref[i] = r;
    __syncthreads();
    if (threadIdx.x == 0) h.bsum[blk] = tot;
    __syncthreads();
  }
}

// One block: exclusive scan of the block sums (in chunks), the total to pref[n].
__global__ void __launch_bounds__(HC_SCAN) k_hc_scan_sums(HcArgs h) {
  __shared__ int32_t wsum[32];
  __shared__ int32_t tot;
  int32_t carry = 0;
  for (int64_t c0 = 0; c0 < h.nblocks; c0 += HC_SCAN) {
    const int64_t i = c0 + threadIdx.x;
    const int32_t v = i < h.nblocks ? h.bsum[i] : 0;
    const int32_t r = hc_block_scan(v, wsum, threadIdx.x == 0 ? &tot : nullptr);
    if (i < h.nblocks) h.bsum[i] = carry + r;
    __syncthreads();
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) h.pref[h.a.n] = carry;
}

__global__ void k_hc_scan_add(HcArgs h) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < h.a.n; i += (int64_t)gridDim.x * blockDim.x)
    h.pref[i] += h.bsum[i / HC_SCAN];
}

// Per active node: the left size (a degenerate split cuts at ceil(m / 2)),
// and its two children, listed as active nodes or leaves.
__global__ void k_hc_split(HcArgs h) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < h.nn; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = h.nb[k], m = h.nm[k];
    int64_t l = m - (int64_t)(h.pref[b + m] - h.pref[b]);
    const bool dg = l == 0 || l == m;
    if (dg) l = (m + 1) / 2;
    h.lsize[k] = (int32_t)l;
    h.degen[k] = dg;
    const int64_t cb[2] = {b, b + l}, cm[2] = {l, m - l};
    for (int s = 0; s < 2; s++) {
      if (cm[s] > h.leaf) {
        const unsigned long long j = atomicAdd(h.counters + 0, 1ull);
        h.next_b[j] = cb[s];
        h.next_m[j] = cm[s];
      } else {
        const unsigned long long j = atomicAdd(h.counters + 1, 1ull);
        h.leaf_b[j] = cb[s];
        h.leaf_m[j] = cm[s];
      }
    }
  }
}

// The next order: each active node's left points, then its right points,
// both in their current order; other positions keep their point.
__global__ void k_hc_scatter(HcArgs h) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < h.a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = h.node_of[i];
    int64_t dst = i;
    if (k >= 0 && !h.degen[k]) {
      const int64_t b = h.nb[k];
      const int64_t ones = h.pref[i] - h.pref[b];
      dst = h.flag[i] ? b + h.lsize[k] + ones : b + (i - b) - ones;
    }
    h.order2[dst] = h.order[i];
  }
}

// Pair keys of a leaf: order bits of dis (32) | smaller local index (8) |
// larger local index (8); local order = ascending id.
__device__ __forceinline__ uint64_t hc_pair_key(float dis, int i, int j) {
  return ((uint64_t)f2ord(dis) << 32) | ((uint32_t)i << 8) | (uint32_t)j;
}

__device__ __forceinline__ int32_t hc_find(int32_t* parent, int32_t x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]];
    x = parent[x];
  }
  return x;
}

// One CTA per leaf: all pair distances (warp per row), a bitonic sort of the
// pair keys in shared memory (padding past the end reads as +inf and never
// moves: every comparator puts its minimum at the lower index), then
// Kruskal's scan with the degree bound by one thread; each taken edge is
// appended to both ends' candidate lists.
// Shared memory: keys[pairs] u64 | ids[leaf] | parent[leaf] | deg[leaf] |
// per warp ckeys[leaf] u64 + cids[leaf].
template <int DT, int METRIC, int W, int CPL>
__global__ void __launch_bounds__(HC_THREADS) k_hc_leaf_forest(HcArgs h) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int L = h.leaf;
  const int P = L * (L - 1) / 2;
  uint64_t* keys = reinterpret_cast<uint64_t*>(smem);
  int32_t* ids = reinterpret_cast<int32_t*>(keys + P);
  int32_t* parent = ids + L;
  int32_t* deg = parent + L;
  // per-warp pieces start on 16-byte boundaries (u64 keys)
  uint8_t* wbase = smem + (((size_t)P * 8 + (size_t)L * 12 + 15) & ~(size_t)15);
  const size_t wstride = ((size_t)L * 12 + 15) & ~(size_t)15;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  WarpSmem w;
  memset(&w, 0, sizeof(w));
  w.ckeys = reinterpret_cast<uint64_t*>(wbase + (size_t)wib * wstride);
  w.cids = reinterpret_cast<int32_t*>(w.ckeys + L);
  for (int64_t lf = blockIdx.x; lf < h.nleaves; lf += gridDim.x) {
    const int64_t b = h.leaf_b[lf];
    const int m = (int)h.leaf_m[lf];
    const int np = m * (m - 1) / 2;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      ids[i] = h.order[b + i];
      parent[i] = i;
      deg[i] = 0;
    }
    __syncthreads();
    // pair keys: row i against j > i, written from row i's offset
    for (int i = wib; i < m - 1; i += nwarps) {
      const int nc = m - 1 - i;
      for (int c = lane; c < nc; c += 32) w.cids[c] = ids[i + 1 + c];
      __syncwarp();
      uint4 qv[CPL];
      load_row<W, CPL, false>(h.a.X + wide_mul(ids[i], h.a.row_bytes), lane % W, h.a.C, qv);
      const int kept = eval_cands<DT, METRIC, W, CPL>(h.a, w, nc, qv, lane);  // every key kept
      const int off = i * (2 * m - i - 1) / 2;
      for (int c = lane; c < kept; c += 32) {
        const uint64_t kk = w.ckeys[c];
        const int32_t id = key_id(kk);
        int lo = i + 1, hi = m - 1;  // local index of id (ids ascending)
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (ids[mid] < id)
            lo = mid + 1;
          else
            hi = mid;
        }
        keys[off + c] = hc_pair_key(key_dis(kk), i, lo);
      }
      __syncwarp();
    }
    __syncthreads();
    int Pp = 1;
    while (Pp < np) Pp <<= 1;
    for (int k = 2; k <= Pp; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < Pp; i += blockDim.x) {
          const int q = j == (k >> 1) ? (i ^ (k - 1)) : (i ^ j);
          if (q > i && q < np) {
            const uint64_t x = keys[i], y = keys[q];
            if (y < x) {
              keys[i] = y;
              keys[q] = x;
            }
          }
        }
        __syncthreads();
      }
    }
    if (threadIdx.x == 0) {
      int taken = 0;
      for (int e = 0; e < np && taken < m - 1; e++) {
        const uint64_t kk = keys[e];
        const int i = (int)((kk >> 8) & 0xff), j = (int)(kk & 0xff);
        if (deg[i] >= h.mst_deg || deg[j] >= h.mst_deg) continue;
        const int32_t ri = hc_find(parent, i), rj = hc_find(parent, j);
        if (ri == rj) continue;
        parent[ri < rj ? rj : ri] = ri < rj ? ri : rj;
        deg[i]++;
        deg[j]++;
        taken++;
        const float dis = ord2f((uint32_t)(kk >> 32));
        const int32_t u = ids[i], v = ids[j];
        const int su = atomicAdd(h.ncand + u, 1), sv = atomicAdd(h.ncand + v, 1);
        if (su < h.cap) {
          h.cand[(int64_t)u * h.cap + su] = v;
          h.cand_dis[(int64_t)u * h.cap + su] = dis;
        }
        if (sv < h.cap) {
          h.cand[(int64_t)v * h.cap + sv] = u;
          h.cand_dis[(int64_t)v * h.cap + sv] = dis;
        }
      }
    }
    __syncthreads();
  }
}

size_t prune_lists_ws_bytes(int64_t n);
cudaError_t run_prune_lists(const DataView& dv, int R, float alpha, const int32_t* ids, const float* dis,
                            const int32_t* cnt, int K, int32_t* G, void* ws, int* d_err, cudaStream_t st);

static size_t hc_al(size_t x) { return (x + 255) & ~(size_t)255; }

size_t hcnng_ws_bytes(int64_t n, int repeats, int leaf, int mst_deg) {
  const int64_t nodes = n / (leaf + 1) + 2;  // active nodes hold more than leaf points each
  const int64_t nblocks = (n + HC_SCAN - 1) / HC_SCAN;
  const size_t cap = (size_t)repeats * mst_deg;
  return 4 * hc_al((size_t)n * 4)            // order, order2, node_of, flag
         + hc_al((size_t)(n + 1) * 4)        // pref
         + hc_al((size_t)nblocks * 4)        // bsum
         + 4 * hc_al((size_t)nodes * 8)      // current and next active nodes
         + 2 * hc_al((size_t)nodes * 8)      // piv (2 x int32), lsize + degen
         + 2 * hc_al((size_t)n * 8)          // leaves
         + hc_al(64)                         // counters
         + 2 * hc_al((size_t)n * cap * 4)    // candidate ids and distances
         + hc_al((size_t)n * 4)              // candidate counts
         + prune_lists_ws_bytes(n);
}

static size_t hc_leaf_smem(int leaf) {
  const size_t head = ((size_t)leaf * (leaf - 1) / 2 * 8 + (size_t)leaf * 12 + 15) & ~(size_t)15;
  return head + (size_t)(HC_THREADS / 32) * (((size_t)leaf * 12 + 15) & ~(size_t)15);
}

// HCNNG: fv FP32 or uint8 rows; G n x R; h_leaves (host, may be NULL): the
// number of leaves of each repeat.
cudaError_t run_hcnng(const DataView& fv, int repeats, int leaf, int mst_deg, float alpha, int R, uint64_t seed,
                      int32_t* G, int64_t* h_leaves, void* ws, int* d_err, cudaStream_t st) {
  const int64_t n = fv.n;
  const int64_t nodes = n / (leaf + 1) + 2;
  const int64_t nblocks = (n + HC_SCAN - 1) / HC_SCAN;
  const int cap = repeats * mst_deg;
  uint8_t* wp = (uint8_t*)ws;
  auto take = [&](size_t bytes) {
    uint8_t* r = wp;
    wp += hc_al(bytes);
    return r;
  };
  int32_t* order = (int32_t*)take((size_t)n * 4);
  int32_t* order2 = (int32_t*)take((size_t)n * 4);
  int32_t* node_of = (int32_t*)take((size_t)n * 4);
  int32_t* flag = (int32_t*)take((size_t)n * 4);
  int32_t* pref = (int32_t*)take((size_t)(n + 1) * 4);
  int32_t* bsum = (int32_t*)take((size_t)nblocks * 4);
  int64_t* cur_b = (int64_t*)take((size_t)nodes * 8);
  int64_t* cur_m = (int64_t*)take((size_t)nodes * 8);
  int64_t* nxt_b = (int64_t*)take((size_t)nodes * 8);
  int64_t* nxt_m = (int64_t*)take((size_t)nodes * 8);
  int32_t* piv = (int32_t*)take((size_t)nodes * 8);
  int32_t* lsize = (int32_t*)take((size_t)nodes * 8);
  int32_t* degen = lsize + nodes;
  int64_t* leaf_b = (int64_t*)take((size_t)n * 8);
  int64_t* leaf_m = (int64_t*)take((size_t)n * 8);
  unsigned long long* counters = (unsigned long long*)take(64);
  int32_t* cand = (int32_t*)take((size_t)n * cap * 4);
  float* cand_dis = (float*)take((size_t)n * cap * 4);
  int32_t* ncand = (int32_t*)take((size_t)n * 4);
  void* prune_ws = take(prune_lists_ws_bytes(n));

  HcArgs h;
  memset(&h, 0, sizeof(h));
  h.a.X = fv.X;
  h.a.row_bytes = fv.row_bytes;
  h.a.n = n;
  h.a.C = fv.C;
  h.a.metric = fv.metric;
  h.a.err = d_err;
  h.seed = seed;
  h.leaf = leaf;
  h.mst_deg = mst_deg;
  h.node_of = node_of;
  h.piv = piv;
  h.flag = flag;
  h.pref = pref;
  h.bsum = bsum;
  h.nblocks = nblocks;
  h.lsize = lsize;
  h.degen = degen;
  h.leaf_b = leaf_b;
  h.leaf_m = leaf_m;
  h.counters = counters;
  h.cand = cand;
  h.cand_dis = cand_dis;
  h.ncand = ncand;
  h.cap = cap;
  const int sms = num_sms();
  auto grid = [&](int64_t work, int per) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + per - 1) / per, (int64_t)sms * 16));
  };
  std::vector<int32_t> iota(n);
  for (int64_t i = 0; i < n; i++) iota[i] = (int32_t)i;
  cudaError_t e;
  if ((e = cudaMemsetAsync(ncand, 0, (size_t)n * 4, st)) != cudaSuccess) return e;
  const size_t lsm = hc_leaf_smem(leaf);
  for (int t = 0; t < repeats; t++) {
    h.t = t;
    set_where("hcnng: order");
    if ((e = cudaMemcpyAsync(order, iota.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(counters, 0, 16, st)) != cudaSuccess) return e;
    int32_t* ord = order;
    int32_t* ord2 = order2;
    int64_t nn = 0;
    int64_t nleaves = 0;
    if (n > leaf) {
      const int64_t root[2] = {0, n};
      if ((e = cudaMemcpyAsync(cur_b, &root[0], 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
      if ((e = cudaMemcpyAsync(cur_m, &root[1], 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
      nn = 1;
    } else {
      const int64_t root[2] = {0, n};
      if ((e = cudaMemcpyAsync(leaf_b, &root[0], 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
      if ((e = cudaMemcpyAsync(leaf_m, &root[1], 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
      nleaves = 1;
    }
    int64_t* cb = cur_b;
    int64_t* cm = cur_m;
    int64_t* xb = nxt_b;
    int64_t* xm = nxt_m;
    while (nn > 0) {
      h.order = ord;
      h.order2 = ord2;
      h.nb = cb;
      h.nm = cm;
      h.nn = nn;
      h.next_b = xb;
      h.next_m = xm;
      set_where("hcnng: split");
      if ((e = cudaMemsetAsync(counters, 0, 8, st)) != cudaSuccess) return e;
      if ((e = cudaMemsetAsync(node_of, 0xff, (size_t)n * 4, st)) != cudaSuccess) return e;
      k_hc_pivots<<<grid(nn, 256), 256, 0, st>>>(h); note_launch();
      k_hc_node_of<<<(unsigned)std::min<int64_t>(nn, (int64_t)sms * 16), 256, 0, st>>>(h); note_launch();
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      e = dispatch_layout(fv, [&](auto dt, auto met, auto wv, auto cpl) -> cudaError_t {
        k_hc_side<decltype(dt)::value, decltype(met)::value, decltype(wv)::value, decltype(cpl)::value>
            <<<grid(n, 4), 128, 0, st>>>(h);
        note_launch();
        return cudaGetLastError();
      });
      if (e != cudaSuccess) return e;
      k_hc_scan_local<<<grid(nblocks, 1), HC_SCAN, 0, st>>>(h); note_launch();
      k_hc_scan_sums<<<1, HC_SCAN, 0, st>>>(h); note_launch();
      k_hc_scan_add<<<grid(n, 256), 256, 0, st>>>(h); note_launch();
      k_hc_split<<<grid(nn, 256), 256, 0, st>>>(h); note_launch();
      k_hc_scatter<<<grid(n, 256), 256, 0, st>>>(h); note_launch();
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      unsigned long long c2[2];
      if ((e = cudaMemcpyAsync(c2, counters, 16, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
      nn = (int64_t)c2[0];
      nleaves = (int64_t)c2[1];
      std::swap(ord, ord2);
      std::swap(cb, xb);
      std::swap(cm, xm);
    }
    if (h_leaves) h_leaves[t] = nleaves;
    // the leaf forests
    h.order = ord;
    h.nleaves = nleaves;
    set_where("hcnng: leaf forests");
    e = dispatch_layout(fv, [&](auto dt, auto met, auto wv, auto cpl) -> cudaError_t {
      auto kern = k_hc_leaf_forest<decltype(dt)::value, decltype(met)::value, decltype(wv)::value,
                                   decltype(cpl)::value>;
      cudaError_t ee = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm);
      if (ee != cudaSuccess) return ee;
      kern<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(nleaves, (int64_t)sms * 8)), HC_THREADS, lsm, st>>>(h);
      note_launch();
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
  }
  // G(u) <- RobustPrune(u, C(u), alpha, R)
  return run_prune_lists(fv, R, alpha, cand, cand_dis, ncand, cap, G, prune_ws, d_err, st);
}

}  // namespace pecann
