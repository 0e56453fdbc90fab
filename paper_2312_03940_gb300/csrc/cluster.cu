// Clusters from the dependent forest (Algorithm 2 lines 5-7): noise filter,
// center selection (threshold, or the n_c largest delta * rho by radix
// select), then union-find. Every union links a point to its dependent
// point, so the union-find forest is the dependent forest with the edges of
// noise and center points cut; Find is done by pointer jumping, and each
// point ends up labelled with the root of its tree (order-independent).
#include "common.cuh"
#include "internal.h"

namespace pecann {

struct SelectState {
  unsigned long long prefix;
  unsigned long long mask;
  long long remaining;  // how many of the largest keys are still to be taken
  int all;              // fewer candidates than n_c: every candidate is taken
};

// Product-center key: larger = preferred (product descending, id ascending).
// 0 marks a noise point (never a center).
__global__ void k_center_keys(int64_t n, const float* rho, const float* delta, float rho_min,
                              unsigned long long* keys, unsigned long long* nonnoise) {
  unsigned long long cnt = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float r = rho[i], dl = delta[i];
    unsigned long long kk = 0;
    if (!(r < rho_min)) {
      float prod = (dl == 0.0f || r == 0.0f) ? 0.0f : __fmul_rn(dl, r);
      kk = ((unsigned long long)f2ord(prod) << 32) | (0xffffffffu - (uint32_t)i);
      cnt++;
    }
    keys[i] = kk;
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) cnt += __shfl_xor_sync(FULL, cnt, off);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(nonnoise, cnt);
}

__global__ void k_select_init(SelectState* s, const unsigned long long* nonnoise, long long nc) {
  s->prefix = 0;
  s->mask = 0;
  s->remaining = nc;
  s->all = (long long)*nonnoise <= nc;
}

// Histogram of 16-bit digit `pass` (0 = most significant) over the keys that
// match the prefix chosen so far.
__global__ void k_select_hist(int64_t n, const unsigned long long* keys, const SelectState* s, int pass,
                              unsigned* hist) {
  if (s->all) return;
  const int shift = 48 - 16 * pass;
  const unsigned long long prefix = s->prefix, mask = s->mask;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long kk = keys[i];
    if (kk == 0 || (kk & mask) != prefix) continue;
    atomicAdd(hist + ((kk >> shift) & 0xffff), 1u);
  }
}

// One block of 1024 threads: find the digit holding the `remaining`-th
// largest key, fix it in the prefix, clear the histogram for the next pass.
__global__ void __launch_bounds__(1024) k_select_pick(SelectState* s, int pass, unsigned* hist) {
  __shared__ unsigned long long part[1024];
  __shared__ int found_digit;
  __shared__ long long found_above;
  const int t = threadIdx.x;
  if (s->all) return;
  // thread t owns digits [64 (1023 - t), 64 (1023 - t) + 64): thread 0 the top ones
  const int d_hi = 65535 - 64 * t;
  unsigned long long local = 0;
  for (int j = 0; j < 64; j++) local += hist[d_hi - j];
  part[t] = local;
  __syncthreads();
  // inclusive scan over threads (top digits first)
  for (int off = 1; off < 1024; off <<= 1) {
    unsigned long long v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  const long long rem = s->remaining;
  const long long before = t ? (long long)part[t - 1] : 0;
  if (before < rem && (long long)part[t] >= rem) {
    long long acc = before;
    for (int j = 0; j < 64; j++) {
      unsigned h = hist[d_hi - j];
      if (acc + h >= rem) {
        found_digit = d_hi - j;
        found_above = acc;
        break;
      }
      acc += h;
    }
  }
  __syncthreads();
  for (int j = 0; j < 64; j++) hist[d_hi - j] = 0;
  if (t == 0) {
    const int shift = 48 - 16 * pass;
    s->prefix |= (unsigned long long)found_digit << shift;
    s->mask |= 0xffffull << shift;
    s->remaining = rem - found_above;
  }
}

__global__ void k_cluster_parent(int64_t n, const float* rho, const float* delta, const int32_t* lam,
                                 int center_fn, float rho_min, float delta_min,
                                 const unsigned long long* keys, const SelectState* s, const int32_t* knn_ids,
                                 int k, const float* rk, int32_t* parent) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    bool noise = rho[i] < rho_min;
    bool center;
    if (center_fn == PECANN_CENTER_THRESHOLD) {
      center = !noise && delta[i] > delta_min;
    } else if (center_fn == PECANN_CENTER_LOCAL) {
      // ranks above each of its k nearest neighbours
      center = !noise;
      const float ki = rk[i];
      for (int t = 0; t < k && center; t++) {
        const int32_t j = knn_ids[i * k + t];
        if (j >= 0 && j != (int32_t)i) {
          const float kj = rk[j];
          if (kj > ki || (kj == ki && j < (int32_t)i)) center = false;
        }
      }
    } else {
      unsigned long long kk = keys[i];
      center = kk != 0 && (s->all || kk >= s->prefix);
    }
    int32_t l = lam[i];
    parent[i] = (noise || center || l < 0) ? (int32_t)i : l;
  }
}

// One pointer-jumping sweep: parent[i] <- parent[parent[i]]. Concurrent
// updates only ever replace a parent by one of its ancestors.
__global__ void k_jump(int64_t n, int32_t* parent) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t p = parent[i];
    int32_t gp = parent[p];
    if (gp != p) parent[i] = gp;
  }
}

__global__ void k_count_roots(int64_t n, const int32_t* parent, unsigned long long* cnt) {
  unsigned long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    c += parent[i] == (int32_t)i;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) c += __shfl_xor_sync(FULL, c, off);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

cudaError_t run_cluster(int64_t n, const float* rho, const int32_t* lam, const float* delta, int center_fn,
                        float rho_min, float delta_min, int32_t n_clusters, const int32_t* knn_ids, int k,
                        const float* rank_key, int32_t* labels, void* ws, unsigned long long* d_roots,
                        cudaStream_t st) {
  // ws: keys n u64 | hist 65536 u32 | state | counters
  uint8_t* w = (uint8_t*)ws;
  unsigned long long* keys = (unsigned long long*)w;
  w += ((size_t)n * 8 + 255) & ~(size_t)255;
  unsigned* hist = (unsigned*)w;
  w += 65536 * 4;
  SelectState* s = (SelectState*)w;
  w += 256;
  unsigned long long* nonnoise = (unsigned long long*)w;
  const int threads = 256;
  const unsigned blocks = (unsigned)std::min<int64_t>((n + threads - 1) / threads, (int64_t)num_sms() * 8);
  cudaError_t e;
  if (center_fn == PECANN_CENTER_PRODUCT) {
    if ((e = cudaMemsetAsync(nonnoise, 0, 8, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(hist, 0, 65536 * 4, st)) != cudaSuccess) return e;
    k_center_keys<<<blocks, threads, 0, st>>>(n, rho, delta, rho_min, keys, nonnoise); note_launch();
    k_select_init<<<1, 1, 0, st>>>(s, nonnoise, n_clusters); note_launch();
    for (int pass = 0; pass < 4; pass++) {
      k_select_hist<<<blocks, threads, 0, st>>>(n, keys, s, pass, hist); note_launch();
      k_select_pick<<<1, 1024, 0, st>>>(s, pass, hist); note_launch();
    }
  }
  k_cluster_parent<<<blocks, threads, 0, st>>>(n, rho, delta, lam, center_fn, rho_min, delta_min, keys, s,
                                               knn_ids, k, rank_key, labels); note_launch();
  int sweeps = 1;
  while (((int64_t)1 << sweeps) < n) sweeps++;
  for (int it = 0; it <= sweeps; it++) {
    k_jump<<<blocks, threads, 0, st>>>(n, labels); note_launch();
  }
  if (d_roots) {
    if ((e = cudaMemsetAsync(d_roots, 0, 8, st)) != cudaSuccess) return e;
    k_count_roots<<<blocks, threads, 0, st>>>(n, labels, d_roots); note_launch();
  }
  return cudaGetLastError();
}

size_t cluster_ws_bytes(int64_t n) { return (((size_t)n * 8 + 255) & ~(size_t)255) + 65536 * 4 + 256 + 256; }

}  // namespace pecann
