// Clusters from the dependent forest (Algorithm 2 lines 5-7): noise filter,
// center selection (threshold, or the n_c largest delta * rho by radix
// select), then union-find. Every union links a point to its dependent
// point, so the union-find forest is the dependent forest with the edges of
// noise and center points cut; Find is done by pointer jumping, and each
// point ends up labelled with the root of its tree (order-independent).
#include <algorithm>
#include <vector>

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

// ---------------------------------------------------------------- many settings in shared passes
//
// A sweep of S settings (Sec. 1: other clusterings from the same dependent
// forest) runs every step once for all settings: one pass computes the
// product keys (without the noise filter, which is per setting), each radix
// pass of the product-center selection histograms every product setting in
// one launch (blockIdx.y = setting), one launch sets all S parent arrays and
// each pointer-jumping sweep advances all S x n entries. The result of every
// setting is that of run_cluster.

namespace pecann {

struct SweepSetting {
  int center;
  float rho_min;
  float delta_min;
  int n_clusters;
};

struct SweepSelect {
  unsigned long long prefix;
  unsigned long long mask;
  long long remaining;
  int all;
  int pad;
};

// Product key of every point (larger = preferred), noise not applied.
__global__ void k_sweep_keys(int64_t n, const float* rho, const float* delta, unsigned long long* keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float r = rho[i], dl = delta[i];
    const float prod = (dl == 0.0f || r == 0.0f) ? 0.0f : __fmul_rn(dl, r);
    keys[i] = ((unsigned long long)f2ord(prod) << 32) | (0xffffffffu - (uint32_t)i);
  }
}

// Non-noise points of product setting blockIdx.y, summed into sel[y].prefix
// (zeroed before; k_sweep_init turns the count into the selection state).
__global__ void k_sweep_count(int64_t n, const float* rho, const SweepSetting* set, const int* prod_ids,
                              SweepSelect* sel) {
  __shared__ unsigned long long tot;
  const int s = prod_ids[blockIdx.y];
  const float rmin = set[s].rho_min;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  unsigned long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += !(rho[i] < rmin);
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) c += __shfl_xor_sync(FULL, c, off);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&tot, c);
  __syncthreads();
  if (threadIdx.x == 0 && tot) atomicAdd(reinterpret_cast<unsigned long long*>(&sel[blockIdx.y].prefix), tot);
}

// After k_sweep_count left the non-noise count in `prefix`: the selection state.
__global__ void k_sweep_init(const SweepSetting* set, const int* prod_ids, int m, SweepSelect* sel) {
  for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < m; y += gridDim.x * blockDim.x) {
    const long long nonnoise = (long long)sel[y].prefix;
    const long long nc = set[prod_ids[y]].n_clusters;
    sel[y].prefix = 0;
    sel[y].mask = 0;
    sel[y].remaining = nc;
    sel[y].all = nonnoise <= nc;
  }
}

// Histogram of 8-bit digit `pass` (0 = most significant) of the non-noise
// keys that match the prefix of product setting blockIdx.y.
__global__ void k_sweep_hist(int64_t n, const unsigned long long* keys, const float* rho, const SweepSetting* set,
                             const int* prod_ids, const SweepSelect* sel, int pass, unsigned* hist) {
  __shared__ unsigned h[256];
  const int y = blockIdx.y;
  if (sel[y].all) return;
  const float rmin = set[prod_ids[y]].rho_min;
  const unsigned long long prefix = sel[y].prefix, mask = sel[y].mask;
  const int shift = 56 - 8 * pass;
  for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long kk = keys[i];
    if (rho[i] < rmin || (kk & mask) != prefix) continue;
    atomicAdd(&h[(kk >> shift) & 0xff], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 256; t += blockDim.x)
    if (h[t]) atomicAdd(hist + (size_t)y * 256 + t, h[t]);
}

// One block per product setting: the digit that holds its remaining-th
// largest key joins the prefix; the histogram is cleared for the next pass.
__global__ void k_sweep_pick(SweepSelect* sel, int pass, unsigned* hist) {
  const int y = blockIdx.x;
  unsigned* hy = hist + (size_t)y * 256;
  if (!sel[y].all && threadIdx.x == 0) {
    const long long rem = sel[y].remaining;
    long long acc = 0;
    int digit = 0;
    for (int dgt = 255; dgt >= 0; dgt--) {
      if (acc + hy[dgt] >= rem) {
        digit = dgt;
        break;
      }
      acc += hy[dgt];
    }
    const int shift = 56 - 8 * pass;
    sel[y].prefix |= (unsigned long long)digit << shift;
    sel[y].mask |= 0xffull << shift;
    sel[y].remaining = rem - acc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 256; t += blockDim.x) hy[t] = 0;
}

// Parent arrays of every setting: parent[s * n + i].
__global__ void k_sweep_parent(int64_t n, int S, const float* rho, const float* delta, const int32_t* lam,
                               const SweepSetting* set, const int* sel_of, const SweepSelect* sel,
                               const unsigned long long* keys, const int32_t* knn_ids, int k, const float* rk,
                               int32_t* parent) {
  const int64_t total = n * (int64_t)S;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(g / n);
    const int64_t i = g - (int64_t)s * n;
    const SweepSetting c = set[s];
    const bool noise = rho[i] < c.rho_min;
    bool center;
    if (c.center == PECANN_CENTER_THRESHOLD) {
      center = !noise && delta[i] > c.delta_min;
    } else if (c.center == PECANN_CENTER_LOCAL) {
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
      const SweepSelect& q = sel[sel_of[s]];
      center = !noise && (q.all || keys[i] >= q.prefix);
    }
    const int32_t l = lam[i];
    parent[g] = (noise || center || l < 0) ? (int32_t)i : l;
  }
}

// One pointer-jumping sweep over every setting's parent array.
__global__ void k_sweep_jump(int64_t n, int S, int32_t* parent) {
  const int64_t total = n * (int64_t)S;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    int32_t* row = parent + (g / n) * n;
    const int32_t p = parent[g];
    const int32_t gp = row[p];
    if (gp != p) parent[g] = gp;
  }
}

__global__ void k_sweep_roots(int64_t n, int S, const int32_t* parent, unsigned long long* cnt) {
  const int s = blockIdx.y;
  unsigned long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += parent[(int64_t)s * n + i] == (int32_t)i;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) c += __shfl_xor_sync(FULL, c, off);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt + s, c);
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t sweep_ws_bytes(int64_t n, int S) {
  return a256((size_t)n * 8) + a256((size_t)S * sizeof(SweepSetting)) + 2 * a256((size_t)S * 4) +
         a256((size_t)S * sizeof(SweepSelect)) + a256((size_t)S * 256 * 4);
}

cudaError_t run_cluster_sweep(int64_t n, const float* rho, const int32_t* lam, const float* delta, int S,
                              const pecann_cluster_setting* h_set, const int32_t* knn_ids, int k,
                              const float* rank_key, int32_t* labels, void* ws, unsigned long long* d_roots,
                              cudaStream_t st) {
  uint8_t* w = (uint8_t*)ws;
  unsigned long long* keys = (unsigned long long*)w;
  w += a256((size_t)n * 8);
  SweepSetting* d_set = (SweepSetting*)w;
  w += a256((size_t)S * sizeof(SweepSetting));
  int* d_prod = (int*)w;  // product settings, in order
  w += a256((size_t)S * 4);
  int* d_selof = (int*)w;  // setting -> its product index
  w += a256((size_t)S * 4);
  SweepSelect* sel = (SweepSelect*)w;
  w += a256((size_t)S * sizeof(SweepSelect));
  unsigned* hist = (unsigned*)w;
  std::vector<SweepSetting> hs((size_t)S);
  std::vector<int> prod, selof((size_t)S, 0);
  for (int s = 0; s < S; s++) {
    hs[s] = {h_set[s].center, h_set[s].rho_min, h_set[s].delta_min, h_set[s].n_clusters};
    if (h_set[s].center == PECANN_CENTER_PRODUCT) {
      selof[s] = (int)prod.size();
      prod.push_back(s);
    }
  }
  const int m = (int)prod.size();
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d_set, hs.data(), (size_t)S * sizeof(SweepSetting), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(d_selof, selof.data(), (size_t)S * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  const int threads = 256;
  const unsigned blocks = (unsigned)std::min<int64_t>((n + threads - 1) / threads, (int64_t)num_sms() * 8);
  if (m > 0) {
    if ((e = cudaMemcpyAsync(d_prod, prod.data(), (size_t)m * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(sel, 0, (size_t)m * sizeof(SweepSelect), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(hist, 0, (size_t)m * 256 * 4, st)) != cudaSuccess) return e;
    k_sweep_keys<<<blocks, threads, 0, st>>>(n, rho, delta, keys); note_launch();
    const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks, std::max<int64_t>(1, 2048 / m)));
    k_sweep_count<<<dim3(bx, (unsigned)m), threads, 0, st>>>(n, rho, d_set, d_prod, sel); note_launch();
    k_sweep_init<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(d_set, d_prod, m, sel); note_launch();
    for (int pass = 0; pass < 8; pass++) {
      k_sweep_hist<<<dim3(bx, (unsigned)m), threads, 0, st>>>(n, keys, rho, d_set, d_prod, sel, pass, hist);
      note_launch();
      k_sweep_pick<<<(unsigned)m, 256, 0, st>>>(sel, pass, hist); note_launch();
    }
  }
  const int64_t total = n * (int64_t)S;
  const unsigned gb = (unsigned)std::min<int64_t>((total + threads - 1) / threads, (int64_t)num_sms() * 16);
  k_sweep_parent<<<gb, threads, 0, st>>>(n, S, rho, delta, lam, d_set, d_selof, sel, keys, knn_ids, k, rank_key,
                                         labels); note_launch();
  int sweeps = 1;
  while (((int64_t)1 << sweeps) < n) sweeps++;
  for (int it = 0; it <= sweeps; it++) {
    k_sweep_jump<<<gb, threads, 0, st>>>(n, S, labels); note_launch();
  }
  if (d_roots) {
    if ((e = cudaMemsetAsync(d_roots, 0, (size_t)S * 8, st)) != cudaSuccess) return e;
    k_sweep_roots<<<dim3(std::min<unsigned>(blocks, 64u), (unsigned)S), threads, 0, st>>>(n, S, labels, d_roots);
    note_launch();
  }
  return cudaGetLastError();
}

}  // namespace pecann
