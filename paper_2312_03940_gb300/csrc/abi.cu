// The C ABI (include/pecann.h): argument checks, workspace layout, and the
// host loops that sequence the kernels.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace pecann {

cudaError_t run_cluster(int64_t n, const float* rho, const int32_t* lam, const float* delta, int center_fn,
                        float rho_min, float delta_min, int32_t n_clusters, const int32_t* knn_ids, int k,
                        const float* rank_key, int32_t* labels, void* ws, unsigned long long* d_roots,
                        cudaStream_t st);
size_t cluster_ws_bytes(int64_t n);
size_t sweep_ws_bytes(int64_t n, int S);
cudaError_t run_cluster_sweep(int64_t n, const float* rho, const int32_t* lam, const float* delta, int S,
                              const pecann_cluster_setting* h_set, const int32_t* knn_ids, int k,
                              const float* rank_key, int32_t* labels, void* ws, unsigned long long* d_roots,
                              cudaStream_t st);
size_t build_ws_bytes(int64_t n, const pecann_params& p, int64_t cap, int vcap);
int64_t batch_cap_of(int64_t n, float frac);
cudaError_t run_build(const DataView& dv, const pecann_params& p, const int32_t* d_order, int32_t* G,
                      int32_t* d_degree, void* ws, int* d_err, int log2h, cudaStream_t st);

__global__ void k_dep_round0(int64_t n, int k, const int32_t* knn_ids, const float* knn_dist, const float* rk,
                             int32_t* lam, float* delta);
__global__ void k_rank_max(int64_t n, const float* rk, unsigned long long* out);
__global__ void k_compact_unfinished(const int32_t* src, int64_t m, const int32_t* lam,
                                     const unsigned long long* gmax, int32_t* dst, int32_t* cnt);
__global__ void k_normalize_density(int64_t n, int k, const int32_t* knn_ids, const float* raw, float* rho,
                                    float* rk);

static thread_local std::string g_last_error;
static thread_local const char* g_where = "";

void set_where(const char* w) { g_where = w; }
const char* get_where() { return g_where; }
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_last_error(const std::string& s) { g_last_error = s; }

int num_sms() {
  static int cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cache[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = v > 0 ? v : 1;
  }
  return cache[dev];
}

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// Header of every workspace: an error word and small counters.
struct WsHeader {
  int err;
  int pad0;
  int32_t counts[14];
  unsigned long long gmax;
  unsigned long long roots;
  unsigned long long work[3];  // byte offset 80: expansions, distance evaluations, beam insertions
};
static const size_t HDR = 256;

static int elem_bytes(int dtype) { return dtype == DT_F32 ? 4 : (dtype == DT_BF16 ? 2 : 1); }

static bool is_reduced(int dtype) { return dtype == DT_BF16 || dtype == DT_FP8; }

// Checks the dataset and fills the view of its rows; f32 (optional) gets the
// FP32 rows: the same view for FP32 / U8 data, data_f32 for BF16 / FP8.
pecann_status check_dataset(const pecann_dataset* ds, DataView* dv, DataView* f32) {
  if (!ds || !ds->data) return set_last_error("dataset or data pointer is NULL"), PECANN_EINVAL;
  if (ds->n < 2 || ds->n >= ((int64_t)1 << 31)) return set_last_error("n out of range"), PECANN_EINVAL;
  if (ds->dtype < 0 || ds->dtype > 3 || ds->metric < 0 || ds->metric > 1)
    return set_last_error("bad dtype or metric"), PECANN_EINVAL;
  int epc = 16 / elem_bytes(ds->dtype);
  if (ds->d <= 0 || ds->d % epc) return set_last_error("d must be a positive multiple of 16 bytes / element size"), PECANN_EINVAL;
  if (((uintptr_t)ds->data) & 15) return set_last_error("rows must be 16-byte aligned"), PECANN_EINVAL;
  if (is_reduced(ds->dtype) && (!ds->data_f32 || (((uintptr_t)ds->data_f32) & 15)))
    return set_last_error("BF16 / FP8 data needs 16-byte aligned FP32 rows in data_f32"), PECANN_EINVAL;
  if (ds->dtype == DT_FP8) {
    if (!ds->dim_scale || (((uintptr_t)ds->dim_scale) & 15))
      return set_last_error("FP8 data needs a 16-byte aligned dim_scale array of d floats"), PECANN_EINVAL;
    if (ds->metric != MET_IP)
      return set_last_error("FP8 traversal supports the inner-product metric only"), PECANN_EUNSUPPORTED;
  }
  Layout L;
  if (!pick_layout(ds->dtype, ds->metric, ds->d, &L))
    return set_last_error("no kernel for this dtype / metric / d"), PECANN_EUNSUPPORTED;
  if (is_reduced(ds->dtype) && !pick_layout(DT_F32, ds->metric, ds->d, &L))
    return set_last_error("no FP32 re-rank kernel for this d"), PECANN_EUNSUPPORTED;
  dv->X = (const uint8_t*)ds->data;
  dv->n = ds->n;
  dv->d = ds->d;
  dv->dtype = ds->dtype;
  dv->metric = ds->metric;
  dv->row_bytes = (int64_t)ds->d * elem_bytes(ds->dtype);
  dv->C = (int)(dv->row_bytes / 16);
  dv->f32_rows = ds->dtype == DT_FP8 ? ds->data_f32 : nullptr;
  dv->scale = ds->dtype == DT_FP8 ? ds->dim_scale : nullptr;
  if (f32) {
    *f32 = *dv;
    if (is_reduced(ds->dtype)) {
      f32->X = (const uint8_t*)ds->data_f32;
      f32->dtype = DT_F32;
      f32->row_bytes = (int64_t)ds->d * 4;
      f32->C = (int)(f32->row_bytes / 16);
    }
  }
  return PECANN_OK;
}

static const int DEP_RERANK = 32;  // dependent rounds: candidates re-scored per query

int rerank_k_of(const pecann_params* p) {
  int K = p->rerank_k > 0 ? p->rerank_k : std::min(p->L_search, 4 * p->k);
  return std::max(K, p->k);
}

int log2_hash(const pecann_params* p, int Lw) {
  int slots = p->hash_slots;
  if (slots <= 0) {
    // 8 slots per beam entry: at a beam of 128 this keeps a warp's shared
    // memory near 6 KB (32 warps per SM); the filter forgets some ids, which
    // costs repeated distances but never changes a result
    slots = 8 * Lw;
    slots = std::max(512, std::min(slots, 16384));
  }
  int l = 0;
  while ((1 << l) < slots) l++;
  return std::max(4, std::min(l, 16));
}

pecann_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PECANN_OK;
  if (e == cudaErrorNotSupported) {
    set_last_error(std::string(what) + ": unsupported combination");
    return PECANN_EUNSUPPORTED;
  }
  set_last_error(std::string(what) + ": " + cudaGetErrorString(e) + (*g_where ? std::string(" (at ") + g_where + ")" : ""));
  g_where = "";
  return PECANN_ECUDA;
}

pecann_status read_err(int* d_err, cudaStream_t st) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "error readback");
  if (h == ERR_TIMEOUT) {
    set_last_error("a pipeline wait of the tensor-core screen ran past its limit");
    return PECANN_ETIMEOUT;
  }
  if (h) {
    set_last_error(h == ERR_BAD_ID ? "graph or query id out of range"
                                   : (h == ERR_NO_PROGRESS ? "search made no progress" : "capacity exceeded"));
    return PECANN_EINTERNAL;
  }
  return PECANN_OK;
}

pecann_status check_params(const pecann_params* p, int64_t n) {
  if (!p) return set_last_error("params is NULL"), PECANN_EINVAL;
  if (p->R < 1 || p->R > 256) return set_last_error("R must be in 1..256"), PECANN_EINVAL;
  if (p->k < 1 || p->k >= n || p->k > 1024) return set_last_error("k must be in 1..min(n-1, 1024)"), PECANN_EINVAL;
  if (p->L_search < p->k || p->L_search > 8192) return set_last_error("L_search must be in k..8192"), PECANN_EINVAL;
  if (p->hash_slots < 0 || (p->hash_slots & (p->hash_slots - 1)))
    return set_last_error("hash_slots must be 0 or a power of 2"), PECANN_EINVAL;
  return PECANN_OK;
}

// Workspace pieces of each call (bytes after the header).
static size_t density_bytes(int64_t n, int reduced_K) {
  size_t b = 2 * al((size_t)n * 4);
  if (reduced_K > 0) b += 2 * al((size_t)n * reduced_K * 4) + al((size_t)n * 4);
  return b;
}
static size_t dep_bytes(int64_t n, bool reduced) {
  size_t b = 2 * al((size_t)n * 4) + al((size_t)n * 8);
  if (reduced) b += al((size_t)n * DEP_RERANK * 4) + al((size_t)n * 4);
  return b;
}
// Brute-force index: the k-NN / dependent pieces above, then its own scratch.
static size_t bf_density_offset(int64_t n) { return 2 * al((size_t)n * 4); }
static size_t bf_dep_offset(int64_t n) { return 2 * al((size_t)n * 4) + al((size_t)n * 8); }

// The brute-force index reads BF16 copies of the rows through TMA (rows of
// d * 2 bytes, a multiple of 16) and keeps 80 candidates per query.
pecann_status check_index(const DataView& dv, const pecann_params* p) {
  if (p->index != PECANN_INDEX_GRAPH && p->index != PECANN_INDEX_BRUTE_FORCE)
    return set_last_error("index must be PECANN_INDEX_GRAPH or PECANN_INDEX_BRUTE_FORCE"), PECANN_EINVAL;
  if (p->index == PECANN_INDEX_BRUTE_FORCE) {
    if (dv.d % 8) return set_last_error("the brute-force index needs d to be a multiple of 8"), PECANN_EUNSUPPORTED;
    if (p->k > 63) return set_last_error("the brute-force index supports k <= 63"), PECANN_EUNSUPPORTED;
  }
  return PECANN_OK;
}

pecann_status check_density_args(const DataView& dv, const int32_t* d_graph, const pecann_params* p,
                                 const int32_t* d_knn_ids, const float* d_knn_dist, const float* d_density,
                                 const float* d_rank_key) {
  pecann_status s = check_params(p, dv.n);
  if (s) return s;
  if ((s = check_index(dv, p))) return s;
  if ((!d_graph && p->index == PECANN_INDEX_GRAPH) || !d_knn_ids || !d_knn_dist || !d_density || !d_rank_key)
    return set_last_error("NULL pointer"), PECANN_EINVAL;
  if (p->density < 0 || p->density > 3) return set_last_error("bad density function"), PECANN_EINVAL;
  if (is_reduced(dv.dtype) && rerank_k_of(p) > p->L_search)
    return set_last_error("rerank_k must be in k..L_search"), PECANN_EINVAL;
  return PECANN_OK;
}

// The optional normalisation (Sec. 4.2), then the error word.
static pecann_status finish_density(const DataView& dv, const pecann_params* p, const int32_t* d_knn_ids,
                                    float* d_density, float* d_rank_key, const DensityScratch& sc, cudaStream_t st) {
  pecann_status s;
  cudaError_t e;
  if (p->normalize_density) {
    if ((e = cudaMemcpyAsync(sc.raw, d_density, (size_t)dv.n * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return cuda_status(e, "copy");
    unsigned blocks = (unsigned)std::min<int64_t>((dv.n + 255) / 256, (int64_t)num_sms() * 8);
    k_normalize_density<<<blocks, 256, 0, st>>>(dv.n, p->k, d_knn_ids, sc.raw, d_density, d_rank_key); note_launch();
    if ((s = cuda_status(cudaGetLastError(), "normalize"))) return s;
  }
  return read_err(sc.err, st);
}

// k-NN + density (Algorithm 2 lines 2-4) on checked arguments: the beam
// search over every point, the FP32 re-rank for reduced-precision rows, the
// brute-force k-NN of the points whose search returned fewer than k, the
// optional normalisation; then the error word is read back, so that a kernel
// that met an out-of-range graph id makes the call return PECANN_EINTERNAL.
// *sc.err and *sc.fb_cnt must be zero on entry.
pecann_status run_density(const DataView& dv, const DataView& fv, const int32_t* d_graph, const pecann_params* p,
                          int32_t* d_knn_ids, float* d_knn_dist, float* d_density, float* d_rank_key,
                          const DensityScratch& sc, cudaStream_t st) {
  const bool reduced = is_reduced(dv.dtype);
  const int K = reduced ? rerank_k_of(p) : 0;
  pecann_status s;
  cudaError_t e;
  if (p->index == PECANN_INDEX_BRUTE_FORCE) {
    // exact k-NN by the tensor-core screen and the exact re-rank (Sec. 5.1,
    // brute force); points it leaves go through the SIMT brute force below
    if (!sc.bf_ws) return set_last_error("no scratch for the brute-force index"), PECANN_EUNSUPPORTED;
    if ((s = run_density_bf(fv, p, d_knn_ids, d_knn_dist, d_density, d_rank_key, sc.fb_list, sc.fb_cnt, sc.err,
                            sc.bf_ws, sc.bf_counts, st)))
      return s;
    e = launch_bruteforce_knn(fv, sc.fb_list, sc.fb_cnt, dv.n, p->k, d_knn_ids, d_knn_dist, d_density, d_rank_key,
                              p->density, sc.err, st);
    if ((s = cuda_status(e, "brute-force k-NN"))) return s;
    return finish_density(dv, p, d_knn_ids, d_density, d_rank_key, sc, st);
  }
  if (reduced && !sc.rr_ids) return set_last_error("no re-rank scratch for BF16 / FP8 rows"), PECANN_EUNSUPPORTED;
  SearchArgs a;
  memset(&a, 0, sizeof(a));
  a.X = dv.X;
  a.row_bytes = dv.row_bytes;
  a.n = dv.n;
  a.C = dv.C;
  a.G = d_graph;
  a.R = p->R;
  a.queries = nullptr;
  a.nq = dv.n;
  a.Lw = p->L_search;
  a.log2h = log2_hash(p, a.Lw);
  a.stage = (p->R + 31) & ~31;
  a.mode = MODE_KNN;
  a.metric = dv.metric;
  a.block_warps = p->block_warps;
  a.warp_bytes = search_warp_bytes(a.Lw, a.log2h, a.stage, 0, false);
  a.k = p->k;
  a.out_ids = d_knn_ids;
  a.out_dis = d_knn_dist;
  a.rho = d_density;
  a.rkey = d_rank_key;
  a.density_fn = p->density;
  a.fb_list = sc.fb_list;
  a.fb_cnt = sc.fb_cnt;
  a.err = sc.err;
  a.work = sc.work;
  if (reduced) {
    // walk the reduced rows, keep the K best candidates, re-rank them in FP32
    a.mode = MODE_RAW;
    a.k = K;
    a.out_ids = sc.rr_ids;
    a.out_dis = sc.rr_dis;
    a.out_cnt = sc.rr_cnt;
    if ((s = cuda_status(launch_search(dv, a, st), "k-NN search"))) return s;
    e = launch_rerank_knn(fv, nullptr, dv.n, sc.rr_ids, sc.rr_cnt, K, p->k, d_knn_ids, d_knn_dist, d_density, d_rank_key,
                          p->density, sc.fb_list, sc.fb_cnt, st);
    if ((s = cuda_status(e, "FP32 re-rank"))) return s;
  } else {
    if ((s = cuda_status(launch_search(dv, a, st), "k-NN search"))) return s;
  }
  // points whose search returned fewer than k: exact k-NN by brute force
  e = launch_bruteforce_knn(fv, sc.fb_list, sc.fb_cnt, dv.n, p->k, d_knn_ids, d_knn_dist, d_density, d_rank_key,
                            p->density, sc.err, st);
  if ((s = cuda_status(e, "brute-force k-NN"))) return s;
  return finish_density(dv, p, d_knn_ids, d_density, d_rank_key, sc, st);
}

// Brute-force index: the points that took the collect pass and those left
// to the exact SIMT kernels, as two int32 at byte offset 24 of the workspace.
static pecann_status write_bf_counts(WsHeader* h, const int64_t* c, cudaStream_t st) {
  const int32_t v[2] = {(int32_t)c[0], (int32_t)c[1]};
  cudaError_t e = cudaMemcpyAsync(&h->counts[4], v, 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_status(e, "counters");
}

}  // namespace pecann

using namespace pecann;

extern "C" {

void pecann_params_default(pecann_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->k = 16;
  p->R = 32;
  p->L_build = 64;
  p->L_search = 64;
  p->L_dep = 64;
  p->alpha = 1.1f;
  p->n_start = 16;
  p->batch_frac = 0.02f;
  p->visit_cap = 0;
  p->dep_threshold = 300;
  p->max_dep_rounds = 30;
  p->max_dep_beam = 8192;
  p->density = PECANN_DENS_KTH;
  p->normalize_density = 0;
  p->center = PECANN_CENTER_PRODUCT;
  p->rho_min = 0.0f;
  p->delta_min = 0.0f;
  p->n_clusters = 1;
  p->hash_slots = 0;
  p->collect_work = 0;
  p->build_passes = 1;
  p->rerank_k = 0;
  p->block_warps = 0;
  p->index = PECANN_INDEX_GRAPH;
  p->seed = 0;
}

const char* pecann_status_string(int s) {
  switch (s) {
    case PECANN_OK: return "ok";
    case PECANN_EINVAL: return "invalid argument";
    case PECANN_ENOMEM: return "workspace too small";
    case PECANN_ECUDA: return "CUDA error";
    case PECANN_ETIMEOUT: return "device wait timed out";
    case PECANN_EUNSUPPORTED: return "unsupported";
    case PECANN_EINTERNAL: return "kernel-detected inconsistency";
    default: return "unknown status";
  }
}

const char* pecann_last_error(void) { return g_last_error.c_str(); }

int32_t pecann_version(void) { return 100; }

int64_t pecann_kernel_launches(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

pecann_status pecann_workspace_size(const pecann_dataset* ds, const pecann_params* p, size_t* bytes) {
  if (!ds || !p || !bytes) return set_last_error("NULL argument"), PECANN_EINVAL;
  int64_t n = ds->n;
  if (n < 2) return set_last_error("n out of range"), PECANN_EINVAL;
  const bool red = is_reduced(ds->dtype);
  size_t b = density_bytes(n, red ? std::min(std::max(rerank_k_of(p), 1), 8192) : 0);
  b = std::max(b, dep_bytes(n, red));
  if (p->index == PECANN_INDEX_BRUTE_FORCE && ds->d > 0)
    b = std::max(b, std::max(bf_density_offset(n), bf_dep_offset(n)) + bf_ws_bytes(n, ds->d));
  b = std::max(b, cluster_ws_bytes(n));
  if (p->R >= 1 && p->L_build >= 1) {
    int vcap = p->visit_cap > 0 ? p->visit_cap : 2 * p->L_build;
    b = std::max(b, build_ws_bytes(n, *p, batch_cap_of(n, p->batch_frac > 0 ? p->batch_frac : 0.02f), vcap));
  }
  *bytes = HDR + b + 4096;
  return PECANN_OK;
}

pecann_status pecann_search(const pecann_dataset* ds, const int32_t* d_graph, int32_t R,
                            const int32_t* d_queries, int64_t m, const int32_t* d_start, int32_t n_start,
                            int32_t L, int32_t k, int32_t* d_ids, float* d_dis, int32_t* d_count,
                            const pecann_params* p, void* ws, size_t ws_bytes, void* stream) {
  DataView dv;
  pecann_status s = check_dataset(ds, &dv);
  if (s) return s;
  if (!d_graph || !d_ids || !d_dis || !d_count || !ws) return set_last_error("NULL pointer"), PECANN_EINVAL;
  if (R < 1 || R > 256 || L < 1 || L > 8192 || k < 1 || k > L || m < 0)
    return set_last_error("R, L, k or m out of range"), PECANN_EINVAL;
  if (d_start && (n_start < 1 || n_start > 65536)) return set_last_error("n_start out of range"), PECANN_EINVAL;
  if (ws_bytes < HDR) return set_last_error("workspace too small"), PECANN_ENOMEM;
  pecann_params dp;
  pecann_params_default(&dp);
  if (!p) p = &dp;
  cudaStream_t st = (cudaStream_t)stream;
  WsHeader* h = (WsHeader*)ws;
  cudaError_t e = cudaMemsetAsync(h, 0, HDR, st);
  if (e != cudaSuccess) return cuda_status(e, "memset");
  SearchArgs a;
  memset(&a, 0, sizeof(a));
  a.X = dv.X;
  a.row_bytes = dv.row_bytes;
  a.n = dv.n;
  a.C = dv.C;
  a.G = d_graph;
  a.R = R;
  a.queries = d_queries;
  a.nq = m;
  a.S = d_start;
  a.nS = d_start ? n_start : 0;
  a.Lw = L;
  a.log2h = log2_hash(p, L);
  a.stage = (std::max(R, 64) + 31) & ~31;
  a.mode = MODE_RAW;
  a.metric = dv.metric;
  a.block_warps = p->block_warps;
  a.warp_bytes = search_warp_bytes(a.Lw, a.log2h, a.stage, 0, false);
  a.k = k;
  a.out_ids = d_ids;
  a.out_dis = d_dis;
  a.out_cnt = d_count;
  a.err = &h->err;
  a.work = p->collect_work ? h->work : nullptr;
  if ((s = cuda_status(launch_search(dv, a, st), "search"))) return s;
  return read_err(&h->err, st);
}

pecann_status pecann_build_graph(const pecann_dataset* ds, const pecann_params* p, const int32_t* d_order,
                                 int32_t* d_graph, int32_t* d_degree, void* ws, size_t ws_bytes, void* stream) {
  DataView dv0, dv;
  pecann_status s = check_dataset(ds, &dv0, &dv);  // the build always uses the FP32 (or U8) rows
  if (s) return s;
  if (!p || !d_graph || !ws) return set_last_error("NULL pointer"), PECANN_EINVAL;
  if (p->R < 1 || p->R > 256) return set_last_error("R must be in 1..256"), PECANN_EINVAL;
  if (p->L_build < 1 || p->L_build > 1024) return set_last_error("L_build must be in 1..1024"), PECANN_EINVAL;
  if (!(p->alpha >= 1.0f)) return set_last_error("alpha must be >= 1"), PECANN_EINVAL;
  if (p->n_start < 1 || p->n_start > dv.n || p->n_start > 65536)
    return set_last_error("n_start must be in 1..min(n, 65536)"), PECANN_EINVAL;
  if (!(p->batch_frac > 0.0f) || p->batch_frac > 1.0f) return set_last_error("batch_frac must be in (0, 1]"), PECANN_EINVAL;
  if (p->build_passes != 1 && p->build_passes != 2) return set_last_error("build_passes must be 1 or 2"), PECANN_EINVAL;
  int vcap = p->visit_cap > 0 ? p->visit_cap : 2 * p->L_build;
  if (vcap + p->R > 4096) return set_last_error("visit_cap + R must be <= 4096"), PECANN_EINVAL;
  if (p->hash_slots < 0 || (p->hash_slots & (p->hash_slots - 1)))
    return set_last_error("hash_slots must be 0 or a power of 2"), PECANN_EINVAL;
  size_t need = HDR + build_ws_bytes(dv.n, *p, batch_cap_of(dv.n, p->batch_frac), vcap);
  if (ws_bytes < need) return set_last_error("workspace too small"), PECANN_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  WsHeader* h = (WsHeader*)ws;
  cudaError_t e = cudaMemsetAsync(h, 0, HDR, st);
  if (e != cudaSuccess) return cuda_status(e, "memset");
  e = run_build(dv, *p, d_order, d_graph, d_degree, (uint8_t*)ws + HDR, &h->err, log2_hash(p, p->L_build), st);
  if ((s = cuda_status(e, "build"))) return s;
  return read_err(&h->err, st);
}

static pecann_status check_nndescent(const DataView& dv, const pecann_params* p, int32_t K, int32_t repeats,
                                     int32_t rounds) {
  if (K < 1 || K > 64 || K >= dv.n) return set_last_error("K must be in 1..min(64, n - 1)"), PECANN_EINVAL;
  if (repeats < 1 || repeats > 64) return set_last_error("repeats must be in 1..64"), PECANN_EINVAL;
  if (rounds < 0 || rounds > 1000) return set_last_error("rounds must be in 0..1000"), PECANN_EINVAL;
  if (p->R < 1 || p->R > 256) return set_last_error("R must be in 1..256"), PECANN_EINVAL;
  if (!(p->alpha >= 1.0f)) return set_last_error("alpha must be >= 1"), PECANN_EINVAL;
  return PECANN_OK;
}

pecann_status pecann_nndescent_workspace_size(const pecann_dataset* ds, const pecann_params* p, int32_t K,
                                              int32_t repeats, size_t* bytes) {
  DataView dv0, dv;
  pecann_status s = check_dataset(ds, &dv0, &dv);
  if (s) return s;
  if (!p || !bytes) return set_last_error("NULL argument"), PECANN_EINVAL;
  if ((s = check_nndescent(dv, p, K, repeats, 0))) return s;
  *bytes = HDR + nndescent_ws_bytes(dv.n, K, repeats, p->R);
  return PECANN_OK;
}

pecann_status pecann_build_nndescent(const pecann_dataset* ds, const pecann_params* p, int32_t K, int32_t repeats,
                                     const int32_t* d_init, int32_t rounds, int32_t* d_graph, int32_t* d_degree,
                                     int32_t* d_knn, int64_t* h_changes, void* ws, size_t ws_bytes, void* stream) {
  DataView dv0, dv;
  pecann_status s = check_dataset(ds, &dv0, &dv);  // FP32 (or U8) rows, like the Vamana build
  if (s) return s;
  if (!p || !d_init || !d_graph || !ws) return set_last_error("NULL pointer"), PECANN_EINVAL;
  if ((s = check_nndescent(dv, p, K, repeats, rounds))) return s;
  if (ws_bytes < HDR + nndescent_ws_bytes(dv.n, K, repeats, p->R))
    return set_last_error("workspace too small"), PECANN_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  WsHeader* h = (WsHeader*)ws;
  cudaError_t e = cudaMemsetAsync(h, 0, HDR, st);
  if (e != cudaSuccess) return cuda_status(e, "memset");
  if (h_changes)
    for (int64_t i = 0; i < (int64_t)repeats * rounds; i++) h_changes[i] = 0;
  e = run_nndescent(dv, K, repeats, d_init, rounds, p->alpha, p->R, d_graph, d_knn, h_changes, (uint8_t*)ws + HDR,
                    &h->err, st);
  if ((s = cuda_status(e, "nn-descent"))) return s;
  if (d_degree) {
    k_degree<<<(unsigned)std::min<int64_t>((dv.n + 255) / 256, (int64_t)num_sms() * 8), 256, 0, st>>>(
        dv.n, p->R, d_graph, d_degree);
    note_launch();
    if ((s = cuda_status(cudaGetLastError(), "degree"))) return s;
  }
  return read_err(&h->err, st);
}

static pecann_status check_hcnng(const DataView& dv, const pecann_params* p, int32_t repeats, int32_t leaf_size,
                                 int32_t mst_deg) {
  if (repeats < 1 || repeats > 64) return set_last_error("repeats must be in 1..64"), PECANN_EINVAL;
  if (leaf_size < 2 || leaf_size > HCNNG_MAX_LEAF)
    return set_last_error("leaf_size must be in 2..200"), PECANN_EINVAL;
  if (mst_deg < 1 || mst_deg > HCNNG_MAX_DEG) return set_last_error("mst_deg must be in 1..16"), PECANN_EINVAL;
  if (p->R < 1 || p->R > 256) return set_last_error("R must be in 1..256"), PECANN_EINVAL;
  if (!(p->alpha >= 1.0f)) return set_last_error("alpha must be >= 1"), PECANN_EINVAL;
  (void)dv;
  return PECANN_OK;
}

pecann_status pecann_hcnng_workspace_size(const pecann_dataset* ds, const pecann_params* p, int32_t repeats,
                                          int32_t leaf_size, int32_t mst_deg, size_t* bytes) {
  DataView dv0, dv;
  pecann_status s = check_dataset(ds, &dv0, &dv);
  if (s) return s;
  if (!p || !bytes) return set_last_error("NULL argument"), PECANN_EINVAL;
  if ((s = check_hcnng(dv, p, repeats, leaf_size, mst_deg))) return s;
  *bytes = HDR + hcnng_ws_bytes(dv.n, repeats, leaf_size, mst_deg);
  return PECANN_OK;
}

pecann_status pecann_build_hcnng(const pecann_dataset* ds, const pecann_params* p, int32_t repeats,
                                 int32_t leaf_size, int32_t mst_deg, int32_t* d_graph, int32_t* d_degree,
                                 int64_t* h_leaves, void* ws, size_t ws_bytes, void* stream) {
  DataView dv0, dv;
  pecann_status s = check_dataset(ds, &dv0, &dv);  // FP32 (or U8) rows, like the other builds
  if (s) return s;
  if (!p || !d_graph || !ws) return set_last_error("NULL pointer"), PECANN_EINVAL;
  if ((s = check_hcnng(dv, p, repeats, leaf_size, mst_deg))) return s;
  if (ws_bytes < HDR + hcnng_ws_bytes(dv.n, repeats, leaf_size, mst_deg))
    return set_last_error("workspace too small"), PECANN_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  WsHeader* h = (WsHeader*)ws;
  cudaError_t e = cudaMemsetAsync(h, 0, HDR, st);
  if (e != cudaSuccess) return cuda_status(e, "memset");
  e = run_hcnng(dv, repeats, leaf_size, mst_deg, p->alpha, p->R, p->seed, d_graph, h_leaves, (uint8_t*)ws + HDR,
                &h->err, st);
  if ((s = cuda_status(e, "hcnng"))) return s;
  if (d_degree) {
    k_degree<<<(unsigned)std::min<int64_t>((dv.n + 255) / 256, (int64_t)num_sms() * 8), 256, 0, st>>>(
        dv.n, p->R, d_graph, d_degree);
    note_launch();
    if ((s = cuda_status(cudaGetLastError(), "degree"))) return s;
  }
  return read_err(&h->err, st);
}

pecann_status pecann_density(const pecann_dataset* ds, const int32_t* d_graph, const pecann_params* p,
                             int32_t* d_knn_ids, float* d_knn_dist, float* d_density, float* d_rank_key,
                             void* ws, size_t ws_bytes, void* stream) {
  DataView dv, fv;
  pecann_status s = check_dataset(ds, &dv, &fv);
  if (s) return s;
  if ((s = check_density_args(dv, d_graph, p, d_knn_ids, d_knn_dist, d_density, d_rank_key))) return s;
  if (!ws) return set_last_error("NULL pointer"), PECANN_EINVAL;
  const bool reduced = is_reduced(dv.dtype);
  const bool bf = p->index == PECANN_INDEX_BRUTE_FORCE;
  const int K = reduced && !bf ? rerank_k_of(p) : 0;
  const size_t need = bf ? bf_density_offset(dv.n) + bf_ws_bytes(dv.n, dv.d) : density_bytes(dv.n, K);
  if (ws_bytes < HDR + need) return set_last_error("workspace too small"), PECANN_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  WsHeader* h = (WsHeader*)ws;
  uint8_t* w = (uint8_t*)ws + HDR;
  DensityScratch sc;
  int64_t bf_counts[2] = {0, 0};
  if (bf) {
    sc.bf_ws = w + bf_density_offset(dv.n);
    sc.bf_counts = bf_counts;
  }
  sc.fb_list = (int32_t*)w;
  sc.raw = (float*)(w + al((size_t)dv.n * 4));
  sc.fb_cnt = &h->counts[0];
  sc.err = &h->err;
  sc.work = p->collect_work ? h->work : nullptr;
  if (reduced && !bf) {
    sc.rr_ids = (int32_t*)(w + 2 * al((size_t)dv.n * 4));
    sc.rr_dis = (float*)((uint8_t*)sc.rr_ids + al((size_t)dv.n * K * 4));
    sc.rr_cnt = (int32_t*)((uint8_t*)sc.rr_dis + al((size_t)dv.n * K * 4));
  }
  cudaError_t e = cudaMemsetAsync(h, 0, HDR, st);
  if (e != cudaSuccess) return cuda_status(e, "memset");
  if ((s = run_density(dv, fv, d_graph, p, d_knn_ids, d_knn_dist, d_density, d_rank_key, sc, st))) return s;
  if (bf) return write_bf_counts(h, bf_counts, st);
  return PECANN_OK;
}

pecann_status pecann_dependent_points(const pecann_dataset* ds, const int32_t* d_graph, const pecann_params* p,
                                      const float* d_rank_key, const int32_t* d_knn_ids, const float* d_knn_dist,
                                      int32_t* d_dep, float* d_dep_dist, int64_t* h_stats, void* ws,
                                      size_t ws_bytes, void* stream) {
  DataView dv, fv;
  pecann_status s = check_dataset(ds, &dv, &fv);
  if (s) return s;
  if ((s = check_params(p, dv.n))) return s;
  if (!d_rank_key || !d_knn_ids || !d_knn_dist || !d_dep || !d_dep_dist || !ws)
    return set_last_error("NULL pointer"), PECANN_EINVAL;
  const bool reduced = is_reduced(dv.dtype);
  if (p->L_dep < 1 || p->max_dep_beam < 1 || p->max_dep_beam > 8192 || p->dep_threshold < 0 ||
      p->max_dep_rounds < 0)
    return set_last_error("L_dep, max_dep_beam (<= 8192), dep_threshold or max_dep_rounds out of range"),
           PECANN_EINVAL;
  if ((s = check_index(dv, p))) return s;
  const bool bf = p->index == PECANN_INDEX_BRUTE_FORCE;
  if (!d_graph && !bf) return set_last_error("NULL pointer"), PECANN_EINVAL;
  if (ws_bytes < HDR + (bf ? bf_dep_offset(dv.n) + bf_ws_bytes(dv.n, dv.d) : dep_bytes(dv.n, reduced)))
    return set_last_error("workspace too small"), PECANN_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  WsHeader* h = (WsHeader*)ws;
  uint8_t* w = (uint8_t*)ws + HDR;
  int32_t* U0 = (int32_t*)w;
  int32_t* U1 = (int32_t*)(w + al((size_t)dv.n * 4));
  unsigned long long* best = (unsigned long long*)(w + 2 * al((size_t)dv.n * 4));
  int32_t* rr_ids = (int32_t*)((uint8_t*)best + al((size_t)dv.n * 8));
  int32_t* rr_cnt = (int32_t*)((uint8_t*)rr_ids + al((size_t)dv.n * DEP_RERANK * 4));
  int64_t stats[64];
  memset(stats, 0, sizeof(stats));
  cudaError_t e = cudaMemsetAsync(h, 0, HDR, st);
  if (e != cudaSuccess) return cuda_status(e, "memset");
  const unsigned blocks = (unsigned)std::min<int64_t>((dv.n + 255) / 256, (int64_t)num_sms() * 8);
  // the maximum-rank point has no dependent point
  k_rank_max<<<blocks, 256, 0, st>>>(dv.n, d_rank_key, &h->gmax); note_launch();
  // round 0: lambda_i <- DPBruteForce(x_i, N_i)
  k_dep_round0<<<blocks, 256, 0, st>>>(dv.n, p->k, d_knn_ids, d_knn_dist, d_rank_key, d_dep, d_dep_dist); note_launch();
  // P_unfinished, the maximum skipped
  k_compact_unfinished<<<blocks, 256, 0, st>>>(nullptr, dv.n, d_dep, &h->gmax, U0, &h->counts[1]); note_launch();
  if ((s = cuda_status(cudaGetLastError(), "round 0"))) return s;
  int32_t nu = 0;
  if ((e = cudaMemcpyAsync(&nu, &h->counts[1], 4, cudaMemcpyDeviceToHost, st)) == cudaSuccess)
    e = cudaStreamSynchronize(st);
  if ((s = cuda_status(e, "readback"))) return s;
  stats[1] = nu;
  if (bf) {
    // with the brute-force index FindKnn is exact, so a doubling round finds
    // a point's dependent point exactly when DPBruteForce over all of P
    // would: every unfinished point goes straight to the exact search
    int64_t c[2] = {0, 0};
    if ((s = run_dep_bf(fv, d_rank_key, U0, nu, d_dep, d_dep_dist, &h->err, w + bf_dep_offset(dv.n), c, st)))
      return s;
    if ((s = read_err(&h->err, st))) return s;
    stats[60] = c[0];
    stats[61] = c[1];
    stats[63] = nu;
    if ((s = write_bf_counts(h, c, st))) return s;
    if (h_stats) memcpy(h_stats, stats, sizeof(stats));
    return PECANN_OK;
  }
  int64_t kdep = p->L_dep;
  int rounds = 0;
  while (nu > p->dep_threshold && rounds < p->max_dep_rounds && kdep <= p->max_dep_beam) {
    SearchArgs a;
    memset(&a, 0, sizeof(a));
    a.X = dv.X;
    a.row_bytes = dv.row_bytes;
    a.n = dv.n;
    a.C = dv.C;
    a.G = d_graph;
    a.R = p->R;
    a.queries = U0;
    a.nq = nu;
    a.Lw = (int)kdep;
    a.log2h = log2_hash(p, a.Lw);
    a.stage = (p->R + 31) & ~31;
    a.mode = MODE_DEP;
    a.metric = dv.metric;
    a.block_warps = p->block_warps;
  a.warp_bytes = search_warp_bytes(a.Lw, a.log2h, a.stage, 0, false);
    a.rank_key = d_rank_key;
    a.lam = d_dep;
    a.delta = d_dep_dist;
    a.err = &h->err;
    if (reduced) {
      a.mode = MODE_DEPCAND;
      a.k = DEP_RERANK;
      a.out_ids = rr_ids;
      a.out_cnt = rr_cnt;
    }
    // N_candidates <- FindKnn(i, k_dep); lambda_i <- DPBruteForce(x_i, N_candidates)
    if ((s = cuda_status(launch_search(dv, a, st), "dependent search"))) return s;
    if (reduced) {
      e = launch_rerank_dep(fv, U0, nu, rr_ids, rr_cnt, DEP_RERANK, d_dep, d_dep_dist, st);
      if ((s = cuda_status(e, "FP32 re-rank"))) return s;
    }
    if ((e = cudaMemsetAsync(&h->counts[2], 0, 4, st)) != cudaSuccess) return cuda_status(e, "memset");
    unsigned ub = (unsigned)std::min<int64_t>((nu + 255) / 256, (int64_t)num_sms() * 8);
    k_compact_unfinished<<<ub, 256, 0, st>>>(U0, nu, d_dep, &h->gmax, U1, &h->counts[2]); note_launch();
    if ((s = cuda_status(cudaGetLastError(), "compact"))) return s;
    if ((e = cudaMemcpyAsync(&nu, &h->counts[2], 4, cudaMemcpyDeviceToHost, st)) == cudaSuccess)
      e = cudaStreamSynchronize(st);
    if ((s = cuda_status(e, "readback"))) return s;
    std::swap(U0, U1);
    kdep *= 2;
    if (rounds < 60) stats[2 + rounds] = nu;
    rounds++;
  }
  stats[0] = rounds;
  stats[63] = nu;
  // the rest: DPBruteForce over all of P
  e = launch_dep_bruteforce(fv, U0, nu, d_rank_key, best, d_dep, d_dep_dist, st);
  if ((s = cuda_status(e, "brute-force tail"))) return s;
  if ((s = read_err(&h->err, st))) return s;
  if (h_stats) memcpy(h_stats, stats, sizeof(stats));
  return PECANN_OK;
}

pecann_status pecann_cluster(int64_t n, const float* d_density, const int32_t* d_dep, const float* d_dep_dist,
                             const pecann_params* p, int32_t* d_labels, int64_t* h_n_clusters, void* ws,
                             size_t ws_bytes, void* stream) {
  if (!p || !d_density || !d_dep || !d_dep_dist || !d_labels || !ws)
    return set_last_error("NULL pointer"), PECANN_EINVAL;
  if (n < 1 || n >= ((int64_t)1 << 31)) return set_last_error("n out of range"), PECANN_EINVAL;
  if (p->center == PECANN_CENTER_LOCAL)
    return set_last_error("the local center needs the k-NN lists: use pecann_cluster_sweep"), PECANN_EINVAL;
  if (p->center != PECANN_CENTER_THRESHOLD && p->center != PECANN_CENTER_PRODUCT)
    return set_last_error("bad center function"), PECANN_EINVAL;
  if (p->center == PECANN_CENTER_PRODUCT && p->n_clusters < 1)
    return set_last_error("n_clusters must be >= 1"), PECANN_EINVAL;
  if (ws_bytes < HDR + cluster_ws_bytes(n)) return set_last_error("workspace too small"), PECANN_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  WsHeader* h = (WsHeader*)ws;
  cudaError_t e = run_cluster(n, d_density, d_dep, d_dep_dist, p->center, p->rho_min, p->delta_min, p->n_clusters,
                              nullptr, 0, nullptr, d_labels, (uint8_t*)ws + HDR,
                              h_n_clusters ? &h->roots : nullptr, st);
  pecann_status s = cuda_status(e, "cluster");
  if (s) return s;
  if (h_n_clusters) {
    unsigned long long r = 0;
    e = cudaMemcpyAsync(&r, &h->roots, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if ((s = cuda_status(e, "readback"))) return s;
    *h_n_clusters = (int64_t)r;
  }
  return PECANN_OK;
}

static size_t sweep_counts_offset(int64_t n, int32_t n_settings) {
  return (HDR + sweep_ws_bytes(n, n_settings) + 255) & ~(size_t)255;
}

pecann_status pecann_cluster_workspace_size(int64_t n, int32_t n_settings, size_t* bytes) {
  if (!bytes) return set_last_error("NULL argument"), PECANN_EINVAL;
  if (n < 1 || n >= ((int64_t)1 << 31)) return set_last_error("n out of range"), PECANN_EINVAL;
  if (n_settings < 1 || n_settings > 4096) return set_last_error("n_settings must be in 1..4096"), PECANN_EINVAL;
  // (also enough for pecann_cluster, the single-setting call)
  *bytes = std::max(sweep_counts_offset(n, n_settings) + (size_t)n_settings * 8, HDR + cluster_ws_bytes(n));
  return PECANN_OK;
}

pecann_status pecann_cluster_sweep(int64_t n, const float* d_density, const int32_t* d_dep, const float* d_dep_dist,
                                   const int32_t* d_knn_ids, int32_t k, const float* d_rank_key, int32_t n_settings,
                                   const pecann_cluster_setting* h_settings, int32_t* d_labels,
                                   int64_t* h_n_clusters, void* ws, size_t ws_bytes, void* stream) {
  size_t need = 0;
  pecann_status s = pecann_cluster_workspace_size(n, n_settings, &need);
  if (s) return s;
  if (!d_density || !d_dep || !d_dep_dist || !h_settings || !d_labels || !ws)
    return set_last_error("NULL pointer"), PECANN_EINVAL;
  for (int32_t i = 0; i < n_settings; i++) {
    const pecann_cluster_setting& c = h_settings[i];
    if (c.center != PECANN_CENTER_THRESHOLD && c.center != PECANN_CENTER_PRODUCT && c.center != PECANN_CENTER_LOCAL)
      return set_last_error("setting " + std::to_string(i) + ": bad center function"), PECANN_EINVAL;
    if (c.center == PECANN_CENTER_PRODUCT && c.n_clusters < 1)
      return set_last_error("setting " + std::to_string(i) + ": n_clusters must be >= 1"), PECANN_EINVAL;
    if (c.center == PECANN_CENTER_LOCAL && (!d_knn_ids || !d_rank_key || k < 1))
      return set_last_error("setting " + std::to_string(i) + ": the local center needs d_knn_ids, k >= 1 and "
                            "d_rank_key"), PECANN_EINVAL;
  }
  if (ws_bytes < need) return set_last_error("workspace too small"), PECANN_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* counts = (unsigned long long*)((uint8_t*)ws + sweep_counts_offset(n, n_settings));
  // every setting in the same passes: shared select passes, one parent
  // launch and shared pointer-jumping sweeps
  cudaError_t e = run_cluster_sweep(n, d_density, d_dep, d_dep_dist, n_settings, h_settings, d_knn_ids, k,
                                    d_rank_key, d_labels, (uint8_t*)ws + HDR, h_n_clusters ? counts : nullptr, st);
  if ((s = cuda_status(e, "cluster sweep"))) return s;
  if (h_n_clusters) {
    std::vector<unsigned long long> r((size_t)n_settings);
    e = cudaMemcpyAsync(r.data(), counts, (size_t)n_settings * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if ((s = cuda_status(e, "readback"))) return s;
    for (int32_t i = 0; i < n_settings; i++) h_n_clusters[i] = (int64_t)r[i];
  }
  return PECANN_OK;
}

}  // extern "C"
