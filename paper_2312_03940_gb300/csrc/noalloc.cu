// pecann_density_noalloc: the k-NN + density entry point for callers that
// cannot allocate GPU memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- inside a
// host callback or a real-time loop that must not take the allocator's lock,
// under an external memory manager that owns every device byte, or in a
// process whose allocations are frozen after start-up. Such a caller can hand
// over its inputs and outputs but cannot provide the workspace that
// pecann_density needs. This entry point keeps that scratch in a fixed,
// file-scope device array instead: it is created when the library is loaded
// on a device and stays there until the process exits, so the call itself
// allocates nothing.
//
// The array is shared by every call in the process: calls that overlap on the
// GPU (different streams, or different host threads) race on it and must be
// serialised by the caller. Each call clears the parts that have to start at
// zero; the rest keeps whatever the previous call left.
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace pecann {

__global__ void k_normalize_density(int64_t n, int k, const int32_t* knn_ids, const float* raw, float* rho,
                                    float* rk);

// Layout of the fixed scratch: a 256-byte header (error word, fallback
// counter) followed by the fallback list and the raw-density copy of up to
// PECANN_NOALLOC_MAX_POINTS points each.
static const size_t NOALLOC_HDR = 256;
static const size_t NOALLOC_LIST = (size_t)PECANN_NOALLOC_MAX_POINTS * 4;
static const size_t NOALLOC_BYTES = NOALLOC_HDR + 2 * NOALLOC_LIST;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of g_noalloc_scratch, looked up once per device. In host
// code the symbol itself is only a host-side handle, never a device address.
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};

static cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

static int elem_size(int dtype) { return dtype == DT_F32 ? 4 : (dtype == DT_BF16 ? 2 : 1); }

}  // namespace pecann

using namespace pecann;

extern "C" pecann_status pecann_density_noalloc(const pecann_dataset* ds, const int32_t* d_graph,
                                                const pecann_params* p, int32_t* d_knn_ids, float* d_knn_dist,
                                                float* d_density, float* d_rank_key, void* stream) {
  if (!ds || !p || !ds->data || !d_graph || !d_knn_ids || !d_knn_dist || !d_density || !d_rank_key) {
    set_last_error("pecann_density_noalloc: NULL argument");
    return PECANN_EINVAL;
  }
  if (ds->n > PECANN_NOALLOC_MAX_POINTS) {
    set_last_error("pecann_density_noalloc: n exceeds PECANN_NOALLOC_MAX_POINTS (1048576); "
                   "use pecann_density with a workspace");
    return PECANN_EINVAL;
  }
  if (ds->n < 2 || ds->dtype < 0 || ds->dtype > 3 || ds->metric < 0 || ds->metric > 1) {
    set_last_error("pecann_density_noalloc: n, dtype or metric out of range");
    return PECANN_EINVAL;
  }
  if (ds->d <= 0 || ds->d % (16 / elem_size(ds->dtype)) || (((uintptr_t)ds->data) & 15)) {
    set_last_error("pecann_density_noalloc: d must fill whole 16-byte chunks and rows must be 16-byte aligned");
    return PECANN_EINVAL;
  }
  if (ds->dtype == DT_BF16 || ds->dtype == DT_FP8) {
    set_last_error("pecann_density_noalloc: BF16 / FP8 traversal needs pecann_density (its re-rank scratch)");
    return PECANN_EUNSUPPORTED;
  }
  Layout L;
  if (!pick_layout(ds->dtype, ds->metric, ds->d, &L)) {
    set_last_error("pecann_density_noalloc: no kernel for this dtype / metric / d");
    return PECANN_EUNSUPPORTED;
  }
  if (p->R < 1 || p->R > 256 || p->k < 1 || p->k >= ds->n || p->k > 1024 || p->L_search < p->k ||
      p->L_search > 8192 || p->density < 0 || p->density > 3 || p->hash_slots < 0 ||
      (p->hash_slots & (p->hash_slots - 1))) {
    set_last_error("pecann_density_noalloc: R, k, L_search, density or hash_slots out of range");
    return PECANN_EINVAL;
  }
  void* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) {
    set_last_error(std::string("pecann_density_noalloc: scratch lookup: ") + cudaGetErrorString(e));
    return PECANN_ECUDA;
  }
  DataView dv;
  dv.X = (const uint8_t*)ds->data;
  dv.n = ds->n;
  dv.d = ds->d;
  dv.dtype = ds->dtype;
  dv.metric = ds->metric;
  dv.row_bytes = (int64_t)ds->d * elem_size(ds->dtype);
  dv.C = (int)(dv.row_bytes / 16);
  cudaStream_t st = (cudaStream_t)stream;
  uint8_t* base = (uint8_t*)scratch;
  int* err = (int*)base;
  int32_t* fb_cnt = (int32_t*)(base + 8);
  int32_t* fb_list = (int32_t*)(base + NOALLOC_HDR);
  float* raw = (float*)(base + NOALLOC_HDR + NOALLOC_LIST);
  // the error word and the fallback counter must start at zero
  if ((e = cudaMemsetAsync(base, 0, NOALLOC_HDR, st)) != cudaSuccess) {
    set_last_error(std::string("pecann_density_noalloc: memset: ") + cudaGetErrorString(e));
    return PECANN_ECUDA;
  }
  int slots = p->hash_slots > 0 ? p->hash_slots : std::max(512, std::min(8 * p->L_search, 16384));
  int log2h = 0;
  while ((1 << log2h) < slots) log2h++;
  log2h = std::max(4, std::min(log2h, 16));
  SearchArgs a;
  memset(&a, 0, sizeof(a));
  a.X = dv.X;
  a.row_bytes = dv.row_bytes;
  a.n = dv.n;
  a.C = dv.C;
  a.G = d_graph;
  a.R = p->R;
  a.nq = dv.n;
  a.Lw = p->L_search;
  a.log2h = log2h;
  a.stage = (std::max(p->R, 64) + 31) & ~31;
  a.mode = MODE_KNN;
  a.metric = dv.metric;
  a.warp_bytes = search_warp_bytes(a.Lw, a.log2h, a.stage, 0, false);
  a.k = p->k;
  a.out_ids = d_knn_ids;
  a.out_dis = d_knn_dist;
  a.rho = d_density;
  a.rkey = d_rank_key;
  a.density_fn = p->density;
  a.fb_list = fb_list;
  a.fb_cnt = fb_cnt;
  a.err = err;
  if ((e = launch_search(dv, a, st)) == cudaSuccess)
    e = launch_bruteforce_knn(dv, fb_list, fb_cnt, dv.n, p->k, d_knn_ids, d_knn_dist, d_density, d_rank_key,
                              p->density, err, st);
  if (e == cudaSuccess && p->normalize_density) {
    e = cudaMemcpyAsync(raw, d_density, (size_t)dv.n * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
      unsigned blocks = (unsigned)std::min<int64_t>((dv.n + 255) / 256, (int64_t)num_sms() * 8);
      k_normalize_density<<<blocks, 256, 0, st>>>(dv.n, p->k, d_knn_ids, raw, d_density, d_rank_key);
      note_launch();
      e = cudaGetLastError();
    }
  }
  if (e == cudaErrorNotSupported) {
    set_last_error("pecann_density_noalloc: unsupported combination");
    return PECANN_EUNSUPPORTED;
  }
  if (e != cudaSuccess) {
    set_last_error(std::string("pecann_density_noalloc: ") + cudaGetErrorString(e));
    return PECANN_ECUDA;
  }
  return PECANN_OK;
}
