// pecann_density_noalloc: the k-NN + density entry point for callers that
// cannot allocate GPU memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- a
// real-time loop that must not take the allocator's lock (a cudaMalloc can
// synchronise the device), code under an external memory manager that owns
// every device byte, or a process whose allocations are frozen after
// start-up. Such a caller can hand
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

#include <string>

#include "common.cuh"
#include "internal.h"

namespace pecann {

// Layout of the fixed scratch: a 256-byte header (error word, fallback
// counter) followed by the fallback list and the raw-density copy of up to
// PECANN_NOALLOC_MAX_POINTS points each.
static const size_t NOALLOC_HDR = 256;
static const size_t NOALLOC_LIST = (size_t)PECANN_NOALLOC_MAX_POINTS * 4;
static const size_t NOALLOC_BYTES = NOALLOC_HDR + 2 * NOALLOC_LIST;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

}  // namespace pecann

using namespace pecann;

extern "C" pecann_status pecann_density_noalloc(const pecann_dataset* ds, const int32_t* d_graph,
                                                const pecann_params* p, int32_t* d_knn_ids, float* d_knn_dist,
                                                float* d_density, float* d_rank_key, void* stream) {
  // the same checks as pecann_density, then the limits of this entry point
  DataView dv, fv;
  pecann_status s = check_dataset(ds, &dv, &fv);
  if (s) return s;
  if ((s = check_density_args(dv, d_graph, p, d_knn_ids, d_knn_dist, d_density, d_rank_key))) return s;
  if (dv.n > PECANN_NOALLOC_MAX_POINTS) {
    set_last_error("pecann_density_noalloc: n exceeds PECANN_NOALLOC_MAX_POINTS (1048576); "
                   "use pecann_density with a workspace");
    return PECANN_EINVAL;
  }
  if (dv.dtype == DT_BF16 || dv.dtype == DT_FP8) {
    set_last_error("pecann_density_noalloc: BF16 / FP8 traversal needs pecann_density (its re-rank scratch)");
    return PECANN_EUNSUPPORTED;
  }
  // The device address of the scratch array in the current device's context.
  // In host code the symbol is only a host-side handle, never a device
  // address. The address is looked up on every call (a cheap query), so a
  // context that was destroyed and created again -- the module loaded at
  // another address -- is never written through a stale pointer.
  void* scratch = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
  if (e != cudaSuccess) {
    set_last_error(std::string("pecann_density_noalloc: scratch lookup: ") + cudaGetErrorString(e));
    return PECANN_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  uint8_t* base = (uint8_t*)scratch;
  DensityScratch sc;
  sc.err = (int*)base;
  sc.fb_cnt = (int32_t*)(base + 8);
  sc.fb_list = (int32_t*)(base + NOALLOC_HDR);
  sc.raw = (float*)(base + NOALLOC_HDR + NOALLOC_LIST);
  // the error word and the fallback counter must start at zero; the list
  // and the density copy are written before they are read
  if ((e = cudaMemsetAsync(base, 0, NOALLOC_HDR, st)) != cudaSuccess) return cuda_status(e, "memset");
  return run_density(dv, fv, d_graph, p, d_knn_ids, d_knn_dist, d_density, d_rank_key, sc, st);
}
