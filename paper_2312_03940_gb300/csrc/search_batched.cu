// Beam-search instances of the batched form (many FP32 point sets, one launch).
#include "search_kernel.cuh"

namespace pecann {

cudaError_t launch_search_batched(const DataView& dv, const SearchArgs& a, const Layout& L, cudaStream_t st) {
  if (dv.dtype != DT_F32) return cudaErrorNotSupported;
  return dispatch_wc<DT_F32>(L, [&](auto wv, auto cpl) -> cudaError_t {
    constexpr int W = decltype(wv)::value, CPL = decltype(cpl)::value;
    if (dv.metric == MET_IP) return launch_inst<DT_F32, MET_IP, W, CPL, true>(a, st);
    return launch_inst<DT_F32, MET_L2, W, CPL, true>(a, st);
  });
}

}  // namespace pecann
