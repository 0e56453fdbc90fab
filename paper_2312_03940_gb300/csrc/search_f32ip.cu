// Beam-search instances for FP32 rows, inner product.
#include "search_kernel.cuh"

namespace pecann {

cudaError_t launch_search_f32_ip(const DataView& dv, const SearchArgs& a, const Layout& L, cudaStream_t st) {
  (void)dv;
  return dispatch_wc<DT_F32>(L, [&](auto wv, auto cpl) -> cudaError_t {
    return launch_inst<DT_F32, MET_IP, decltype(wv)::value, decltype(cpl)::value, false>(a, st);
  });
}

}  // namespace pecann
