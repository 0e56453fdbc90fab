// Beam-search instances for uint8 rows (L2).
#include "search_kernel.cuh"

namespace pecann {

cudaError_t launch_search_u8(const DataView& dv, const SearchArgs& a, const Layout& L, cudaStream_t st) {
  (void)dv;
  return dispatch_wc<DT_U8>(L, [&](auto wv, auto cpl) -> cudaError_t {
    return launch_inst<DT_U8, MET_L2, decltype(wv)::value, decltype(cpl)::value, false>(a, st);
  });
}

}  // namespace pecann
