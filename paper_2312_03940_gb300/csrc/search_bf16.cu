// Beam-search instances for BF16 traversal rows (L2 and inner product).
#include "search_kernel.cuh"

namespace pecann {

cudaError_t launch_search_bf16(const DataView& dv, const SearchArgs& a, const Layout& L, cudaStream_t st) {
  return dispatch_wc<DT_BF16>(L, [&](auto wv, auto cpl) -> cudaError_t {
    constexpr int W = decltype(wv)::value, CPL = decltype(cpl)::value;
    if (dv.metric == MET_IP) return launch_inst<DT_BF16, MET_IP, W, CPL, false>(a, st);
    return launch_inst<DT_BF16, MET_L2, W, CPL, false>(a, st);
  });
}

}  // namespace pecann
