// Beam-search instances for FP8 e4m3 rows (inner product, per-dimension
// scale; the FP32 rows give the query side).
#include "search_kernel.cuh"

namespace pecann {

cudaError_t launch_search_fp8(const DataView& dv, const SearchArgs& a, const Layout& L, cudaStream_t st) {
  (void)dv;
  if (L.W == 8) return launch_inst<DT_FP8, MET_IP, 8, 1, false>(a, st);
  if (L.W == 16) return launch_inst<DT_FP8, MET_IP, 16, 1, false>(a, st);
  if (L.CPL == 1) return launch_inst<DT_FP8, MET_IP, 32, 1, false>(a, st);
  return launch_inst<DT_FP8, MET_IP, 32, 2, false>(a, st);
}

}  // namespace pecann
