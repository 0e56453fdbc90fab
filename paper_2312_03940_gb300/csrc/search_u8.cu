// Beam-search instances for uint8 rows (L2).
#include "search_kernel.cuh"

namespace pecann {

cudaError_t launch_search_u8(const DataView& dv, const SearchArgs& a, const Layout& L, cudaStream_t st) {
  (void)dv;
  // 128-byte rows on a 32-byte aligned base: 4 lanes per row, one 32-byte
  // load each (the 16-byte row alignment the interface asks for is not
  // enough for that load, so other bases take the 8-lane layout)
  if (L.W == 8 && a.C == 8 && a.row_bytes == 128 && (((uintptr_t)a.X) & 31) == 0)
    return launch_inst<DT_U8, MET_L2, 4, 2, false>(a, st);
  return dispatch_wc<DT_U8>(L, [&](auto wv, auto cpl) -> cudaError_t {
    return launch_inst<DT_U8, MET_L2, decltype(wv)::value, decltype(cpl)::value, false>(a, st);
  });
}

}  // namespace pecann
