// Maps a dataset (dtype, metric, d) to the compiled distance layout
// instance: f(dt, metric, W, CPL) is called with std::integral_constant
// arguments for the one combination that serves the dataset.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace pecann {

template <int V>
using IC = std::integral_constant<int, V>;

// f(W, CPL) for the compiled layout of dtype DT that serves L.
template <int DT, class F>
cudaError_t dispatch_wc(const Layout& L, F&& f) {
  if constexpr (DT == DT_U8) {
    if (L.W == 8) return f(IC<8>{}, IC<1>{});
    return f(IC<16>{}, IC<1>{});
  } else {
    if (L.W == 8) return f(IC<8>{}, IC<1>{});
    if (L.W == 16) return f(IC<16>{}, IC<1>{});
    if (L.CPL == 1) return f(IC<32>{}, IC<1>{});
    if (L.CPL == 2) return f(IC<32>{}, IC<2>{});
    if (L.CPL == 3) return f(IC<32>{}, IC<3>{});
    if (L.CPL == 4) return f(IC<32>{}, IC<4>{});
    return f(IC<32>{}, IC<8>{});
  }
}

template <class F>
cudaError_t dispatch_layout(const DataView& dv, F&& f) {
  Layout L;
  if (!pick_layout(dv.dtype, dv.metric, dv.d, &L)) return cudaErrorNotSupported;
  auto go = [&](auto dt, auto met) -> cudaError_t {
    if (L.W == 8) return f(dt, met, IC<8>{}, IC<1>{});
    if (L.W == 16) return f(dt, met, IC<16>{}, IC<1>{});
    if (L.CPL == 1) return f(dt, met, IC<32>{}, IC<1>{});
    if (L.CPL == 2) return f(dt, met, IC<32>{}, IC<2>{});
    if (L.CPL == 3) return f(dt, met, IC<32>{}, IC<3>{});
    if (L.CPL == 4) return f(dt, met, IC<32>{}, IC<4>{});
    return f(dt, met, IC<32>{}, IC<8>{});
  };
  if (dv.dtype == DT_F32 && dv.metric == MET_L2) return go(IC<DT_F32>{}, IC<MET_L2>{});
  if (dv.dtype == DT_F32 && dv.metric == MET_IP) return go(IC<DT_F32>{}, IC<MET_IP>{});
  if (dv.dtype == DT_BF16 && dv.metric == MET_L2) return go(IC<DT_BF16>{}, IC<MET_L2>{});
  if (dv.dtype == DT_BF16 && dv.metric == MET_IP) return go(IC<DT_BF16>{}, IC<MET_IP>{});
  if (dv.dtype == DT_U8 && dv.metric == MET_L2) {
    if (L.W == 8) return f(IC<DT_U8>{}, IC<MET_L2>{}, IC<8>{}, IC<1>{});
    return f(IC<DT_U8>{}, IC<MET_L2>{}, IC<16>{}, IC<1>{});
  }
  return cudaErrorNotSupported;
}

}  // namespace pecann
