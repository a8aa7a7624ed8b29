// Explicit instantiations of the batched wave kernel, one translation unit
// per snapshot type so that the library compiles in parallel.
#pragma once
#include "wave.cuh"

namespace vip {

// Kernel address for (rows per thread V, mode, snapshot type, coefficients in
// global memory); nullptr when that combination is not built.
const void *wave_kernel_f32(int V, int mode, bool gw);
const void *wave_kernel_bf16(int V, int mode, bool gw);
const void *wave_kernel_f16(int V, int mode, bool gw);
const void *wave_kernel_fwd(int V, bool gw);
// the coefficients-in-global-memory instantiations, one translation unit each
const void *wave_gw_f32(int V, int mode);
const void *wave_gw_bf16(int V, int mode);
const void *wave_gw_f16(int V, int mode);
const void *wave_gw_fwd(int V);

// Largest CTA size the kernel for V rows per thread is built for.
inline int wave_max_threads(int V, bool gw) {
  if (gw) return WaveMaxThreads<4, true>::value;
  return V >= 10 ? WaveMaxThreads<10>::value
                 : (V >= 8 ? WaveMaxThreads<8>::value : WaveMaxThreads<4>::value);
}

// Gradient / adjoint kernels; the global-coefficient variant exists for
// 4, 5 and 8 rows per thread (the tall bands it is meant for).
template <class DT, bool GW>
const void *wave_kernel_table(int V, int mode) {
#define VIP_K(VV, MM)                                                  \
  if (V == VV && mode == MM)                                           \
    return reinterpret_cast<const void *>(&wave_cluster_kernel<VV, MM, DT, GW>);
  VIP_K(4, WM_GRADIENT) VIP_K(4, WM_ADJOINT)
  VIP_K(5, WM_GRADIENT) VIP_K(5, WM_ADJOINT)
  VIP_K(8, WM_GRADIENT) VIP_K(8, WM_ADJOINT)
  if constexpr (!GW) {
    VIP_K(10, WM_GRADIENT) VIP_K(10, WM_ADJOINT)
  }
#undef VIP_K
  return nullptr;
}

// Forward-only kernels (traces, no snapshots).
template <bool GW>
const void *wave_fwd_table(int V) {
  if (V == 4) return reinterpret_cast<const void *>(&wave_cluster_kernel<4, WM_FORWARD, float, GW>);
  if (V == 5) return reinterpret_cast<const void *>(&wave_cluster_kernel<5, WM_FORWARD, float, GW>);
  if (V == 8) return reinterpret_cast<const void *>(&wave_cluster_kernel<8, WM_FORWARD, float, GW>);
  if constexpr (!GW) {
    if (V == 10)
      return reinterpret_cast<const void *>(&wave_cluster_kernel<10, WM_FORWARD, float, GW>);
  }
  return nullptr;
}

}  // namespace vip
