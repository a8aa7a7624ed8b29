// Explicit instantiations of the batched wave kernel, one translation unit
// per snapshot type so that the library compiles in parallel.
#pragma once
#include "wave.cuh"

namespace vip {

// Kernel address for (rows per thread V, mode, snapshot type); nullptr when
// that combination is not built.
const void *wave_kernel_f32(int V, int mode);
const void *wave_kernel_bf16(int V, int mode);
const void *wave_kernel_f16(int V, int mode);
const void *wave_kernel_fwd(int V);

// Largest CTA size the kernel for V rows per thread is built for.
inline int wave_max_threads(int V) {
  return V >= 10 ? WaveMaxThreads<10>::value : (V >= 8 ? WaveMaxThreads<8>::value : WaveMaxThreads<4>::value);
}

template <class DT>
const void *wave_kernel_table(int V, int mode) {
#define VIP_K(VV, MM)                                                  \
  if (V == VV && mode == MM)                                           \
    return reinterpret_cast<const void *>(&wave_cluster_kernel<VV, MM, DT>);
  VIP_K(4, WM_GRADIENT) VIP_K(4, WM_ADJOINT)
  VIP_K(5, WM_GRADIENT) VIP_K(5, WM_ADJOINT)
  VIP_K(8, WM_GRADIENT) VIP_K(8, WM_ADJOINT)
  VIP_K(10, WM_GRADIENT) VIP_K(10, WM_ADJOINT)
#undef VIP_K
  return nullptr;
}

}  // namespace vip
