// Batched wave kernels with FP32 snapshots (and the forward-only kernels).
#include "wave_inst.cuh"
namespace vip {
const void *wave_kernel_f32(int V, int mode) {
  if (mode == WM_FORWARD) {
    if (V == 4) return reinterpret_cast<const void *>(&wave_cluster_kernel<4, WM_FORWARD, float>);
    if (V == 8) return reinterpret_cast<const void *>(&wave_cluster_kernel<8, WM_FORWARD, float>);
    return nullptr;
  }
  return wave_kernel_table<float>(V, mode);
}
}  // namespace vip
