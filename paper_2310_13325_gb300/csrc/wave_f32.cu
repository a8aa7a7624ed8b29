// Batched wave kernels with FP32 snapshots.
#include "wave_inst.cuh"
namespace vip {
const void *wave_kernel_f32(int V, int mode) {
  if (mode == WM_FORWARD) return wave_kernel_fwd(V);
  return wave_kernel_table<float>(V, mode);
}
}  // namespace vip
