// Batched wave kernels with FP32 snapshots.
#include "wave_inst.cuh"
namespace vip {
const void *wave_kernel_f32(int V, int mode, bool gw) {
  if (mode == WM_FORWARD) return wave_kernel_fwd(V, gw);
  return gw ? wave_gw_f32(V, mode) : wave_kernel_table<float, false>(V, mode);
}
}  // namespace vip
