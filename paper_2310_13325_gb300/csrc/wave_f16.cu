// Batched wave kernels with FP16 snapshots and power-of-two block scales.
#include "wave_inst.cuh"
namespace vip {
const void *wave_kernel_f16(int V, int mode, bool gw) {
  return gw ? wave_gw_f16(V, mode) : wave_kernel_table<__half, false>(V, mode);
}
}  // namespace vip
