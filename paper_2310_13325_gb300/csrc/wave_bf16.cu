// Batched wave kernels with BF16 snapshots.
#include "wave_inst.cuh"
namespace vip {
const void *wave_kernel_bf16(int V, int mode, bool gw) {
  return gw ? wave_gw_bf16(V, mode) : wave_kernel_table<__nv_bfloat16, false>(V, mode);
}
}  // namespace vip
