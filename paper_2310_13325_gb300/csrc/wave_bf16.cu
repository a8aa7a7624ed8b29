// Batched wave kernels with BF16 snapshots.
#include "wave_inst.cuh"
namespace vip {
const void *wave_kernel_bf16(int V, int mode) { return wave_kernel_table<__nv_bfloat16>(V, mode); }
}  // namespace vip
