// Batched wave kernels with w' and the gradient accumulator in global memory
// (tall bands): BF16 snapshots.
#include "wave_inst.cuh"
namespace vip {
const void *wave_gw_bf16(int V, int mode) { return wave_kernel_table<__nv_bfloat16, true>(V, mode); }
}  // namespace vip
