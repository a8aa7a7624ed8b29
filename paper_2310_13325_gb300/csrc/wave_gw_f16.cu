// Batched wave kernels with w' and the gradient accumulator in global memory
// (tall bands): FP16 snapshots with power-of-two block scales.
#include "wave_inst.cuh"
namespace vip {
const void *wave_gw_f16(int V, int mode) { return wave_kernel_table<__half, true>(V, mode); }
}  // namespace vip
