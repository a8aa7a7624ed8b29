// Batched wave kernels with w' and the gradient accumulator in global memory
// (tall bands): FP32 snapshots and forward-only.
#include "wave_inst.cuh"
namespace vip {
const void *wave_gw_f32(int V, int mode) { return wave_kernel_table<float, true>(V, mode); }
const void *wave_gw_fwd(int V) { return wave_fwd_table<true>(V); }
}  // namespace vip
