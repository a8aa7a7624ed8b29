// Batched forward-only wave kernels (traces, no snapshots).
#include "wave_inst.cuh"
namespace vip {
const void *wave_kernel_fwd(int V, bool gw) { return gw ? wave_gw_fwd(V) : wave_fwd_table<false>(V); }
}  // namespace vip
