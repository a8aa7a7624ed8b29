// Batched forward-only wave kernels (traces, no snapshots).
#include "wave_inst.cuh"
namespace vip {
const void *wave_kernel_fwd(int V) {
  if (V == 4) return reinterpret_cast<const void *>(&wave_cluster_kernel<4, WM_FORWARD, float>);
  if (V == 5) return reinterpret_cast<const void *>(&wave_cluster_kernel<5, WM_FORWARD, float>);
  if (V == 8) return reinterpret_cast<const void *>(&wave_cluster_kernel<8, WM_FORWARD, float>);
  if (V == 10) return reinterpret_cast<const void *>(&wave_cluster_kernel<10, WM_FORWARD, float>);
  return nullptr;
}
}  // namespace vip
