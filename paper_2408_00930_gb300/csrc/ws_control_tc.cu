// ws_control_tc.cu -- fused persistent BF16 tensor-core control kernel.
#include "ws_kernels.cuh"

namespace ws {
size_t control_tc_packed_bytes(const PolicyShape &) { return 0; }
bool control_tc_supported(const PolicyShape &) { return false; }
void launch_control_tc_pack(const Dev &, void *, cudaStream_t) {}
cudaError_t launch_control_tc(const Dev &, const void *, uint32_t, int, cudaStream_t) {
  return cudaErrorNotSupported;
}
int control_tc_default_grid(const Dev &) { return 0; }
}  // namespace ws
