// FP32 (complex64) instantiations of the fused axis pass. The tables they read
// were computed in FP64 on the host and rounded once to FP32.
#include "sfac_pass.cuh"

namespace sfac {
cudaError_t launch_pass_f32(int N, const PassArgs& a, cudaStream_t s) {
    return launch_pass_any<float, false>(N, a, s);
}
}  // namespace sfac
