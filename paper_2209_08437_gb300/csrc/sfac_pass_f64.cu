// FP64 instantiations of the fused axis pass (one translation unit per
// precision so that the two compile in parallel).
#include "sfac_pass.cuh"

namespace sfac {
cudaError_t launch_pass_f64(int N, const PassArgs& a, cudaStream_t s) {
    return launch_pass_any<double, false>(N, a, s);
}
}  // namespace sfac
