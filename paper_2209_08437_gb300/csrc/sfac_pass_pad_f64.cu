// FP64 instantiations of the zero-padded axis pass (grid lengths that
// are not powers of two, run as linear convolutions of power-of-two length).
#include "sfac_pass.cuh"

namespace sfac {
cudaError_t launch_pass_padded_f64(int N, const PassArgs& a, cudaStream_t s) {
    return launch_pass_any<double, true>(N, a, s);
}
}  // namespace sfac
