// FP32 batch kernels (values per thread 8 or 16 for lines up to 256 points).
// The batch kernel runs the rolled FP32 chain (sfac_pass.cuh) for lines of up
// to 128 points only: measured on GB300, its 256-point passes were faster
// unrolled (mixed 2D batch 52.6 against 48.9 G point-steps/s) while batches
// of 3D n = 64 and 128 instances ran the same.
#define SFAC_ROLLED_MAX_N 128
#include "sfac_batch.cuh"

namespace sfac {
cudaError_t setup_batch_f32(int wpb, int es, int stage, int sms, int* grid) {
    if (es == 16) return setup_batch<float, 16>(wpb, stage, sms, grid);
    if (es == 8) return setup_batch<float, 8>(wpb, stage, sms, grid);
    return cudaErrorInvalidValue;
}
cudaError_t launch_batch_f32(int wpb, int es, int grid, const BatchSchedule& sc, cudaStream_t s) {
    if (es == 16) return launch_batch<float, 16>(wpb, grid, sc, s);
    if (es == 8) return launch_batch<float, 8>(wpb, grid, sc, s);
    return cudaErrorInvalidValue;
}
}  // namespace sfac
