// FP64 batch kernel (16 values per thread).
#include "sfac_batch.cuh"

namespace sfac {
cudaError_t setup_batch_f64(int wpb, int es, int stage, int sms, int* grid) {
    (void)es;
    (void)stage;  // FP64 items are not staged
    return setup_batch<double, 16>(wpb, 0, sms, grid);
}
cudaError_t launch_batch_f64(int wpb, int es, int grid, const BatchSchedule& sc, cudaStream_t s) {
    (void)es;
    return launch_batch<double, 16>(wpb, grid, sc, s);
}
}  // namespace sfac
