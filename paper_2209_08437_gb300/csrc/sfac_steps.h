// sfac_steps.h - the whole-call launch for small grids (sfac_steps.cu).
// Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include "sfac_internal.h"

namespace sfac {

// Arguments of one launch that runs `nsteps` whole steps of a small grid.
struct StepsArgs {
    PassArgs ax[3];      // one pass per axis (tables, field view); J^Q set per step in the kernel
    int n[3];            // FFT length of each axis: a power of two in [32, 256]
    int dim;
    long long nsteps;    // >= 1
    double jq_half_E, jq_half_1mE, jq_full_E, jq_full_1mE;
    unsigned int* bar;   // device: [0] arrivals, [1] generation (reset by the launch)
    unsigned int* status;  // device: SFAC_PASS_TIMEOUT when a barrier wait ran out
    long long wait_cycles;  // limit of each barrier wait, SM clock cycles
    int hold;            // test hook: the first barrier wait of every CTA never completes
};

// CTAs the launch needs: the largest number of warp-groups of an axis pass.
long long steps_grid(const StepsArgs& g);
// Whether that many CTAs are resident at once in a cooperative launch on the
// current device (precision SFAC_FP64 / SFAC_FP32).
bool steps_fit(int prec, const StepsArgs& g);
// Reset the barrier and enqueue the cooperative launch on `s`;
// cudaErrorNotSupported (nothing enqueued) when steps_fit is false.
cudaError_t launch_steps(int prec, const StepsArgs& g, cudaStream_t s);

}  // namespace sfac
