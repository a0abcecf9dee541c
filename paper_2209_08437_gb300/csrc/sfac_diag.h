// sfac_diag.h - launchers of the diagnostic reductions (sfac_diag.cu).
#pragma once

#include <cuda_runtime.h>

#include "sfac_internal.h"

namespace sfac {

// Number of per-CTA partials one diagnostic pass over `clines` complex lines of
// FFT length N writes.
long long diag_partials_needed(long long clines, int N);

// One diagnostic pass over the lines of `a` (field of doubles or floats,
// f64_field): accumulates into out[0] the sum of x . B x over its lines, into
// out[1] (first_axis only) the sum of (u^2 - 1)^2 and into out[2] the max of
// |u|. Tables are FP64: non-padded axes mA = lambda/N, mB = mu/N with a.twist,
// a.twid FP64; zero-padded axes mA = the real multiplier of B as a padded
// linear convolution (incl. 1/L), mB unused. `partial` holds at least
// diag_partials_needed(...) entries.
cudaError_t launch_diag_axis(bool f64_field, bool padded, int N, const PassArgs& a, const double* mA,
                             const double* mB, int first_axis, double3* partial, double* out, cudaStream_t s);

}  // namespace sfac
