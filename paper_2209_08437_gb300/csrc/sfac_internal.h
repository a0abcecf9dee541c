// sfac_internal.h - declarations shared by the host side of libsfac and the
// kernel translation units. Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "sfac.h"

namespace sfac {

// Record the message returned by sfac_last_error() for the calling thread.
void set_last_error(const std::string& msg);

// Status of a C ABI entry point whose body threw: called from the entry
// point's catch handler, it records a message and returns SFAC_ENOMEM (host
// memory, threads or other host resources ran out). No exception leaves the ABI.
sfac_status abi_exception_status() noexcept;

// Arguments of one fused axis pass over the field (see sfac_pass.cuh).
//
// The field is viewed along the pass axis as [outer][N][inner] reals:
// element k of the line (o, i) sits at (o * N + k) * inner + i.
//  - contiguous pass (inner == 1): real lines are the `outer` rows; rows 2c and
//    2c+1 form complex line c (the odd last row, if any, pairs with zeros);
//  - strided pass (inner > 1, even): columns 2c and 2c+1 of one outer slab form
//    complex line c, read and written as one 2-real vector.
// Tables (device pointers, plan precision R):
//  eC[j]  = e^{tau/2 lambda_j} / N   circulant factor incl. the inverse-FFT 1/N
//  eS[j]  = e^{tau mu_j} / N         skew-circulant factor incl. 1/N
//  (FP32 plans: expm1(tau/2 lambda_j) / N and expm1(tau mu_j) / N, the
//   increments the FP32 passes add; see sfac_pass.cuh)
//  twist  = N complex e^{i pi k / N} (interleaved re, im)
//  twid   = N complex e^{-2 pi i m / N}
//  rtwid  = FP64 CTA passes (E values per thread as below): the ratio-twiddle
//           records of the FFT passes (sfac_fft.cuh, FftPassRatio)
// J^Q_s(v) = v / sqrt(E + (1 - E) v^2) with E = e^{-2 s} is applied to every
// value on load when jq_in != 0 and on store when jq_out != 0.
struct PassArgs {
    void* u;
    long long outer;
    long long inner;
    long long clines;  // number of complex lines
    int nmem;          // line length in memory: N, or n < N for a zero-padded pass
    const void* eC;
    const void* eS;
    const void* twist;
    const void* twid;
    const void* rtwid = nullptr;
    // FP32 warp-local passes: the per-thread twiddle rows of TwRows<N, E>
    // (sfac_fft.cuh), built in shared memory by the kernel (NULL otherwise).
    const void* twrows = nullptr;
    double jq_in_E, jq_in_1mE;
    double jq_out_E, jq_out_1mE;
    int jq_in, jq_out;
    // Device word where a kernel that gave up waiting for one of its own
    // asynchronous copies records SFAC_PASS_TIMEOUT (NULL: not recorded).
    unsigned int* status = nullptr;
    // Limit of each such wait in SM clock cycles (about two seconds by
    // default), and a test hook: hold != 0 makes the first wait of every CTA
    // wait for a barrier that nothing completes, so that the limit runs out.
    long long wait_cycles = 4LL << 30;
    int hold = 0;
    // Store base minus load base, in elements: 0 for a pass in place. A pass
    // that moves the field between host memory mapped into the device's
    // address space and device memory loads from u and stores to u + out_shift
    // (host_io != 0); such passes run on the plain-load kernels, never TMA.
    long long out_shift = 0;
    int host_io = 0;
};

constexpr unsigned int SFAC_PASS_TIMEOUT = 1u;

// Values per thread of the FP64 CTA pass for FFT length N; its FFTs run on
// ratio twiddles (radix 8/4/2, and radix 16 at 4096 points). 4096-point lines
// take 16 values (256 threads a line: 8 values would need 512 threads of about
// 180 registers, more than an SM holds).
__host__ __device__ constexpr int f64_elems_per_thread(int N) { return N >= 4096 ? 16 : (N < 8 ? N : 8); }

// Launch one pass for line length N (a power of two in [4, 4096]).
// Returns cudaErrorInvalidValue for an unsupported N.
cudaError_t launch_pass_f64(int N, const PassArgs& a, cudaStream_t s);
cudaError_t launch_pass_f32(int N, const PassArgs& a, cudaStream_t s);

// Zero-padded pass: lines of a.nmem < N points, FFT length N = L (a power of two
// >= 2 nmem - 1, in [4, 4096]). The tables are then eC = multiplier of e^{tau/2 C}
// and eS = multiplier of e^{tau S} as linear convolutions (real, incl. 1/L;
// increment forms for FP32), twist = NULL, twid = L twiddles. Each factor is
// FFT, multiply, inverse FFT, zero the values past nmem.
cudaError_t launch_pass_padded_f64(int N, const PassArgs& a, cudaStream_t s);
cudaError_t launch_pass_padded_f32(int N, const PassArgs& a, cudaStream_t s);

// FP32 strided pass with TMA-staged tiles (sfac_pass_staged.cuh). Returns
// cudaErrorNotSupported, having enqueued nothing, when the pass does not
// qualify (see staged_pass_eligible); the caller then uses launch_pass_f32.
cudaError_t launch_pass_staged_f32(int N, const PassArgs& a, cudaStream_t s);
// Whether launch_pass_staged_f32 takes this pass: FP32 lines of a power-of-two
// N in [32, 512] (not zero-padded), a strided axis with inner % 4 == 0 and
// inner >= the tile width, at least one tile per SM, u 16-byte aligned, and the
// driver's tensor-map encoder available.
bool staged_pass_eligible(int N, const PassArgs& a);

}  // namespace sfac
