// sfac_probe.cu - microbenchmark of the SMs' multiply-add rate, the ALU
// roofline that the FP64 and FP32 axis passes are reported against; and the
// nonlinear flow J^Q evaluated value by value with the passes' own code.
//
// Every thread runs PROBE_CHAINS independent chains x <- fma(x, a, b), so the
// pipes see enough independent work to issue back to back; a and b keep the
// chains bounded (|a| < 1). Each thread stores the sum of its chains, so the
// compiler cannot drop the loop. The caller times the launch with events.
#include <cuda_runtime.h>

#include <string>

#include "sfac.h"
#include "sfac_internal.h"
#include "sfac_pass.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_UNROLL = 16;

template <typename R>
__global__ void __launch_bounds__(PROBE_THREADS) fma_rate_kernel(R* out, long long iters, R a, R b) {
    R x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = R(threadIdx.x + k) * R(1e-3);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < PROBE_UNROLL; ++r) {
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fma(x[k], a, b);
        }
    }
    R s = R(0);
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
    out[(long long)blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

// The same with the packed two-lane FP32 multiply-add of sm_100+ (each chain a
// pair of floats).
__global__ void __launch_bounds__(PROBE_THREADS) fma2_rate_kernel(float* out, long long iters, float a, float b) {
    float2 x[PROBE_CHAINS];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = make_float2((threadIdx.x + k) * 1e-3f, (threadIdx.x - k) * 1e-3f);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < PROBE_UNROLL; ++r) {
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k].x + x[k].y;
    out[(long long)blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

// J^Q on n values, two per thread as the passes hold them (C2 pairs).
template <typename R>
__global__ void __launch_bounds__(256) jq_probe_kernel(const R* v, R* out, long long n, double E0, double om) {
    const long long i = 2 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= n) return;
    sfac::C2<R> x[1] = {{v[i], i + 1 < n ? v[i + 1] : R(0)}};
    if constexpr (sizeof(R) == 8) {
        sfac::jq_all<R, 1>(x, E0, om);
    } else {
        const float omf = float(om);
        x[0] = {x[0].x + sfac::jq_increment(x[0].x, omf), x[0].y + sfac::jq_increment(x[0].y, omf)};
    }
    out[i] = x[0].x;
    if (i + 1 < n) out[i + 1] = x[0].y;
}

}  // namespace

extern "C" sfac_status sfac_probe_jq(int prec, const void* v_dev, void* out_dev, long long n, double E,
                                     double one_minus_E, void* stream) try {
    if (prec != SFAC_FP64 && prec != SFAC_FP32) {
        sfac::set_last_error("prec must be SFAC_FP64 or SFAC_FP32");
        return SFAC_EINVAL;
    }
    if (n < 0 || n > (1LL << 36) || (n > 0 && (!v_dev || !out_dev)) || !(E > 0.0 && E <= 1.0)) {
        sfac::set_last_error("need 0 <= n <= 2^36, device buffers for n > 0 and E in (0, 1]");
        return SFAC_EINVAL;
    }
    if (n == 0) return SFAC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long blocks = ((n + 1) / 2 + 255) / 256;
    if (prec == SFAC_FP64)
        jq_probe_kernel<double><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const double*>(v_dev),
                                                                static_cast<double*>(out_dev), n, E, one_minus_E);
    else
        jq_probe_kernel<float><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const float*>(v_dev),
                                                               static_cast<float*>(out_dev), n, E, one_minus_E);
    const cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        sfac::set_last_error(std::string("probe launch: ") + cudaGetErrorString(err));
        return SFAC_ECUDA;
    }
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

extern "C" sfac_status sfac_probe_fma(int kind, int blocks, long long iters, void* out_dev, void* stream) try {
    if (kind < 0 || kind > 2) {
        sfac::set_last_error("kind must be 0 (FP64), 1 (FP32) or 2 (packed FP32)");
        return SFAC_EINVAL;
    }
    if (blocks < 1 || iters < 1 || !out_dev) {
        sfac::set_last_error("need blocks >= 1, iters >= 1 and an output buffer");
        return SFAC_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (kind == 0)
        fma_rate_kernel<double><<<blocks, PROBE_THREADS, 0, s>>>(static_cast<double*>(out_dev), iters, 0.999, 1e-4);
    else if (kind == 1)
        fma_rate_kernel<float><<<blocks, PROBE_THREADS, 0, s>>>(static_cast<float*>(out_dev), iters, 0.999f, 1e-4f);
    else
        fma2_rate_kernel<<<blocks, PROBE_THREADS, 0, s>>>(static_cast<float*>(out_dev), iters, 0.999f, 1e-4f);
    const cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        sfac::set_last_error(std::string("probe launch: ") + cudaGetErrorString(err));
        return SFAC_ECUDA;
    }
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}
