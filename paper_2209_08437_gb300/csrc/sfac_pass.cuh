// sfac_pass.cuh - the fused axis pass of the two-level Strang step.
//
// One launch applies, to every grid line of one axis,
//   [J^Q on load]  e^{tau/2 C} e^{tau S} e^{tau/2 C}  [J^Q on store]
// (eqs. (hatv), (finalstrang), Sec. 2.2) with the field read once from and
// written once to global memory. Two real lines travel as one complex line
// z = v_a + i v_b: the factor is a real matrix (C and S are real symmetric), so
// applying it complex-linearly to z gives P v_a + i P v_b and halves the FFTs.
// Per complex line the chain is
//   FFT, * e^{tau/2 lambda}/N, IFFT, * e^{i pi k/N},
//   FFT, * e^{tau mu}/N,       IFFT, * e^{-i pi k/N},
//   FFT, * e^{tau/2 lambda}/N, IFFT
// with the spectra of Remark 1, all in registers between shared-memory
// exchanges of the Stockham passes (sfac_fft.cuh).
#pragma once

#include "sfac_fft.cuh"
#include "sfac_internal.h"

namespace sfac {

template <typename R>
struct Vec2T;
template <>
struct Vec2T<double> { using type = double2; };
template <>
struct Vec2T<float> { using type = float2; };

__device__ __forceinline__ double rsqrt_r(double v) { return rsqrt(v); }
__device__ __forceinline__ float rsqrt_r(float v) { return rsqrtf(v); }

// Exact nonlinear flow J^Q_s(v) = v / sqrt(E + (1 - E) v^2), E = e^{-2s}
// (eq. (nonlinear_operator)); E and 1 - E come from the host in FP64.
template <typename R>
__device__ __forceinline__ R jq_flow(R v, R E, R omE) {
    return v * rsqrt_r(fma(v * v, omE, E));
}

template <typename R>
__device__ __forceinline__ C2<R> ldg_c2(const C2<R>* p) {
    using V = typename Vec2T<R>::type;
    const V v = __ldg(reinterpret_cast<const V*>(p));
    return {v.x, v.y};
}

// Shared-memory exchange with a bank-spreading pad: element a is stored at
// a + (a >> LOG) where 2^LOG complex values fill 128 bytes.
template <typename R, int N, int LPC, bool IDX_MAJOR>
struct PadExchange {
    static constexpr int LOG = (sizeof(R) == 8) ? 3 : 4;
    C2<R>* base;
    int j;
    __device__ __forceinline__ int addr(int idx) const {
        const int a = IDX_MAJOR ? idx * LPC + j : j * N + idx;
        return a + (a >> LOG);
    }
    __device__ __forceinline__ void put(int idx, C2<R> v) const { base[addr(idx)] = v; }
    __device__ __forceinline__ C2<R> get(int idx) const { return base[addr(idx)]; }
    static __device__ __forceinline__ void sync() { __syncthreads(); }
    static constexpr int elems() { return N * LPC + ((N * LPC) >> LOG) + 1; }
};

template <typename R, int N, int E, int LPC, bool STRIDED>
__global__ void __launch_bounds__(LPC*(N / E))
axis_pass_kernel(const PassArgs a) {
    constexpr int T = N / E;
    using Ex = PadExchange<R, N, LPC, STRIDED>;
    using V = typename Vec2T<R>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int tid = threadIdx.x;
    const int j = STRIDED ? (tid % LPC) : (tid / T);
    const int t = STRIDED ? (tid / LPC) : (tid % T);
    const long long cl = (long long)blockIdx.x * LPC + j;
    const bool active = cl < a.clines;
    const Ex ex{reinterpret_cast<C2<R>*>(smem_raw), j};

    R* __restrict__ u = static_cast<R*>(a.u);
    const C2<R>* __restrict__ tw = static_cast<const C2<R>*>(a.twid);
    const C2<R>* __restrict__ twist = static_cast<const C2<R>*>(a.twist);
    const R* __restrict__ eC = static_cast<const R*>(a.eC);
    const R* __restrict__ eS = static_cast<const R*>(a.eS);

    // ---- load (and J^Q) -------------------------------------------------
    C2<R> x[E];
    R* p0;
    R* p1 = nullptr;
    long long stride = 1;
    if (STRIDED) {
        const long long pairs = a.inner >> 1;
        const long long o = active ? cl / pairs : 0;
        const long long c = active ? cl - o * pairs : 0;
        p0 = u + o * (long long)N * a.inner + 2 * c;
        stride = a.inner;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = t + e * T;
            if (active) {
                const V v = *reinterpret_cast<const V*>(p0 + idx * stride);
                x[e] = {v.x, v.y};
            } else {
                x[e] = {R(0), R(0)};
            }
        }
    } else {
        const long long r0 = active ? 2 * cl : 0;
        const bool has1 = active && (r0 + 1 < a.outer);
        p0 = u + r0 * N;
        p1 = has1 ? p0 + N : nullptr;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = t + e * T;
            x[e].x = active ? p0[idx] : R(0);
            x[e].y = has1 ? p1[idx] : R(0);
        }
    }
    if (a.jq_in) {
        const R E0 = R(a.jq_in_E), om = R(a.jq_in_1mE);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            x[e].x = jq_flow(x[e].x, E0, om);
            x[e].y = jq_flow(x[e].y, E0, om);
        }
    }

    // ---- e^{tau/2 C} ------------------------------------------------------
    line_fft<R, N, E, false>(x, t, tw, ex);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const R s = __ldg(eC + t + e * T);
        x[e].x *= s;
        x[e].y *= s;
    }
    line_fft<R, N, E, true>(x, t, tw, ex);
    // ---- e^{tau S} = Theta^{-1} F^{-1} e^{tau Lambda_S} F Theta -------------
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = cmul(x[e], ldg_c2(twist + t + e * T));
    line_fft<R, N, E, false>(x, t, tw, ex);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const R s = __ldg(eS + t + e * T);
        x[e].x *= s;
        x[e].y *= s;
    }
    line_fft<R, N, E, true>(x, t, tw, ex);
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = cmulc(x[e], ldg_c2(twist + t + e * T));
    // ---- e^{tau/2 C} ------------------------------------------------------
    line_fft<R, N, E, false>(x, t, tw, ex);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const R s = __ldg(eC + t + e * T);
        x[e].x *= s;
        x[e].y *= s;
    }
    line_fft<R, N, E, true>(x, t, tw, ex);

    // ---- (J^Q and) store --------------------------------------------------
    if (a.jq_out) {
        const R E0 = R(a.jq_out_E), om = R(a.jq_out_1mE);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            x[e].x = jq_flow(x[e].x, E0, om);
            x[e].y = jq_flow(x[e].y, E0, om);
        }
    }
    if (!active) return;
    if (STRIDED) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = t + e * T;
            V v;
            v.x = x[e].x;
            v.y = x[e].y;
            *reinterpret_cast<V*>(p0 + idx * stride) = v;
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = t + e * T;
            p0[idx] = x[e].x;
            if (p1) p1[idx] = x[e].y;
        }
    }
}

// Elements per thread: 8 for most lengths (radix-8 passes), 16 from N = 2048.
template <int N>
constexpr int elems_per_thread() {
    return N >= 2048 ? 16 : (N < 8 ? N : 8);
}

template <typename R, int N, int LPC, bool STRIDED>
cudaError_t launch_cfg(const PassArgs& a, cudaStream_t s) {
    constexpr int E = elems_per_thread<N>();
    constexpr int T = N / E;
    using Ex = PadExchange<R, N, LPC, STRIDED>;
    const size_t smem = sizeof(C2<R>) * (size_t)Ex::elems();
    auto kern = axis_pass_kernel<R, N, E, LPC, STRIDED>;
    static bool configured = false;
    if (!configured) {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
        if (err != cudaSuccess) return err;
        configured = true;
    }
    const long long grid = (a.clines + LPC - 1) / LPC;
    if (grid <= 0) return cudaSuccess;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
    kern<<<(unsigned)grid, LPC * T, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename R, int N>
cudaError_t launch_n(const PassArgs& a, cudaStream_t s) {
    constexpr int E = elems_per_thread<N>();
    constexpr int T = N / E;
    // Strided passes: at least 32 bytes of each row per CTA (one sector);
    // both mappings aim at about 256 threads per CTA.
    // (Lines of 2048+ points keep 256 threads per CTA and take one line pair.)
    constexpr int MIN_S = (T >= 256) ? 1 : 32 / (2 * (int)sizeof(R));
    constexpr int LPC_S = (256 / T) > MIN_S ? (256 / T) : MIN_S;
    constexpr int LPC_C = (256 / T) > 1 ? (256 / T) : 1;
    if (a.inner > 1) return launch_cfg<R, N, LPC_S, true>(a, s);
    return launch_cfg<R, N, LPC_C, false>(a, s);
}

template <typename R>
cudaError_t launch_pass_any(int N, const PassArgs& a, cudaStream_t s) {
    switch (N) {
        case 4: return launch_n<R, 4>(a, s);
        case 8: return launch_n<R, 8>(a, s);
        case 16: return launch_n<R, 16>(a, s);
        case 32: return launch_n<R, 32>(a, s);
        case 64: return launch_n<R, 64>(a, s);
        case 128: return launch_n<R, 128>(a, s);
        case 256: return launch_n<R, 256>(a, s);
        case 512: return launch_n<R, 512>(a, s);
        case 1024: return launch_n<R, 1024>(a, s);
        case 2048: return launch_n<R, 2048>(a, s);
        case 4096: return launch_n<R, 4096>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sfac
