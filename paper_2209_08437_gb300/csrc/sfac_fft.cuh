// sfac_fft.cuh - device building blocks of the fused axis passes: complex
// arithmetic, small in-register DFTs and a register-resident Stockham FFT.
//
// The linear flow of the two-level scheme applies, along every grid line of an
// axis, e^{tau/2 C} e^{tau S} e^{tau/2 C} with C circulant and S skew-circulant
// (eq. (hatv), Sec. 2.2). Remark 1 diagonalises both with the Fourier matrix:
// C = F^* Lambda_C F and S = Theta^{-1} F^* Lambda_S F Theta with the twist
// Theta = diag(e^{i pi k / n}). So each factor is FFT -> diagonal multiply ->
// inverse FFT, and the S factor sits between the twist and its inverse.
//
// FFT organisation (written for this library). A line of N complex values is
// held by T = N / E threads, thread t holding elements t + e*T, e in [0, E).
// The transform runs as passes of a self-sorting (Stockham) decimation-in-time
// FFT: a pass with current span P and radix RAD does N / RAD butterflies; the
// butterfly i (k = i mod P) reads elements i + r N/RAD, multiplies input r by
// w^{r k} with w = e^{-2 pi i / (P RAD)}, does a RAD-point DFT and writes output
// r to position (i - k) RAD + k + r P. Thread t owns butterflies t + q T, whose
// inputs are exactly its registers, so only the outputs of non-final passes go
// through shared memory. In the final pass P = N / RAD, the outputs land on
// positions t + e T again: the transform starts and ends in the same register
// distribution, in natural order, and the diagonal multiplies that follow need
// no reordering.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sfac {

// A complex value, aligned to its size: shared-memory exchanges and table reads
// then move it as one 64-bit (FP32) or 128-bit (FP64) access.
template <typename R>
struct alignas(2 * sizeof(R)) C2 {
    R x, y;
};

template <typename R>
__device__ __forceinline__ C2<R> cadd(C2<R> a, C2<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R>
__device__ __forceinline__ C2<R> csub(C2<R> a, C2<R> b) { return {a.x - b.x, a.y - b.y}; }
// a * b
template <typename R>
__device__ __forceinline__ C2<R> cmul(C2<R> a, C2<R> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename R>
__device__ __forceinline__ C2<R> cmulc(C2<R> a, C2<R> b) {
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
// a * s for real s
template <typename R>
__device__ __forceinline__ C2<R> cscale(C2<R> a, R s) { return {a.x * s, a.y * s}; }

// SFAC_PACKED_F32 (default on): FP32 complex arithmetic on the packed two-lane
// FP32 instructions of sm_100+ (__fadd2_rn, __fmul2_rn, __ffma2_rn; each lane
// rounds as the scalar _rn operation; a - b is fma(b, -1, a)). The FP32 passes
// are bound by instruction issue; measured side by side on GB300 the packed
// forms made the 256-point 3D passes 3-7% and the 128-point strided passes 11%
// faster, and 3D batches 6-8%.
#ifndef SFAC_PACKED_F32
#define SFAC_PACKED_F32 1
#endif
#if SFAC_PACKED_F32
__device__ __forceinline__ float2 as_f2(C2<float> a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ C2<float> as_c2(float2 v) { return {v.x, v.y}; }
template <>
__device__ __forceinline__ C2<float> cadd<float>(C2<float> a, C2<float> b) {
    return as_c2(__fadd2_rn(as_f2(a), as_f2(b)));
}
template <>
__device__ __forceinline__ C2<float> csub<float>(C2<float> a, C2<float> b) {
    return as_c2(__ffma2_rn(as_f2(b), make_float2(-1.f, -1.f), as_f2(a)));
}
// a * b = a * b.x + (-a.y, a.x) * b.y
template <>
__device__ __forceinline__ C2<float> cmul<float>(C2<float> a, C2<float> b) {
    const float2 t = __fmul2_rn(as_f2(a), make_float2(b.x, b.x));
    return as_c2(__ffma2_rn(make_float2(-a.y, a.x), make_float2(b.y, b.y), t));
}
// a * conj(b) = a * b.x + (a.y, -a.x) * b.y
template <>
__device__ __forceinline__ C2<float> cmulc<float>(C2<float> a, C2<float> b) {
    const float2 t = __fmul2_rn(as_f2(a), make_float2(b.x, b.x));
    return as_c2(__ffma2_rn(make_float2(a.y, -a.x), make_float2(b.y, b.y), t));
}
template <>
__device__ __forceinline__ C2<float> cscale<float>(C2<float> a, float s) {
    return as_c2(__fmul2_rn(as_f2(a), make_float2(s, s)));
}
#endif

// cos(2 pi q / 32) for q = 1 .. 7 to 21 digits (sin(2 pi q/32) = cos(2 pi (8-q)/32)).
#define SFAC_C32_1 0.980785280403230449126
#define SFAC_C32_2 0.923879532511286756128
#define SFAC_C32_3 0.831469612302545237079
#define SFAC_C32_4 0.707106781186547524401
#define SFAC_C32_5 0.555570233019602224743
#define SFAC_C32_6 0.382683432365089771728
#define SFAC_C32_7 0.195090322016128267848

// cos(2 pi q / 32) for q in [0, 8].
template <typename R>
__device__ __forceinline__ R cos32(int q) {
    switch (q) {
        case 0: return R(1);
        case 1: return R(SFAC_C32_1);
        case 2: return R(SFAC_C32_2);
        case 3: return R(SFAC_C32_3);
        case 4: return R(SFAC_C32_4);
        case 5: return R(SFAC_C32_5);
        case 6: return R(SFAC_C32_6);
        case 7: return R(SFAC_C32_7);
        default: return R(0);
    }
}

// v * e^{-+ 2 pi i q / 32} (forward: minus sign; INV: plus sign), q in [0, 16).
// q is a compile-time constant after unrolling, so the branches fold away and
// the multiplications by 1, -i and (1 -+ i)/sqrt 2 cost no general complex product.
template <typename R, bool INV>
__device__ __forceinline__ C2<R> rot32(C2<R> v, int q) {
    if (q == 0) return v;
    if (q == 8) return INV ? C2<R>{-v.y, v.x} : C2<R>{v.y, -v.x};
    const R r2 = R(SFAC_C32_4);
    if (q == 4) return INV ? C2<R>{r2 * (v.x - v.y), r2 * (v.x + v.y)}
                           : C2<R>{r2 * (v.x + v.y), r2 * (v.y - v.x)};
    if (q == 12) return INV ? C2<R>{-r2 * (v.x + v.y), r2 * (v.x - v.y)}
                            : C2<R>{r2 * (v.y - v.x), -r2 * (v.x + v.y)};
    // cos and sin of 2 pi q / 32
    const R co = q < 8 ? cos32<R>(q) : -cos32<R>(16 - q);
    const R si = q < 8 ? cos32<R>(8 - q) : cos32<R>(q - 8);
    return INV ? cmul(v, C2<R>{co, si}) : cmulc(v, C2<R>{co, si});
}

// In-register M-point DFT (M = 1, 2, 4, ..., 32), natural order in and out:
// y_s = sum_r x_r e^{-+2 pi i r s / M}. Radix-2 decimation in time.
template <typename R, int M, bool INV>
struct Dft {
    static __device__ __forceinline__ void run(C2<R>* x) {
        C2<R> ev[M / 2], od[M / 2];
#pragma unroll
        for (int i = 0; i < M / 2; ++i) {
            ev[i] = x[2 * i];
            od[i] = x[2 * i + 1];
        }
        Dft<R, M / 2, INV>::run(ev);
        Dft<R, M / 2, INV>::run(od);
#pragma unroll
        for (int s = 0; s < M / 2; ++s) {
            const C2<R> w = rot32<R, INV>(od[s], s * (32 / M));
            x[s] = cadd(ev[s], w);
            x[s + M / 2] = csub(ev[s], w);
        }
    }
};
template <typename R, bool INV>
struct Dft<R, 1, INV> {
    static __device__ __forceinline__ void run(C2<R>*) {}
};

// One Stockham pass (span P) and, recursively, the ones after it.
// tw[m] = e^{-2 pi i m / N}, m in [0, N).
template <typename R, int N, int E, int P, bool INV>
struct FftPass {
    static constexpr int RAD = (P * E <= N) ? E : (N / P);
    static constexpr bool LAST = (P * RAD == N);
    static constexpr int T = N / E;
    static constexpr int Q = E / RAD;
    static_assert(RAD >= 2 && (RAD & (RAD - 1)) == 0 && RAD <= 32, "radix");

    template <class Ex>
    static __device__ __forceinline__ void run(C2<R> (&x)[E], int t, const C2<R>* __restrict__ tw,
                                               const Ex& ex) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int i = t + q * T;
            const int k = i & (P - 1);
            C2<R> a[RAD];
#pragma unroll
            for (int r = 0; r < RAD; ++r) a[r] = x[q + r * Q];
            if constexpr (P > 1) {
#pragma unroll
                for (int r = 1; r < RAD; ++r) {
                    const C2<R> w = tw[r * k * (N / (P * RAD))];
                    a[r] = INV ? cmulc(a[r], w) : cmul(a[r], w);
                }
            }
            Dft<R, RAD, INV>::run(a);
            if constexpr (LAST) {
#pragma unroll
                for (int r = 0; r < RAD; ++r) x[q + r * Q] = a[r];
            } else {
                const int j = (i - k) * RAD + k;
#pragma unroll
                for (int r = 0; r < RAD; ++r) ex.put(j + r * P, a[r]);
            }
        }
        if constexpr (!LAST) {
            Ex::sync();
#pragma unroll
            for (int e = 0; e < E; ++e) x[e] = ex.get(t + e * T);
            Ex::sync();
            FftPass<R, N, E, P * RAD, INV>::run(x, t, tw, ex);
        }
    }
};

// Unnormalised FFT of one line held as described above (INV: inverse, no 1/N).
template <typename R, int N, int E, bool INV, class Ex>
__device__ __forceinline__ void line_fft(C2<R> (&x)[E], int t, const C2<R>* __restrict__ tw,
                                         const Ex& ex) {
    FftPass<R, N, E, 1, INV>::run(x, t, tw, ex);
}

}  // namespace sfac
