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

#if SFAC_PACKED_F32
// FP32 butterfly a = e + w, b = e - w with w = v e^{-+2 pi i q/32}, q not 0 or
// 8 (compile-time after unrolling). With c, s the cosine and sine of
// 2 pi q / 32, w = k u where either k = c and u = (v.x +- rho v.y, v.y -+ rho v.x),
// rho = s / c, or k = s and u = (rho' v.x +- v.y, rho' v.y -+ v.x), rho' = c / s,
// whichever ratio is at most 1 in size: u takes two scalar multiply-adds and
// the factor k rides in the butterfly's two packed multiply-adds, e +- k u.
// That is two operations less than forming w on its own, one rounding less,
// and no data movement between the lanes.
template <bool INV>
__device__ __forceinline__ void rot_butterfly(C2<float> e, C2<float> v, int q, C2<float>& a, C2<float>& b) {
    const float co = q < 8 ? (float)cos32<double>(q) : -(float)cos32<double>(16 - q);
    const float si = q < 8 ? (float)cos32<double>(8 - q) : (float)cos32<double>(q - 8);
    const bool by_cos = (co < 0 ? -co : co) >= (si < 0 ? -si : si);
    float k;
    C2<float> u;
    if (by_cos) {
        const float r = (float)((q < 8 ? cos32<double>(8 - q) : cos32<double>(q - 8)) /
                                (q < 8 ? cos32<double>(q) : -cos32<double>(16 - q)));
        k = co;
        u = INV ? C2<float>{fmaf(-r, v.y, v.x), fmaf(r, v.x, v.y)} : C2<float>{fmaf(r, v.y, v.x), fmaf(-r, v.x, v.y)};
    } else {
        const float r = (float)((q < 8 ? cos32<double>(q) : -cos32<double>(16 - q)) /
                                (q < 8 ? cos32<double>(8 - q) : cos32<double>(q - 8)));
        k = si;
        u = INV ? C2<float>{fmaf(r, v.x, -v.y), fmaf(r, v.y, v.x)} : C2<float>{fmaf(r, v.x, v.y), fmaf(r, v.y, -v.x)};
    }
    a = as_c2(__ffma2_rn(as_f2(u), make_float2(k, k), as_f2(e)));
    b = as_c2(__ffma2_rn(as_f2(u), make_float2(-k, -k), as_f2(e)));
}
#endif

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
#if SFAC_PACKED_F32
            if constexpr (sizeof(R) == 4) {
                const int q = s * (32 / M);
                if (q != 0 && q != 8) {
                    rot_butterfly<INV>(ev[s], od[s], q, x[s], x[s + M / 2]);
                    continue;
                }
            }
#endif
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

// Twiddle sources of the Stockham passes. get<P, RAD>(q, t, k, w) fills w[r],
// r in [1, RAD), with e^{-2 pi i r k / (P RAD)} for butterfly k = (t + q T)
// mod P of the pass of span P (w[0] is left as it is).
//
// TwTable reads them from the length-N table tw[m] = e^{-2 pi i m / N}.
template <typename R, int N>
struct TwTable {
    const C2<R>* __restrict__ tw;
    template <int P, int RAD>
    __device__ __forceinline__ void get(int, int, int k, C2<R> (&w)[RAD]) const {
#pragma unroll
        for (int r = 1; r < RAD; ++r) w[r] = tw[r * k * (N / (P * RAD))];
    }
};

// TwRows (FP32) reads them from rows laid out per pass and thread: for every
// pass of span P > 1, for q in [0, Q) and t in [0, T), one row holding the RAD
// factors of butterfly (t + q T) mod P (entry 0 is 1), padded to
// tw_row_stride(RAD) values. A thread loads its row with 16-byte loads (two
// factors each), and the rows of the 8 lanes of a quarter-warp start in
// distinct 16-byte bank groups, so the loads are free of bank conflicts; the
// table-indexed loads of TwTable hit the same bank for r k multiples of 16 and
// were the largest share of shared-memory traffic of the FP32 passes. The
// values are the table's, so results are bit-identical to TwTable's.
__host__ __device__ constexpr int tw_row_stride(int rad) { return rad == 2 ? 2 : rad + 2; }

// Radix of the pass of span P for a line of N points with E values per thread.
__host__ __device__ constexpr int fft_pass_radix(int N, int E, int P) { return (P * E <= N) ? E : (N / P); }

// Complex values of the rows of every pass of span < P_END (P_END = N: all).
__host__ __device__ constexpr int tw_rows_elems(int N, int E, int P_END) {
    int total = 0;
    for (int P = fft_pass_radix(N, E, 1); P < N && P < P_END; P *= fft_pass_radix(N, E, P)) {
        const int rad = fft_pass_radix(N, E, P);
        total += (E / rad) * (N / E) * tw_row_stride(rad);
    }
    return total;
}

template <int N, int E>
struct TwRows {
    const C2<float>* __restrict__ rows;
    template <int P, int RAD>
    __device__ __forceinline__ void get(int q, int t, int, C2<float> (&w)[RAD]) const {
        constexpr int T = N / E, S = tw_row_stride(RAD);
        const float4* row = reinterpret_cast<const float4*>(rows + tw_rows_elems(N, E, P) + (q * T + t) * S);
#pragma unroll
        for (int h = 0; h < RAD / 2; ++h) {
            const float4 v = row[h];
            if (h > 0) w[2 * h] = {v.x, v.y};
            w[2 * h + 1] = {v.z, v.w};
        }
    }
};

// Fill the rows of TwRows<N, E> from the table tw (threads tid of nth share the work).
template <int N, int E>
__device__ __forceinline__ void build_tw_rows(C2<float>* rows, const C2<float>* tw, int tid, int nth) {
    constexpr int T = N / E;
    for (int P = fft_pass_radix(N, E, 1); P < N; P *= fft_pass_radix(N, E, P)) {
        const int rad = fft_pass_radix(N, E, P), S = tw_row_stride(rad), Q = E / rad;
        C2<float>* base = rows + tw_rows_elems(N, E, P);
        for (int f = tid; f < Q * T * S; f += nth) {
            const int q = f / (T * S), t = (f / S) % T, r = f % S;
            const int k = (t + q * T) & (P - 1);
            base[f] = r < rad ? tw[r * k * (N / (P * rad))] : C2<float>{0.f, 0.f};
        }
    }
}

// One Stockham pass (span P) and, recursively, the ones after it; twiddles
// from `tws` (TwTable or TwRows).
template <typename R, int N, int E, int P, bool INV>
struct FftPass {
    static constexpr int RAD = fft_pass_radix(N, E, P);
    static constexpr bool LAST = (P * RAD == N);
    static constexpr int T = N / E;
    static constexpr int Q = E / RAD;
    static_assert(RAD >= 2 && (RAD & (RAD - 1)) == 0 && RAD <= 32, "radix");

    template <class Ex, class Tw>
    static __device__ __forceinline__ void run(C2<R> (&x)[E], int t, const Tw& tws, const Ex& ex) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int i = t + q * T;
            const int k = i & (P - 1);
            C2<R> a[RAD];
#pragma unroll
            for (int r = 0; r < RAD; ++r) a[r] = x[q + r * Q];
            if constexpr (P > 1) {
                C2<R> w[RAD];
                tws.template get<P, RAD>(q, t, k, w);
#pragma unroll
                for (int r = 1; r < RAD; ++r) a[r] = INV ? cmulc(a[r], w[r]) : cmul(a[r], w[r]);
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
            FftPass<R, N, E, P * RAD, INV>::run(x, t, tws, ex);
        }
    }
};

// Unnormalised FFT of one line held as described above (INV: inverse, no 1/N),
// twiddles from the table tw[m] = e^{-2 pi i m / N}.
template <typename R, int N, int E, bool INV, class Ex>
__device__ __forceinline__ void line_fft(C2<R> (&x)[E], int t, const C2<R>* __restrict__ tw,
                                         const Ex& ex) {
    FftPass<R, N, E, 1, INV>::run(x, t, TwTable<R, N>{tw}, ex);
}

// The same with the twiddles from a source object (TwTable or TwRows).
template <typename R, int N, int E, bool INV, class Ex, class Tw>
__device__ __forceinline__ void line_fft_tw(C2<R> (&x)[E], int t, const Tw& tws, const Ex& ex) {
    FftPass<R, N, E, 1, INV>::run(x, t, tws, ex);
}

// ---------------------------------------------------------------------------
// FP64 passes with ratio twiddles (radix 8/4/2 for lines of up to 2048 points,
// radix 16 for 4096).
//
// The FP64 passes are bound by the FP64 pipe, so what counts is the number of
// FP64 instructions. A twiddle w = c + i s is stored as c and the ratio
// rho = s / c: w a = c t with t = (1 + i rho) a, two FMAs instead of the four
// instructions of a complex product. The scale c is not applied on its own: it
// rides in the FMA of the butterfly that consumes the product
// (u + c t = fma(c, t, u)). Where both operands of a butterfly carry a scale
// (c_a t_a +- c_b t_b), the butterfly computes t_a +- (c_b / c_a) t_b and hands
// c_a on to the next butterfly. This is the same arithmetic rewritten around
// FMAs; each rounding stays relative to the values it rounds, also for large
// rho (c near 0 multiplies the large t back down in one FMA). Twiddles stored
// as a cosine and a ratio so that products fold into multiply-adds are the
// idea of FMA-oriented FFT kernels (Linzer and Feig, IEEE Trans. Signal
// Process. 1993; Goedecker, SIAM J. Sci. Comput. 1997); the scale bookkeeping
// through the three radix-2 stages of the radix-8 butterfly is this file's.
//
// Records, per pass of span P > 1 and radix RAD, one per k in [0, P), in pass
// order; c_r + i s_r = e^{-2 pi i r k / (P RAD)}, rho_r = s_r / c_r:
//   RAD 8 (16 values): rho_1..rho_7, c_4, c_6/c_2, c_5/c_1, c_7/c_3, c_3/c_1,
//                      c_2, c_1, c_1/sqrt 2, 0
//   RAD 4 (8 values):  rho_1, rho_2, rho_3, c_2, c_3/c_1, c_1, 0, 0
//   RAD 2 (2 values):  rho_1, c_1
//   RAD 16 (36 values): as DftRatio16 below describes
// Pass P = 1 has no twiddles and no records.

__device__ __forceinline__ C2<double> cfma_d(double s, C2<double> u, C2<double> e) {
    return {fma(s, u.x, e.x), fma(s, u.y, e.y)};
}
// (1 -+ i rho) a (forward: w = c (1 + i rho); inverse: conj(w) = c (1 - i rho))
template <bool INV>
__device__ __forceinline__ C2<double> ratio_mul(C2<double> a, double rho) {
    return INV ? C2<double>{fma(rho, a.y, a.x), fma(-rho, a.x, a.y)}
               : C2<double>{fma(-rho, a.y, a.x), fma(rho, a.x, a.y)};
}
// v e^{-+ i pi / 2}
template <bool INV>
__device__ __forceinline__ C2<double> rot_quarter(C2<double> v) {
    return INV ? C2<double>{-v.y, v.x} : C2<double>{v.y, -v.x};
}
// v e^{-+ i pi / 4} = u / sqrt 2 and v e^{-+ 3 i pi / 4} = u / sqrt 2: the u
template <bool INV>
__device__ __forceinline__ C2<double> rot_eighth_u(C2<double> v) {
    return INV ? C2<double>{v.x - v.y, v.x + v.y} : C2<double>{v.x + v.y, v.y - v.x};
}
template <bool INV>
__device__ __forceinline__ C2<double> rot_3eighth_u(C2<double> v) {
    return INV ? C2<double>{-(v.x + v.y), v.x - v.y} : C2<double>{v.y - v.x, -(v.x + v.y)};
}

__device__ __forceinline__ double2 ld_rec2(const double* p) { return *reinterpret_cast<const double2*>(p); }

// a_r <- sum_r w_r a_r e^{-+2 pi i r s / 8} with the twiddles of record p: the
// radix-2 decimation of Dft<double, 8>, scales carried as described above.
template <bool INV>
__device__ __forceinline__ void dft8_ratio(C2<double> (&a)[8], const double* __restrict__ p) {
    const double2 p01 = ld_rec2(p), p23 = ld_rec2(p + 2), p45 = ld_rec2(p + 4), p67 = ld_rec2(p + 6);
    const double2 p89 = ld_rec2(p + 8), pab = ld_rec2(p + 10), pcd = ld_rec2(p + 12), pef = ld_rec2(p + 14);
    const C2<double> t1 = ratio_mul<INV>(a[1], p01.x), t2 = ratio_mul<INV>(a[2], p01.y);
    const C2<double> t3 = ratio_mul<INV>(a[3], p23.x), t4 = ratio_mul<INV>(a[4], p23.y);
    const C2<double> t5 = ratio_mul<INV>(a[5], p45.x), t6 = ratio_mul<INV>(a[6], p45.y);
    const C2<double> t7 = ratio_mul<INV>(a[7], p67.x);
    const double c4 = p67.y, q62 = p89.x, q51 = p89.y, q73 = pab.x, q31 = pab.y;
    const double c2 = pcd.x, c1 = pcd.y, c1r = pef.x;
    // first stage: pairs (r, r + 4); the pairs other than (0, 4) keep a scale
    const C2<double> l0p = cfma_d(c4, t4, a[0]), l0m = cfma_d(-c4, t4, a[0]);
    const C2<double> l2p = cfma_d(q62, t6, t2), l2m = cfma_d(-q62, t6, t2);  // x c_2
    const C2<double> l1p = cfma_d(q51, t5, t1), l1m = cfma_d(-q51, t5, t1);  // x c_1
    const C2<double> l3p = cfma_d(q73, t7, t3), l3m = cfma_d(-q73, t7, t3);  // x c_3
    // second stage, even half: scale 1
    const C2<double> r2 = rot_quarter<INV>(l2m);
    const C2<double> e0 = cfma_d(c2, l2p, l0p), e2 = cfma_d(-c2, l2p, l0p);
    const C2<double> e1 = cfma_d(c2, r2, l0m), e3 = cfma_d(-c2, r2, l0m);
    // second stage, odd half: x c_1
    const C2<double> r3 = rot_quarter<INV>(l3m);
    const C2<double> o0 = cfma_d(q31, l3p, l1p), o2 = cfma_d(-q31, l3p, l1p);
    const C2<double> o1 = cfma_d(q31, r3, l1m), o3 = cfma_d(-q31, r3, l1m);
    // third stage
    a[0] = cfma_d(c1, o0, e0);
    a[4] = cfma_d(-c1, o0, e0);
    const C2<double> u1 = rot_eighth_u<INV>(o1);
    a[1] = cfma_d(c1r, u1, e1);
    a[5] = cfma_d(-c1r, u1, e1);
    const C2<double> v2 = rot_quarter<INV>(o2);
    a[2] = cfma_d(c1, v2, e2);
    a[6] = cfma_d(-c1, v2, e2);
    const C2<double> u3 = rot_3eighth_u<INV>(o3);
    a[3] = cfma_d(c1r, u3, e3);
    a[7] = cfma_d(-c1r, u3, e3);
}

template <bool INV>
__device__ __forceinline__ void dft4_ratio(C2<double> (&a)[4], const double* __restrict__ p) {
    const double2 p01 = ld_rec2(p), p23 = ld_rec2(p + 2), p45 = ld_rec2(p + 4);
    const C2<double> t1 = ratio_mul<INV>(a[1], p01.x), t2 = ratio_mul<INV>(a[2], p01.y);
    const C2<double> t3 = ratio_mul<INV>(a[3], p23.x);
    const double c2 = p23.y, q31 = p45.x, c1 = p45.y;
    const C2<double> ep = cfma_d(c2, t2, a[0]), em = cfma_d(-c2, t2, a[0]);
    const C2<double> op = cfma_d(q31, t3, t1), om = cfma_d(-q31, t3, t1);  // x c_1
    const C2<double> r = rot_quarter<INV>(om);
    a[0] = cfma_d(c1, op, ep);
    a[2] = cfma_d(-c1, op, ep);
    a[1] = cfma_d(c1, r, em);
    a[3] = cfma_d(-c1, r, em);
}

template <bool INV>
__device__ __forceinline__ void dft2_ratio(C2<double> (&a)[2], const double* __restrict__ p) {
    const double2 rc = ld_rec2(p);
    const C2<double> t1 = ratio_mul<INV>(a[1], rc.x);
    const C2<double> a0 = a[0];
    a[0] = cfma_d(rc.y, t1, a0);
    a[1] = cfma_d(-rc.y, t1, a0);
}

// Radix 16 (FP64 lines of 4096 points, 16 values a thread). The same
// bookkeeping, written once for every level of the radix-2 decimation in time
// (Dft above): the node over the inputs R0 + S j (j < 16/S) returns its DFT
// scaled by 1/c_R0; it combines its even half (scale c_R0) and its odd half
// (scale c_{R0+S}) as u +- g W^s v with g = c_{R0+S}/c_R0 from the record.
// W^s = 1 and -+i take g as it is; W^s = e^{-+i pi/4}, e^{-+3i pi/4} are
// u/sqrt 2 and take h = g/sqrt 2; the other angles of the 16-point node
// (odd multiples of pi/8) are k w with w = v turned and divided by
// k = +-cos(pi/8) in two multiply-adds (the larger of the cosine and the sine,
// ratio tan(pi/8) = sqrt 2 - 1 to the other), and take g cos(pi/8).
// Record (36 doubles): rho_1..rho_15; g of node (S, R0) at 15 + S - 1 + R0 for
// S = 1, 2, 4, 8; h of the nodes (1, 0), (2, 0), (2, 1) at 30..32;
// g(1, 0) cos(pi/8) at 33; two doubles of padding.
constexpr double kTanPi8 = 0.414213562373095048801688724209698;  // sqrt 2 - 1

// v e^{-+ 2 pi i q / 32} = k w for q in {2, 6, 10, 14}, |k| = cos(pi/8):
// returns w; *neg says k < 0 (q = 14).
template <bool INV>
__device__ __forceinline__ C2<double> turn_pi8(C2<double> v, int q, bool* neg) {
    *neg = (q == 14);
    if (q == 2 || q == 14) {
        // k = cos(2 pi q/32); ratio r = sin/cos = +tan(pi/8) (q = 2), -tan(pi/8) (q = 14)
        const double r = q == 2 ? kTanPi8 : -kTanPi8;
        return INV ? C2<double>{fma(-r, v.y, v.x), fma(r, v.x, v.y)} : C2<double>{fma(r, v.y, v.x), fma(-r, v.x, v.y)};
    }
    // q = 6, 10: k = sin(2 pi q/32) = cos(pi/8); ratio r = cos/sin = +tan(pi/8) (6), -tan(pi/8) (10)
    const double r = q == 6 ? kTanPi8 : -kTanPi8;
    return INV ? C2<double>{fma(r, v.x, -v.y), fma(r, v.y, v.x)} : C2<double>{fma(r, v.x, v.y), fma(r, v.y, -v.x)};
}

template <int M, int S, int R0, bool INV>
struct DftRatio16 {
    // x[j]: input R0 + S j carrying the scale c_{R0 + S j} (leaves already
    // turned by 1 + i rho); on return the node's DFT with scale c_R0
    static __device__ __forceinline__ void run(C2<double>* x, const double* __restrict__ p) {
        C2<double> ev[M / 2], od[M / 2];
#pragma unroll
        for (int j = 0; j < M / 2; ++j) {
            ev[j] = x[2 * j];
            od[j] = x[2 * j + 1];
        }
        DftRatio16<M / 2, 2 * S, R0, INV>::run(ev, p);
        DftRatio16<M / 2, 2 * S, R0 + S, INV>::run(od, p);
        const double g = p[15 + S - 1 + R0];
#pragma unroll
        for (int s = 0; s < M / 2; ++s) {
            const int q = s * (32 / M);
            if (q == 0) {
                x[s] = cfma_d(g, od[s], ev[s]);
                x[s + M / 2] = cfma_d(-g, od[s], ev[s]);
            } else if (q == 8) {
                const C2<double> w = rot_quarter<INV>(od[s]);
                x[s] = cfma_d(g, w, ev[s]);
                x[s + M / 2] = cfma_d(-g, w, ev[s]);
            } else if (q == 4 || q == 12) {
                const double h = p[30 + (S - 1) + R0];
                const C2<double> w = q == 4 ? rot_eighth_u<INV>(od[s]) : rot_3eighth_u<INV>(od[s]);
                x[s] = cfma_d(h, w, ev[s]);
                x[s + M / 2] = cfma_d(-h, w, ev[s]);
            } else {
                const double gk = p[33];
                bool neg;
                const C2<double> w = turn_pi8<INV>(od[s], q, &neg);
                x[s] = cfma_d(neg ? -gk : gk, w, ev[s]);
                x[s + M / 2] = cfma_d(neg ? gk : -gk, w, ev[s]);
            }
        }
    }
};
template <int S, int R0, bool INV>
struct DftRatio16<1, S, R0, INV> {
    static __device__ __forceinline__ void run(C2<double>*, const double*) {}
};

// a_r <- sum_r w_r a_r e^{-+2 pi i r s / 16} with the twiddles of record p.
template <bool INV>
__device__ __forceinline__ void dft16_ratio(C2<double> (&a)[16], const double* __restrict__ p) {
#pragma unroll
    for (int r = 1; r < 16; ++r) a[r] = ratio_mul<INV>(a[r], p[r - 1]);
    DftRatio16<16, 1, 0, INV>::run(a, p);
}

// Doubles per record of a radix-RAD pass.
constexpr int ratio_record(int rad) { return rad == 16 ? 36 : (rad == 8 ? 16 : (rad == 4 ? 8 : 2)); }

// The Stockham passes of FftPass with ratio twiddles (double, radix 2/4/8/16).
// OFF: offset of this pass's records in the table.
template <int N, int E, int P, int OFF, bool INV>
struct FftPassRatio {
    static constexpr int RAD = (P * E <= N) ? E : (N / P);
    static constexpr bool LAST = (P * RAD == N);
    static constexpr int T = N / E;
    static constexpr int Q = E / RAD;
    static constexpr int REC = ratio_record(RAD);
    static constexpr int NEXT_OFF = OFF + (P > 1 ? P * REC : 0);
    static_assert(RAD == 2 || RAD == 4 || RAD == 8 || RAD == 16, "ratio twiddles: radix 2, 4, 8 or 16");

    template <class Ex>
    static __device__ __forceinline__ void run(C2<double> (&x)[E], int t, const double* __restrict__ rt,
                                               const Ex& ex) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int i = t + q * T;
            const int k = i & (P - 1);
            C2<double> a[RAD];
#pragma unroll
            for (int r = 0; r < RAD; ++r) a[r] = x[q + r * Q];
            if constexpr (P == 1) {
                Dft<double, RAD, INV>::run(a);
            } else {
                const double* rec = rt + OFF + k * REC;
                if constexpr (RAD == 16) dft16_ratio<INV>(a, rec);
                else if constexpr (RAD == 8) dft8_ratio<INV>(a, rec);
                else if constexpr (RAD == 4) dft4_ratio<INV>(a, rec);
                else dft2_ratio<INV>(a, rec);
            }
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
            FftPassRatio<N, E, P * RAD, NEXT_OFF, INV>::run(x, t, rt, ex);
        }
    }
};

// Unnormalised FFT of one FP64 line with ratio twiddles (table `rt`, records as
// described above for this N and E).
template <int N, int E, bool INV, class Ex>
__device__ __forceinline__ void line_fft_ratio(C2<double> (&x)[E], int t, const double* __restrict__ rt,
                                               const Ex& ex) {
    FftPassRatio<N, E, 1, 0, INV>::run(x, t, rt, ex);
}

}  // namespace sfac
