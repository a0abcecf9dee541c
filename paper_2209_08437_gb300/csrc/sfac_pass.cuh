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
//
// Kernel shapes that share that chain:
//  - axis_pass_kernel: a line's T = N/E threads may span several warps, so the
//    exchanges synchronise the CTA (FP64 at every N; FP32 below 32 and at
//    1024 points);
//  - axis_pass_cta_rows_kernel: the same lines in persistent CTAs that keep
//    the tables and twiddle rows in shared memory (FP32, 2048 and 4096 points);
//  - axis_pass_warp_kernel: 16 values per thread, so a line of N <= 512 points
//    lives inside one warp (with 32/T lines per warp); the exchanges need only
//    warp-level synchronisation; persistent CTAs keep the tables in shared
//    memory (FP32, 32 <= N <= 512);
//  - the TMA-staged kernel of sfac_pass_staged_f32.cu (FP32 strided axes) and
//    the batch kernel of sfac_batch.cuh run the same warp-local lines.
// The FP32 chain is the increment form, rolled for N <= SFAC_ROLLED_MAX_N.
// The FP64 CTA kernel runs its FFTs on ratio twiddles (FftPassRatio in
// sfac_fft.cuh, records in PassArgs::rtwid); the batch kernel uses the complex
// twiddle table.
#pragma once

#include <atomic>

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

// Increment of J^Q for the FP32 passes: with q = (1 - E)(1 - v^2) the
// flow is v / sqrt(1 - q) = v + v q / (s (1 + s)), s = sqrt(1 - q); this returns
// the added term v q / (s (1 + s)) = v q r / (1 + s) with r = 1/s. The term is
// about tau |v| at most, so the few-ulp reciprocal square root and fast divide
// used here change the result by far less than the final rounding of x0 + d.
// (1 - q >= E > 0, so both are in range.)
__device__ __forceinline__ float jq_increment(float v, float omE) {
    const float q = omE * fmaf(-v, v, 1.f);  // (1 - E)(1 - v^2), 1 - v^2 rounded once
    const float r = rsqrtf(1.f - q);
    const float s = (1.f - q) * r;
    return __fdividef(v * q * r, 1.f + s);
}

// Table reads. Tables may sit in global memory or, in the persistent kernels,
// in shared memory: plain loads serve both (the address space is inferred
// where the pointer is known).
template <typename R>
__device__ __forceinline__ C2<R> ldg_c2(const C2<R>* p) {
    using V = typename Vec2T<R>::type;
    const V v = *reinterpret_cast<const V*>(p);
    return {v.x, v.y};
}

template <typename R, int E>
__device__ __forceinline__ void jq_all(C2<R> (&x)[E], double E0d, double omd) {
    const R E0 = R(E0d), om = R(omd);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        x[e].x = jq_flow(x[e].x, E0, om);
        x[e].y = jq_flow(x[e].y, E0, om);
    }
}

// x <- F^{-1} diag(m) F x for the line held in x (m includes the 1/N).
template <typename R, int N, int E, class Ex>
__device__ __forceinline__ void apply_spectral(C2<R> (&x)[E], int t, const C2<R>* __restrict__ tw,
                                               const Ex& ex, const R* __restrict__ m) {
    constexpr int T = N / E;
    line_fft<R, N, E, false>(x, t, tw, ex);
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = cscale(x[e], m[t + e * T]);
    line_fft<R, N, E, true>(x, t, tw, ex);
}

// The same with the twiddles from a source object (TwTable or TwRows).
template <typename R, int N, int E, class Ex, class Tw>
__device__ __forceinline__ void apply_spectral_tw(C2<R> (&x)[E], int t, const Tw& tws, const Ex& ex,
                                                  const R* __restrict__ m) {
    constexpr int T = N / E;
    line_fft_tw<R, N, E, false>(x, t, tws, ex);
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = cscale(x[e], m[t + e * T]);
    line_fft_tw<R, N, E, true>(x, t, tws, ex);
}

// Twiddle source of the FP32 passes: the per-thread rows a.twrows (ROWS) or
// the table a.twid.
template <typename R, int N, int E, bool ROWS>
struct TwOf {
    static __device__ __forceinline__ TwTable<R, N> make(const PassArgs& a) {
        return TwTable<R, N>{static_cast<const C2<R>*>(a.twid)};
    }
};
template <int N, int E>
struct TwOf<float, N, E, true> {
    static __device__ __forceinline__ TwRows<N, E> make(const PassArgs& a) {
        return TwRows<N, E>{static_cast<const C2<float>*>(a.twrows)};
    }
};

// The same with the FFTs on ratio twiddles (FP64, E <= 16; table rt).
template <int N, int E, class Ex>
__device__ __forceinline__ void apply_spectral_ratio(C2<double> (&x)[E], int t, const double* __restrict__ rt,
                                                     const Ex& ex, const double* __restrict__ m) {
    constexpr int T = N / E;
    line_fft_ratio<N, E, false>(x, t, rt, ex);
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = cscale(x[e], m[t + e * T]);
    line_fft_ratio<N, E, true>(x, t, rt, ex);
}

// Twiddle source of the FP64 chain: the complex table, or (RATIO) the
// ratio-twiddle records.
template <typename R, int N, int E, bool RATIO>
struct Spectral {
    const C2<R>* __restrict__ tw;
    const double* __restrict__ rt;
    template <class Ex>
    __device__ __forceinline__ void apply(C2<R> (&x)[E], int t, const Ex& ex, const R* __restrict__ m) const {
        if constexpr (RATIO) apply_spectral_ratio<N, E>(x, t, rt, ex, m);
        else apply_spectral<R, N, E>(x, t, tw, ex, m);
    }
};

// Zero the values at positions >= nmem (the padding of a zero-padded pass).
template <typename R, int N, int E>
__device__ __forceinline__ void zero_tail(C2<R> (&x)[E], int t, int nmem) {
    constexpr int T = N / E;
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (t + e * T >= nmem) x[e] = {R(0), R(0)};
}

// e^{tau/2 C} e^{tau S} e^{tau/2 C} on the line held in x (FP64 passes; the
// tables hold e^{t lambda} / N). PADDED: three zero-padded linear convolutions
// with real multipliers, no twist.
template <typename R, int N, int E, bool PADDED, bool RATIO, class Ex>
__device__ __forceinline__ void two_level_chain(C2<R> (&x)[E], int t, const PassArgs& a, const Ex& ex) {
    constexpr int T = N / E;
    static_assert(!RATIO || (sizeof(R) == 8 && E <= 16), "ratio twiddles: FP64, E <= 16");
    const Spectral<R, N, E, RATIO> sp{static_cast<const C2<R>*>(a.twid), static_cast<const double*>(a.rtwid)};
    if constexpr (PADDED) {
        sp.apply(x, t, ex, static_cast<const R*>(a.eC));
        zero_tail<R, N, E>(x, t, a.nmem);
        sp.apply(x, t, ex, static_cast<const R*>(a.eS));
        zero_tail<R, N, E>(x, t, a.nmem);
        sp.apply(x, t, ex, static_cast<const R*>(a.eC));
        return;
    }
    const C2<R>* __restrict__ twist = static_cast<const C2<R>*>(a.twist);
    // e^{tau/2 C}
    sp.apply(x, t, ex, static_cast<const R*>(a.eC));
    // e^{tau S} = Theta^{-1} F^{-1} e^{tau Lambda_S} F Theta
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = cmul(x[e], ldg_c2(twist + t + e * T));
    sp.apply(x, t, ex, static_cast<const R*>(a.eS));
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = cmulc(x[e], ldg_c2(twist + t + e * T));
    // e^{tau/2 C}
    sp.apply(x, t, ex, static_cast<const R*>(a.eC));
}

// For lines of up to SFAC_ROLLED_MAX_N points the FP32 chain runs rolled: one
// loop over the three factors, and each F^{-1} diag(m) F computed as
// conj(F(conj(m F y))) (m is real), so the kernel holds one forward-FFT body
// instead of six unrolled FFTs, whose code stalled the passes on instruction
// fetch. Longer lines keep the unrolled chain: measured on GB300, rolling made
// the 1024-point CTA kernel and the 512-point batch passes slower and the
// passes of 256 points and less faster (strided 256-point passes by 9%,
// batches of 3D n = 128 instances by 18%).
#ifndef SFAC_ROLLED_MAX_N
#define SFAC_ROLLED_MAX_N 256
#endif

// d += the increments of e^{tau/2 C}, e^{tau S}, e^{tau/2 C} in turn (each
// applied to x0 + d), rolled as described above.
template <typename R, int N, int E, bool PADDED, bool ROWS, class Ex, class X0>
__device__ __forceinline__ void three_factors_rolled(const X0& x0, C2<R> (&d)[E], int t, const PassArgs& a,
                                                     const Ex& ex) {
    constexpr int T = N / E;
    const auto tws = TwOf<R, N, E, ROWS>::make(a);
    const C2<R>* __restrict__ twist = static_cast<const C2<R>*>(a.twist);
    C2<R> y[E];
#pragma unroll 1
    for (int f = 0; f < 3; ++f) {
        const bool skew = !PADDED && f == 1;
        const R* __restrict__ m = static_cast<const R*>(f == 1 ? a.eS : a.eC);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            y[e] = cadd(x0.get(e), d[e]);
            if (skew) y[e] = cmul(y[e], ldg_c2(twist + t + e * T));
        }
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            line_fft_tw<R, N, E, false>(y, t, tws, ex);
            if (h == 0) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const R sc = m[t + e * T];
                    y[e] = {y[e].x * sc, -(y[e].y * sc)};
                }
            }
        }
        // y holds the conjugate of the factor's increment
        if constexpr (PADDED) zero_tail<R, N, E>(y, t, a.nmem);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            C2<R> r = {y[e].x, -y[e].y};
            if (skew) r = cmulc(r, ldg_c2(twist + t + e * T));
            d[e] = cadd(d[e], r);
        }
    }
}

// The whole FP32 pass in increment form. The loaded line x0 is kept as it is
// and every change the pass makes is summed in d:
//   J^Q (load)  d += v q / (s (1 + s))                        (jq_increment)
//   e^{t C}     d += F^{-1} (expm1(t lambda)/N) F (x0 + d)
//   e^{tau S}   d += Theta^{-1} F^{-1} (expm1(tau mu)/N) F Theta (x0 + d)
//   J^Q (store) d += its increment at x0 + d
// and the result x0 + d is rounded once. Each increment is small against x0,
// so its FP32 rounding is too, and the field itself is rounded once per pass
// instead of after every factor. The tables hold expm1(t lambda) / N.
// PADDED: the three factors are zero-padded linear convolutions (no twist) and
// the padding of each increment is zeroed before it is added.
//
// X0 gives x0 element by element (x0.get(e) = element t + e T, see RegX0).
// On return d holds the total increment.
template <typename R, int N, int E, bool PADDED, bool ROWS, class Ex, class X0>
__device__ __forceinline__ void two_level_increment(const X0& x0, C2<R> (&d)[E], int t, const PassArgs& a,
                                                    const Ex& ex) {
    if (a.jq_in) {
        const R om = R(a.jq_in_1mE);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const C2<R> v = x0.get(e);
            d[e] = {jq_increment(v.x, om), jq_increment(v.y, om)};
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) d[e] = {R(0), R(0)};
    }
    if constexpr (N <= SFAC_ROLLED_MAX_N) {
        three_factors_rolled<R, N, E, PADDED, ROWS>(x0, d, t, a, ex);
    } else {
        constexpr int T = N / E;
        const auto tw = TwOf<R, N, E, ROWS>::make(a);
        const C2<R>* __restrict__ twist = static_cast<const C2<R>*>(a.twist);
        const R* __restrict__ eC = static_cast<const R*>(a.eC);
        const R* __restrict__ eS = static_cast<const R*>(a.eS);
        C2<R> y[E];
        // e^{tau/2 C}
#pragma unroll
        for (int e = 0; e < E; ++e) y[e] = cadd(x0.get(e), d[e]);
        apply_spectral_tw<R, N, E>(y, t, tw, ex, eC);
        if constexpr (PADDED) zero_tail<R, N, E>(y, t, a.nmem);
#pragma unroll
        for (int e = 0; e < E; ++e) d[e] = cadd(d[e], y[e]);
        // e^{tau S}
        if constexpr (PADDED) {
#pragma unroll
            for (int e = 0; e < E; ++e) y[e] = cadd(x0.get(e), d[e]);
            apply_spectral_tw<R, N, E>(y, t, tw, ex, eS);
            zero_tail<R, N, E>(y, t, a.nmem);
#pragma unroll
            for (int e = 0; e < E; ++e) d[e] = cadd(d[e], y[e]);
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) y[e] = cmul(cadd(x0.get(e), d[e]), ldg_c2(twist + t + e * T));
            apply_spectral_tw<R, N, E>(y, t, tw, ex, eS);
#pragma unroll
            for (int e = 0; e < E; ++e) d[e] = cadd(d[e], cmulc(y[e], ldg_c2(twist + t + e * T)));
        }
        // e^{tau/2 C}
#pragma unroll
        for (int e = 0; e < E; ++e) y[e] = cadd(x0.get(e), d[e]);
        apply_spectral_tw<R, N, E>(y, t, tw, ex, eC);
        if constexpr (PADDED) zero_tail<R, N, E>(y, t, a.nmem);
#pragma unroll
        for (int e = 0; e < E; ++e) d[e] = cadd(d[e], y[e]);
    }
    if (a.jq_out) {
        const R om = R(a.jq_out_1mE);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const C2<R> w = cadd(x0.get(e), d[e]);
            d[e].x += jq_increment(w.x, om);
            d[e].y += jq_increment(w.y, om);
        }
    }
}

template <typename R, int E>
struct RegX0 {
    const C2<R> (&x)[E];
    __device__ __forceinline__ C2<R> get(int e) const { return x[e]; }
};

template <typename R, int N, int E, bool PADDED, bool ROWS, class Ex>
__device__ __forceinline__ void two_level_pass_incr(C2<R> (&x0)[E], int t, const PassArgs& a, const Ex& ex) {
    C2<R> d[E];
    two_level_increment<R, N, E, PADDED, ROWS>(RegX0<R, E>{x0}, d, t, a, ex);
#pragma unroll
    for (int e = 0; e < E; ++e) x0[e] = cadd(x0[e], d[e]);
}

// One whole pass on the line held in x: FP32 in increment form, FP64 plain
// (RATIO: FFTs on the ratio twiddles of a.rtwid; ROWS, FP32: twiddles from
// the per-thread rows a.twrows).
template <typename R, int N, int E, bool PADDED, bool RATIO = false, bool ROWS = false, class Ex>
__device__ __forceinline__ void fused_pass(C2<R> (&x)[E], int t, const PassArgs& a, const Ex& ex) {
    static_assert(!ROWS || sizeof(R) == 4, "twiddle rows: FP32 passes");
    if constexpr (sizeof(R) == 4) {
        two_level_pass_incr<R, N, E, PADDED, ROWS>(x, t, a, ex);
    } else {
        if (a.jq_in) jq_all<R, E>(x, a.jq_in_E, a.jq_in_1mE);
        two_level_chain<R, N, E, PADDED, RATIO>(x, t, a, ex);
        if (a.jq_out) jq_all<R, E>(x, a.jq_out_E, a.jq_out_1mE);
    }
}

// Field loads: plain (may be served by L1) or .cg (L2 only). A persistent kernel
// that reads data another SM wrote during the same launch uses .cg.
template <bool CG, typename T>
__device__ __forceinline__ T ld_field(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// Global addressing of complex line `cl` (see PassArgs): element idx of the
// line is (p0[idx], p1[idx]) for a contiguous pass and the 2-vector at
// p0 + idx * stride for a strided pass. PADDED: lines hold nmem < N values
// (loads beyond them give zeros, stores stop there) and a strided pass with an
// odd inner extent moves its two columns as scalars (the second may not exist).
// Stores go out_shift elements past the loads (PassArgs::out_shift).
template <typename R, int N, bool STRIDED, bool PADDED = false>
struct LineRef {
    R* p0;
    R* p1;
    long long stride;
    long long shift;
    int nmem;
    bool active;
    bool vec;  // strided pass moved as aligned 2-vectors

    __device__ __forceinline__ LineRef(const PassArgs& a, long long cl) {
        R* u = static_cast<R*>(a.u);
        shift = a.out_shift;
        active = cl < a.clines;
        nmem = PADDED ? a.nmem : N;
        if (STRIDED) {
            const long long pairs = (a.inner + 1) >> 1;
            const long long o = active ? cl / pairs : 0;
            const long long c = active ? cl - o * pairs : 0;
            p0 = u + o * (long long)nmem * a.inner + 2 * c;
            vec = !PADDED || (a.inner & 1) == 0;
            p1 = (active && 2 * c + 1 < a.inner) ? p0 + 1 : nullptr;
            stride = a.inner;
        } else {
            const long long r0 = active ? 2 * cl : 0;
            p0 = u + r0 * nmem;
            p1 = (active && r0 + 1 < a.outer) ? p0 + nmem : nullptr;
            stride = 1;
            vec = false;
        }
    }

    template <int E, bool CG = false>
    __device__ __forceinline__ void load(C2<R> (&x)[E], int t) const {
        using V = typename Vec2T<R>::type;
        constexpr int T = N / E;
        if (STRIDED) {
            const R* q = p0 + t * stride;
            const long long step = T * stride;
#pragma unroll
            for (int e = 0; e < E; ++e, q += step) {
                const bool in = active && (!PADDED || t + e * T < nmem);
                if (in && (!PADDED || vec)) {
                    const V v = ld_field<CG>(reinterpret_cast<const V*>(q));
                    x[e] = {v.x, v.y};
                } else if (in) {
                    x[e] = {ld_field<CG>(q), p1 ? ld_field<CG>(q + 1) : R(0)};
                } else {
                    x[e] = {R(0), R(0)};
                }
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int idx = t + e * T;
                const bool in = !PADDED || idx < nmem;
                x[e].x = (active && in) ? ld_field<CG>(p0 + idx) : R(0);
                x[e].y = (p1 && in) ? ld_field<CG>(p1 + idx) : R(0);
            }
        }
    }

    template <int E>
    __device__ __forceinline__ void store(const C2<R> (&x)[E], int t) const {
        using V = typename Vec2T<R>::type;
        constexpr int T = N / E;
        if (!active) return;
        if (STRIDED) {
            R* q = p0 + shift + t * stride;
            const long long step = T * stride;
#pragma unroll
            for (int e = 0; e < E; ++e, q += step) {
                if (PADDED && t + e * T >= nmem) continue;
                if (!PADDED || vec) {
                    V v;
                    v.x = x[e].x;
                    v.y = x[e].y;
                    *reinterpret_cast<V*>(q) = v;
                } else {
                    q[0] = x[e].x;
                    if (p1) q[1] = x[e].y;
                }
            }
        } else {
            R* s0 = p0 + shift;
            R* s1 = p1 ? p1 + shift : nullptr;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int idx = t + e * T;
                if (PADDED && idx >= nmem) continue;
                s0[idx] = x[e].x;
                if (s1) s1[idx] = x[e].y;
            }
        }
    }
};

// Lines of either kind, chosen at run time (the batch kernel): one copy of the
// pass body then serves contiguous and strided passes and only the loads and
// stores branch, which halves the code the batch kernel keeps in flight.
// Power-of-two lines (not zero-padded); a strided pass needs an even inner
// extent (2-vector column pairs). Loads are L2-only (.cg): other SMs wrote the
// field during the same launch.
template <typename R, int N>
struct LineRefAny {
    R* p0;
    R* p1;
    long long stride;
    bool active;
    bool strided;

    __device__ __forceinline__ LineRefAny(const PassArgs& a, long long cl, bool strided_) : strided(strided_) {
        R* u = static_cast<R*>(a.u);
        active = cl < a.clines;
        if (strided) {
            const long long pairs = a.inner >> 1;
            const long long o = active ? cl / pairs : 0;
            const long long c = active ? cl - o * pairs : 0;
            p0 = u + o * (long long)N * a.inner + 2 * c;
            p1 = p0 + 1;
            stride = a.inner;
        } else {
            const long long r0 = active ? 2 * cl : 0;
            p0 = u + r0 * N;
            p1 = (active && r0 + 1 < a.outer) ? p0 + N : nullptr;
            stride = 1;
        }
    }

    template <int E>
    __device__ __forceinline__ void load(C2<R> (&x)[E], int t) const {
        using V = typename Vec2T<R>::type;
        constexpr int T = N / E;
        if (strided) {
            const R* q = p0 + t * stride;
            const long long step = T * stride;
#pragma unroll
            for (int e = 0; e < E; ++e, q += step) {
                if (active) {
                    const V v = __ldcg(reinterpret_cast<const V*>(q));
                    x[e] = {v.x, v.y};
                } else {
                    x[e] = {R(0), R(0)};
                }
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int idx = t + e * T;
                x[e].x = active ? __ldcg(p0 + idx) : R(0);
                x[e].y = p1 ? __ldcg(p1 + idx) : R(0);
            }
        }
    }

    template <int E>
    __device__ __forceinline__ void store(const C2<R> (&x)[E], int t) const {
        using V = typename Vec2T<R>::type;
        constexpr int T = N / E;
        if (!active) return;
        if (strided) {
            R* q = p0 + t * stride;
            const long long step = T * stride;
#pragma unroll
            for (int e = 0; e < E; ++e, q += step) {
                V v;
                v.x = x[e].x;
                v.y = x[e].y;
                *reinterpret_cast<V*>(q) = v;
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
};

// ---------------------------------------------------------------------------
// Kernel 1: CTA-synchronised exchanges.
// ---------------------------------------------------------------------------

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

// MINB: minimum resident CTAs per SM the register allocation must allow.
template <typename R, int N, int E, int LPC, bool STRIDED, int MINB, bool PADDED>
__global__ void __launch_bounds__(LPC*(N / E), MINB)
axis_pass_kernel(const PassArgs a) {
    constexpr int T = N / E;
    using Ex = PadExchange<R, N, LPC, STRIDED>;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int tid = threadIdx.x;
    // Strided passes: lanes walk over neighbouring lines first (coalesced rows);
    // contiguous passes: lanes walk along a line.
    const int j = STRIDED ? (tid % LPC) : (tid / T);
    const int t = STRIDED ? (tid / LPC) : (tid % T);
    const LineRef<R, N, STRIDED, PADDED> line(a, (long long)blockIdx.x * LPC + j);
    const Ex ex{reinterpret_cast<C2<R>*>(smem_raw), j};

    C2<R> x[E];
    line.template load<E>(x, t);
    // ratio-twiddle records exist for the FP64 pass's default values per thread only
    fused_pass<R, N, E, PADDED, (sizeof(R) == 8 && E <= 16 && E == f64_elems_per_thread(N))>(x, t, a, ex);
    line.template store<E>(x, t);
}

// ---------------------------------------------------------------------------
// Kernel 2: warp-local lines (16 values per thread).
// ---------------------------------------------------------------------------

// Per-line exchange region of N + N/E complex values: element a is stored at
// a + a/E. With lanes laid out as (line, t), the first-pass writes (at t*E + r)
// and the reads (at t + e*T) of every pass hit distinct banks in each
// half-warp, also when a half-warp holds several short lines.
// LE: distance of the lines' regions (default N + N/E).
template <typename R, int N, int E, int LE = N + N / E>
struct WarpExchange {
    // (E = 2, 4: one pad per 16 values)
    static constexpr int SH = E == 32 ? 5 : (E == 16 ? 4 : (E == 8 ? 3 : 4));
    C2<R>* base;
    __device__ __forceinline__ void put(int idx, C2<R> v) const { base[idx + (idx >> SH)] = v; }
    __device__ __forceinline__ C2<R> get(int idx) const { return base[idx + (idx >> SH)]; }
    static __device__ __forceinline__ void sync() { __syncwarp(); }
    static constexpr int LINE_ELEMS = LE;
    static_assert(LE >= N + N / E, "line region too small");
};

// Lines [first, first + 32/T) of the pass `a`, processed by one warp. `region`
// is this warp's shared memory: (32/T) * (N + N/E) complex values.
template <typename R, int N, int E, bool STRIDED, bool CG, bool PADDED = false>
__device__ __forceinline__ void warp_pass_lines(const PassArgs& a, long long first, C2<R>* region, int lane) {
    constexpr int T = N / E;
    static_assert(T >= 1 && T <= 32, "line must fit one warp");
    using Ex = WarpExchange<R, N, E>;
    const int j = lane / T, t = lane % T;
    const LineRef<R, N, STRIDED, PADDED> line(a, first + j);
    const Ex ex{region + j * Ex::LINE_ELEMS};
    C2<R> x[E];
    line.template load<E, CG>(x, t);
    fused_pass<R, N, E, PADDED, false, (sizeof(R) == 4)>(x, t, a, ex);
    line.template store<E>(x, t);
}

// Shared-memory tables of one axis for the persistent kernels: eC[N], eS[N],
// twist[N] (not for padded passes), twiddles[N] and, for FP32 passes with E
// values per thread, the twiddle rows of TwRows<N, E>; copied (built) once per
// CTA. The rows start 16-byte aligned (the dynamic shared memory is).
template <typename R, int N, int E, bool PADDED>
struct SmemTables {
    static constexpr bool ROWS = sizeof(R) == 4;
    static constexpr size_t HEAD = 2 * N * sizeof(R) + (PADDED ? 1 : 2) * N * sizeof(C2<R>);
    static constexpr size_t ROWS_OFF = (HEAD + 15) / 16 * 16;
    static constexpr size_t BYTES = ROWS ? ROWS_OFF + sizeof(C2<R>) * (size_t)tw_rows_elems(N, E, N) : HEAD;
    static __device__ __forceinline__ void load(PassArgs& a, unsigned char* smem) {
        R* eC = reinterpret_cast<R*>(smem);
        R* eS = eC + N;
        C2<R>* tw = reinterpret_cast<C2<R>*>(eS + N);
        C2<R>* twist = tw + N;
        const R* gC = static_cast<const R*>(a.eC);
        const R* gS = static_cast<const R*>(a.eS);
        const C2<R>* gtw = static_cast<const C2<R>*>(a.twid);
        const C2<R>* gtwist = static_cast<const C2<R>*>(a.twist);
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            eC[i] = gC[i];
            eS[i] = gS[i];
            tw[i] = gtw[i];
            if (!PADDED) twist[i] = gtwist[i];
        }
        if constexpr (ROWS) {
            C2<float>* rows = reinterpret_cast<C2<float>*>(smem + ROWS_OFF);
            build_tw_rows<N, E>(rows, reinterpret_cast<const C2<float>*>(gtw), threadIdx.x, blockDim.x);
            a.twrows = rows;
        }
        __syncthreads();
        a.eC = eC;
        a.eS = eS;
        a.twid = tw;
        a.twist = PADDED ? nullptr : twist;
    }
};

// Persistent: each CTA copies the axis tables to shared memory once, then its
// warps take warp-groups of lines (32/T lines each) in a grid-stride loop.
template <typename R, int N, int E, int WPB, bool STRIDED, bool PADDED>
__global__ void __launch_bounds__(WPB * 32)
axis_pass_warp_kernel(const PassArgs a0, long long ngroups) {
    constexpr int LPW = 32 / (N / E);  // lines per warp
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PassArgs a = a0;
    SmemTables<R, N, E, PADDED>::load(a, smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C2<R>* region = reinterpret_cast<C2<R>*>(smem_raw + SmemTables<R, N, E, PADDED>::BYTES) +
                    warp * LPW * WarpExchange<R, N, E>::LINE_ELEMS;
    for (long long g = (long long)blockIdx.x * WPB + warp; g < ngroups; g += (long long)gridDim.x * WPB) {
        warp_pass_lines<R, N, E, STRIDED, false, PADDED>(a, g * LPW, region, lane);
        __syncwarp();
    }
}

// Persistent CTA lines (FP32 lines of 2048 and 4096 points): each CTA copies
// the axis tables and builds the twiddle rows in shared memory once (up to
// 205 KB at 4096 points), then takes the groups of LPC lines
// blockIdx.x + k gridDim.x, lanes mapped as in axis_pass_kernel. Table and
// twiddle loads from global memory had kept the LSU queue full there (ncu:
// long-scoreboard and global-throttle stalls, l1tex 70% busy); the results are
// bit-identical to axis_pass_kernel's.
template <typename R, int N, int E, int LPC, bool STRIDED, bool PADDED>
__global__ void __launch_bounds__(LPC * (N / E), 1)
axis_pass_cta_rows_kernel(const PassArgs a0, long long ngroups) {
    constexpr int T = N / E;
    using Ex = PadExchange<R, N, LPC, STRIDED>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PassArgs a = a0;
    SmemTables<R, N, E, PADDED>::load(a, smem_raw);
    const int tid = threadIdx.x;
    const int j = STRIDED ? (tid % LPC) : (tid / T);
    const int t = STRIDED ? (tid / LPC) : (tid % T);
    const Ex ex{reinterpret_cast<C2<R>*>(smem_raw + SmemTables<R, N, E, PADDED>::BYTES), j};
    if constexpr (!PADDED) {
        // the next group's line is loaded into registers while this one is
        // computed (side by side: 2D 4096^2 FP32 step 0.435 -> 0.404 ms,
        // 2048^2 0.107 -> 0.102 ms; the zero-padded passes, near 255 registers
        // already, got slower and load as they go)
        C2<R> xn[E];
        long long g = blockIdx.x;
        if (g < ngroups) LineRef<R, N, STRIDED, PADDED>(a, g * LPC + j).template load<E>(xn, t);
        for (; g < ngroups; g += gridDim.x) {
            C2<R> x[E];
#pragma unroll
            for (int e = 0; e < E; ++e) x[e] = xn[e];
            const long long gn = g + gridDim.x;
            if (gn < ngroups) LineRef<R, N, STRIDED, PADDED>(a, gn * LPC + j).template load<E>(xn, t);
            fused_pass<R, N, E, PADDED, false, true>(x, t, a, ex);
            LineRef<R, N, STRIDED, PADDED>(a, g * LPC + j).template store<E>(x, t);
            __syncthreads();  // the exchange region is reused by the next group
        }
    } else {
        for (long long g = blockIdx.x; g < ngroups; g += gridDim.x) {
            const LineRef<R, N, STRIDED, PADDED> line(a, g * LPC + j);
            C2<R> x[E];
            line.template load<E>(x, t);
            fused_pass<R, N, E, PADDED, false, true>(x, t, a, ex);
            line.template store<E>(x, t);
            __syncthreads();  // the exchange region is reused by the next group
        }
    }
}

// ---------------------------------------------------------------------------
// Launch configuration
// ---------------------------------------------------------------------------

// Elements per thread of kernel 1: 8 for most lengths (radix-8 passes), 16 at N = 4096.
template <int N>
constexpr int elems_per_thread() {
    return N >= 4096 ? 16 : (N < 8 ? N : 8);
}

// Per-kernel launch set-up, done once per device: the shared-memory attribute
// (cudaFuncSetAttribute acts on the current device only) and, for persistent
// kernels, the resident grid (CTAs per SM x SMs).
struct LaunchSetup {
    static constexpr int kMaxDevices = 64;
    std::atomic<unsigned long long> configured{0};  // bit d: attribute set on device d
    std::atomic<int> resident[kMaxDevices] = {};
};

template <class K>
cudaError_t set_smem(K kern, size_t smem, LaunchSetup& ls, int* dev_out) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= LaunchSetup::kMaxDevices) return cudaErrorInvalidDevice;
    *dev_out = dev;
    if ((ls.configured.load() >> dev) & 1ULL) return cudaSuccess;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err == cudaSuccess) ls.configured.fetch_or(1ULL << dev);
    return err;
}

// Resident grid of a persistent kernel on device `dev` (computed once).
template <class K>
cudaError_t resident_grid(K kern, int threads, size_t smem, LaunchSetup& ls, int dev, int* grid) {
    int r = ls.resident[dev].load();
    if (r == 0) {
        int sms = 0, per_sm = 0;
        cudaError_t err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        if (err != cudaSuccess) return err;
        r = (per_sm < 1 ? 1 : per_sm) * (sms < 1 ? 1 : sms);
        ls.resident[dev].store(r);
    }
    *grid = r;
    return cudaSuccess;
}

template <typename R, int N, int E, int LPC, bool STRIDED, bool PADDED>
cudaError_t launch_cfg(const PassArgs& a, cudaStream_t s) {
    constexpr int T = N / E;
    // FP64 with 128-thread CTAs: at least two CTAs per SM, so one CTA's
    // exchanges overlap the other's FP64 arithmetic.
    constexpr int MINB = (sizeof(R) == 8 && LPC * T == 128) ? 2 : 1;
    using Ex = PadExchange<R, N, LPC, STRIDED>;
    const size_t smem = sizeof(C2<R>) * (size_t)Ex::elems();
    auto kern = axis_pass_kernel<R, N, E, LPC, STRIDED, MINB, PADDED>;
    static LaunchSetup setup;
    int dev = 0;
    cudaError_t err = set_smem(kern, smem, setup, &dev);
    if (err != cudaSuccess) return err;
    const long long grid = (a.clines + LPC - 1) / LPC;
    if (grid <= 0) return cudaSuccess;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
    kern<<<(unsigned)grid, LPC * T, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename R, int N, int E, int WPB, bool STRIDED, bool PADDED>
cudaError_t launch_warp(const PassArgs& a, cudaStream_t s) {
    constexpr int LPW = 32 / (N / E);
    const size_t smem = SmemTables<R, N, E, PADDED>::BYTES +
                        sizeof(C2<R>) * (size_t)WPB * LPW * WarpExchange<R, N, E>::LINE_ELEMS;
    auto kern = axis_pass_warp_kernel<R, N, E, WPB, STRIDED, PADDED>;
    static LaunchSetup setup;
    int dev = 0, resident = 0;
    cudaError_t err = set_smem(kern, smem, setup, &dev);
    if (err == cudaSuccess) err = resident_grid(kern, WPB * 32, smem, setup, dev, &resident);
    if (err != cudaSuccess) return err;
    const long long ngroups = (a.clines + LPW - 1) / LPW;
    if (ngroups <= 0) return cudaSuccess;
    const long long want = (ngroups + WPB - 1) / WPB;
    const long long grid = want < resident ? want : resident;
    kern<<<(unsigned)grid, WPB * 32, smem, s>>>(a, ngroups);
    return cudaGetLastError();
}

template <typename R, int N, int E, int LPC, bool STRIDED, bool PADDED>
cudaError_t launch_cta_rows(const PassArgs& a, cudaStream_t s) {
    using Ex = PadExchange<R, N, LPC, STRIDED>;
    const size_t smem = SmemTables<R, N, E, PADDED>::BYTES + sizeof(C2<R>) * (size_t)Ex::elems();
    auto kern = axis_pass_cta_rows_kernel<R, N, E, LPC, STRIDED, PADDED>;
    static LaunchSetup setup;
    int dev = 0, resident = 0;
    cudaError_t err = set_smem(kern, smem, setup, &dev);
    if (err == cudaSuccess) err = resident_grid(kern, LPC * (N / E), smem, setup, dev, &resident);
    if (err != cudaSuccess) return err;
    const long long ngroups = (a.clines + LPC - 1) / LPC;
    if (ngroups <= 0) return cudaSuccess;
    const long long grid = ngroups < resident ? ngroups : resident;
    kern<<<(unsigned)grid, LPC * (N / E), smem, s>>>(a, ngroups);
    return cudaGetLastError();
}

// SMs of the current device (cached per device; 0 if unknown).
inline int current_device_sms() {
    static std::atomic<int> cache[LaunchSetup::kMaxDevices] = {};
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= LaunchSetup::kMaxDevices) {
        cudaGetLastError();
        return 0;
    }
    if ((sms = cache[dev].load()) != 0) return sms;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cache[dev].store(sms);
    return sms;
}

// Values per thread that give a line 32 threads (at least 2 values): the
// shape of the small-grid passes below.
template <int N>
constexpr int warp_line_elems() {
    return N / 32 >= 2 ? N / 32 : 2;
}

template <typename R, int N, bool PADDED>
cudaError_t launch_n(const PassArgs& a, cudaStream_t s) {
    constexpr int E = elems_per_thread<N>();
    constexpr int T = N / E;
    // the host builds the FP64 ratio-twiddle records for this E
    static_assert(sizeof(R) != 8 || E == f64_elems_per_thread(N), "FP64 values per thread");
    // Small grids: when the default shape would leave SMs without work, each
    // line gets a warp of its own (N/32 values per thread, one line per CTA or
    // warp), so that as many SMs as there are lines work on it. The passes are
    // then latency bound; a shorter per-thread chain and more SMs beat fewer,
    // fuller threads. Same arithmetic, other exchange schedule.
    constexpr int ES = warp_line_elems<N>();
    const int sms = current_device_sms();
    if constexpr (sizeof(R) == 4 && N >= 32 && N <= 512) {
        // FP32: warp-local lines with 16 values per thread. Two warps per CTA
        // for long lines (few lines: many small CTAs spread better over 152
        // SMs), four otherwise.
        // A strided pass that stores into mapped host memory: 256-thread CTAs
        // of 256/T lines, so that each row a CTA writes is 64 bytes or more
        // (the warp kernel's 16-byte pieces ran the link at a fraction of its rate).
        if (a.host_io && a.inner > 1) return launch_cfg<R, N, 16, 256 / (N / 16), true, PADDED>(a, s);
        constexpr int WPB = N >= 512 ? 2 : 4;
        constexpr int LPW = 32 / (N / 16);
        // (not below N = 128: on the 64^2 grid one CTA of four 8-line warps was
        // faster than 32 one-line warps, 1.01 against 1.14 ms per 100 steps)
        if constexpr (ES < 16 && N >= 128) {
            if ((a.clines + LPW - 1) / LPW < sms) {
                if (a.inner > 1) return launch_warp<R, N, ES, 1, true, PADDED>(a, s);
                return launch_warp<R, N, ES, 1, false, PADDED>(a, s);
            }
        }
        if (a.inner > 1) return launch_warp<R, N, 16, WPB, true, PADDED>(a, s);
        return launch_warp<R, N, 16, WPB, false, PADDED>(a, s);
    } else if constexpr (sizeof(R) == 4 && N >= 1024) {
        // FP32, long lines: 16 values per thread, which keeps the increment
        // form's arrays in registers. Contiguous passes: one line per CTA (64
        // to 256 threads). Strided passes: 256 threads per CTA, so that lanes
        // next to each other read neighbouring columns (4 lines at N = 1024:
        // 32-byte rows; the strided 1024-point pass went from 18.8 to 12.9 us
        // on a 1024^2 field).
        constexpr int LPC_S = (256 / (N / 16)) > 1 ? 256 / (N / 16) : 1;
        // 2048 and 4096 points: persistent CTAs with the tables and twiddle
        // rows in shared memory (side by side: 2D 4096^2 FP32 step 0.697 ->
        // 0.437 ms, 2048^2 0.140 -> 0.107 ms). At 1024 points the grid is
        // latency bound and the per-CTA table build cost more (0.036 -> 0.046 ms).
        if constexpr (N >= 2048) {
            if (a.inner > 1) return launch_cta_rows<R, N, 16, LPC_S, true, PADDED>(a, s);
            return launch_cta_rows<R, N, 16, 1, false, PADDED>(a, s);
        }
        if (a.inner > 1) return launch_cfg<R, N, 16, LPC_S, true, PADDED>(a, s);
        return launch_cfg<R, N, 16, 1, false, PADDED>(a, s);
    } else {
        // FP64 passes are bound by the FP64 pipe, not by memory: they take
        // 128-thread CTAs (several per SM, so one CTA's exchanges overlap
        // another's arithmetic). FP32 strided passes keep >= 32 bytes of each row
        // per CTA (one sector); lines of 2048+ points keep 256 threads per CTA.
        constexpr int TPB = sizeof(R) == 8 ? 128 : 256;
        constexpr int MIN_S = (T >= 256 || sizeof(R) == 8) ? 1 : 32 / (2 * (int)sizeof(R));
        constexpr int LPC_S = (TPB / T) > MIN_S ? (TPB / T) : MIN_S;
        constexpr int LPC_C = (TPB / T) > 1 ? (TPB / T) : 1;
        if constexpr (sizeof(R) == 8 && N >= 32 && N <= 256) {
            // FP64 small grids: fewer CTAs than the SMs' two CTA slots -> one
            // line per 32-thread CTA (E = N/32; complex twiddles unless E is
            // the default, whose ratio records the plan holds)
            const int lpc = a.inner > 1 ? LPC_S : LPC_C;
            if ((a.clines + lpc - 1) / lpc < 2LL * sms) {
                if (a.inner > 1) return launch_cfg<R, N, ES, 1, true, PADDED>(a, s);
                return launch_cfg<R, N, ES, 1, false, PADDED>(a, s);
            }
        }
        if (a.inner > 1) return launch_cfg<R, N, E, LPC_S, true, PADDED>(a, s);
        return launch_cfg<R, N, E, LPC_C, false, PADDED>(a, s);
    }
}

template <typename R, bool PADDED>
cudaError_t launch_pass_any(int N, const PassArgs& a, cudaStream_t s) {
    switch (N) {
        case 4: return launch_n<R, 4, PADDED>(a, s);
        case 8: return launch_n<R, 8, PADDED>(a, s);
        case 16: return launch_n<R, 16, PADDED>(a, s);
        case 32: return launch_n<R, 32, PADDED>(a, s);
        case 64: return launch_n<R, 64, PADDED>(a, s);
        case 128: return launch_n<R, 128, PADDED>(a, s);
        case 256: return launch_n<R, 256, PADDED>(a, s);
        case 512: return launch_n<R, 512, PADDED>(a, s);
        case 1024: return launch_n<R, 1024, PADDED>(a, s);
        case 2048: return launch_n<R, 2048, PADDED>(a, s);
        case 4096: return launch_n<R, 4096, PADDED>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sfac
