// sfac_diag.cu - fused reductions for monitoring a run: max|u| and the discrete
// energy E(u) = h^d ( (1/4) sum (u^2 - 1)^2 - (1/2) u^T A u ) (Example 5, Sec. 5),
// with A u = sum_l (B_l along axis l) and B_l = C_l + S_l.
//
// u^T A u = sum_l sum_{lines of axis l} x^T B_l x, so each axis pass loads its
// lines (two real lines as one complex line, as in the step passes), forms
// B_l x through the Remark 1 spectra, B x = F^{-1} (lambda/N) F x +
// Theta^{-1} F^{-1} (mu/N) F Theta x (or, for zero-padded axes, one linear
// convolution with the Toeplitz column of B), and accumulates x . B x; the first
// axis pass also accumulates (u^2 - 1)^2 and max|u|. Arithmetic is FP64 for both
// field precisions. Partial sums go to plan-owned scratch, one entry per CTA, and
// a one-CTA kernel adds them in a fixed order, so the result is deterministic.
#include <cuda_runtime.h>

#include "sfac_diag.h"
#include "sfac_pass.cuh"

namespace sfac {

namespace {

constexpr int DIAG_E = 8;
constexpr int DIAG_THREADS = 128;  // at least; a CTA holds LPC whole lines

template <int N>
struct DiagShape {
    static constexpr int E = (N < DIAG_E) ? N : DIAG_E;
    static constexpr int T = N / E;
    static constexpr int LPC = (DIAG_THREADS / T) > 0 ? DIAG_THREADS / T : 1;
    static constexpr int THREADS = LPC * T;
};

template <typename Rin, int N, bool STRIDED, bool PADDED>
__global__ void __launch_bounds__(DiagShape<N>::THREADS)
diag_pass_kernel(const PassArgs a, const double* __restrict__ mA, const double* __restrict__ mB, int first_axis,
                 double3* __restrict__ partial) {
    constexpr int E = DiagShape<N>::E;
    constexpr int T = DiagShape<N>::T;
    constexpr int LPC = DiagShape<N>::LPC;
    constexpr int THREADS = DiagShape<N>::THREADS;
    using Ex = PadExchange<double, N, LPC, STRIDED>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[3][THREADS];

    const int tid = threadIdx.x;
    const int j = STRIDED ? (tid % LPC) : (tid / T);
    const int t = STRIDED ? (tid / LPC) : (tid % T);
    const LineRef<Rin, N, STRIDED, PADDED> line(a, (long long)blockIdx.x * LPC + j);
    const Ex ex{reinterpret_cast<C2<double>*>(smem_raw), j};

    C2<Rin> xin[E];
    line.template load<E>(xin, t);
    C2<double> x[E], y[E], z[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = {double(xin[e].x), double(xin[e].y)};

    double pot = 0.0, mx = 0.0;
    if (first_axis && line.active) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if (PADDED && t + e * T >= line.nmem) continue;
            const double a2 = x[e].x * x[e].x - 1.0, b2 = x[e].y * x[e].y - 1.0;
            pot += a2 * a2;
            mx = fmax(mx, fabs(x[e].x));
            if (line.p1) {
                pot += b2 * b2;
                mx = fmax(mx, fabs(x[e].y));
            }
        }
    }
    const C2<double>* tw = static_cast<const C2<double>*>(a.twid);
    // y = C x (or the whole Toeplitz B for a zero-padded axis)
#pragma unroll
    for (int e = 0; e < E; ++e) y[e] = x[e];
    apply_spectral<double, N, E>(y, t, tw, ex, mA);
    if constexpr (!PADDED) {
        // z = S x = Theta^{-1} F^{-1} (mu/N) F Theta x
        const C2<double>* twist = static_cast<const C2<double>*>(a.twist);
#pragma unroll
        for (int e = 0; e < E; ++e) z[e] = cmul(x[e], ldg_c2(twist + t + e * T));
        apply_spectral<double, N, E>(z, t, tw, ex, mB);
#pragma unroll
        for (int e = 0; e < E; ++e) y[e] = cadd(y[e], cmulc(z[e], ldg_c2(twist + t + e * T)));
    }
    double dot = 0.0;
    if (line.active) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if (PADDED && t + e * T >= line.nmem) continue;
            dot += x[e].x * y[e].x + x[e].y * y[e].y;  // a^T B a + b^T B b (b = 0 when absent)
        }
    }
    red[0][tid] = dot;
    red[1][tid] = pot;
    red[2][tid] = mx;
    __syncthreads();
    for (int w = THREADS / 2; w > 0; w >>= 1) {
        if (tid < w) {
            red[0][tid] += red[0][tid + w];
            red[1][tid] += red[1][tid + w];
            red[2][tid] = fmax(red[2][tid], red[2][tid + w]);
        }
        __syncthreads();
    }
    if (tid == 0) partial[blockIdx.x] = make_double3(red[0][0], red[1][0], red[2][0]);
}

// Adds n partials in a fixed order into out[0..2] (+= for the sums, max for
// the third), one CTA.
__global__ void __launch_bounds__(DIAG_THREADS)
diag_reduce_kernel(const double3* __restrict__ partial, long long n, double* __restrict__ out) {
    __shared__ double red[3][DIAG_THREADS];
    const int tid = threadIdx.x;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (long long i = tid; i < n; i += DIAG_THREADS) {
        const double3 v = partial[i];
        s0 += v.x;
        s1 += v.y;
        s2 = fmax(s2, v.z);
    }
    red[0][tid] = s0;
    red[1][tid] = s1;
    red[2][tid] = s2;
    __syncthreads();
    for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
        if (tid < w) {
            red[0][tid] += red[0][tid + w];
            red[1][tid] += red[1][tid + w];
            red[2][tid] = fmax(red[2][tid], red[2][tid + w]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        out[0] += red[0][0];
        out[1] += red[1][0];
        out[2] = fmax(out[2], red[2][0]);
    }
}

template <typename Rin, int N, bool STRIDED, bool PADDED>
cudaError_t launch_diag_cfg(const PassArgs& a, const double* mA, const double* mB, int first_axis,
                            double3* partial, long long* nblocks, cudaStream_t s) {
    constexpr int LPC = DiagShape<N>::LPC;
    using Ex = PadExchange<double, N, LPC, STRIDED>;
    const size_t smem = sizeof(C2<double>) * (size_t)Ex::elems();
    auto kern = diag_pass_kernel<Rin, N, STRIDED, PADDED>;
    static LaunchSetup setup;
    int dev = 0;
    const cudaError_t err = set_smem(kern, smem, setup, &dev);
    if (err != cudaSuccess) return err;
    const long long grid = (a.clines + LPC - 1) / LPC;
    *nblocks = grid;
    if (grid <= 0) return cudaSuccess;
    kern<<<(unsigned)grid, DiagShape<N>::THREADS, smem, s>>>(a, mA, mB, first_axis, partial);
    return cudaGetLastError();
}

template <typename Rin, int N, bool PADDED>
cudaError_t launch_diag_n(const PassArgs& a, const double* mA, const double* mB, int first_axis, double3* partial,
                          long long* nblocks, cudaStream_t s) {
    if (a.inner > 1) return launch_diag_cfg<Rin, N, true, PADDED>(a, mA, mB, first_axis, partial, nblocks, s);
    return launch_diag_cfg<Rin, N, false, PADDED>(a, mA, mB, first_axis, partial, nblocks, s);
}

template <typename Rin, bool PADDED>
cudaError_t launch_diag_any(int N, const PassArgs& a, const double* mA, const double* mB, int first_axis,
                            double3* partial, long long* nblocks, cudaStream_t s) {
    switch (N) {
#define SFAC_DIAG_CASE(L) \
    case L: return launch_diag_n<Rin, L, PADDED>(a, mA, mB, first_axis, partial, nblocks, s);
        SFAC_DIAG_CASE(4)
        SFAC_DIAG_CASE(8)
        SFAC_DIAG_CASE(16)
        SFAC_DIAG_CASE(32)
        SFAC_DIAG_CASE(64)
        SFAC_DIAG_CASE(128)
        SFAC_DIAG_CASE(256)
        SFAC_DIAG_CASE(512)
        SFAC_DIAG_CASE(1024)
        SFAC_DIAG_CASE(2048)
        SFAC_DIAG_CASE(4096)
#undef SFAC_DIAG_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

long long diag_partials_needed(long long clines, int N) {
    const int E = N < DIAG_E ? N : DIAG_E;
    const int T = N / E;
    const int LPC = (DIAG_THREADS / T) > 0 ? DIAG_THREADS / T : 1;
    return (clines + LPC - 1) / LPC;
}

cudaError_t launch_diag_axis(bool f64_field, bool padded, int N, const PassArgs& a, const double* mA,
                             const double* mB, int first_axis, double3* partial, double* out, cudaStream_t s) {
    long long nb = 0;
    cudaError_t err;
    if (f64_field)
        err = padded ? launch_diag_any<double, true>(N, a, mA, mB, first_axis, partial, &nb, s)
                     : launch_diag_any<double, false>(N, a, mA, mB, first_axis, partial, &nb, s);
    else
        err = padded ? launch_diag_any<float, true>(N, a, mA, mB, first_axis, partial, &nb, s)
                     : launch_diag_any<float, false>(N, a, mA, mB, first_axis, partial, &nb, s);
    if (err != cudaSuccess) return err;
    if (nb <= 0) return cudaSuccess;
    diag_reduce_kernel<<<1, DIAG_THREADS, 0, s>>>(partial, nb, out);
    return cudaGetLastError();
}

}  // namespace sfac
