// Host check of the device FFT core (csrc/sfac_fft.cuh): the register-resident
// Stockham FFT of one line, run by T = N / E host threads that meet at a
// barrier wherever the CTA would synchronise, against a long-double DFT.
//  - complex twiddles, FP64 (E as the FP64 kernels) and FP32 (E = 16, on the
//    packed two-lane FP32 forms, emulated lane by lane by the host shim);
//  - ratio twiddles (FP64, every length) with the table of ratio_twiddles; the table
//    is followed by poison values, so a record read past its end shows up as
//    a wrong result;
//  - FP32 with the per-thread twiddle rows of TwRows (built by build_tw_rows
//    and followed by poison values), which must give bit for bit the results
//    of the table-indexed twiddles.
// Prints one line per case: "<kind> N E INV err" (max error / max |exact|),
// and for the rows "rows32same N E INV 1" when they equal the table results.
#include <barrier>
#include <complex>
#include <cstdio>
#include <random>
#include <thread>
#include <vector>

#include "sfac_fft.cuh"
#include "sfac_host.h"
#include "sfac_internal.h"

using namespace sfac;

template <typename R>
struct HostEx {
    static std::barrier<>* bar;
    std::vector<C2<R>>* buf;
    void put(int idx, C2<R> v) const { (*buf)[idx] = v; }
    C2<R> get(int idx) const { return (*buf)[idx]; }
    static void sync() { bar->arrive_and_wait(); }
};
template <typename R>
std::barrier<>* HostEx<R>::bar = nullptr;

template <typename R, int N, int E, bool INV, bool RATIO, bool ROWS = false>
std::vector<std::complex<double>> run_line(const std::vector<std::complex<double>>& in,
                                           const std::vector<C2<R>>& tw, const std::vector<double>& rt,
                                           const std::vector<C2<R>>* rows = nullptr) {
    constexpr int T = N / E;
    std::vector<C2<R>> buf(N);
    std::barrier<> bar(T);
    HostEx<R>::bar = &bar;
    std::vector<std::complex<double>> out(N);
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t)
        th.emplace_back([&, t] {
            C2<R> x[E];
            for (int e = 0; e < E; ++e) x[e] = {R(in[t + e * T].real()), R(in[t + e * T].imag())};
            HostEx<R> ex{&buf};
            if constexpr (RATIO) line_fft_ratio<N, E, INV>(x, t, rt.data(), ex);
            else if constexpr (ROWS) line_fft_tw<R, N, E, INV>(x, t, TwRows<N, E>{rows->data()}, ex);
            else line_fft<R, N, E, INV>(x, t, tw.data(), ex);
            for (int e = 0; e < E; ++e) out[t + e * T] = {double(x[e].x), double(x[e].y)};
        });
    for (auto& h : th) h.join();
    return out;
}

template <int N, bool INV>
double rel_err(const std::vector<std::complex<double>>& in, const std::vector<std::complex<double>>& got) {
    const long double pi = 3.14159265358979323846264338327950288L;
    double emax = 0, scale = 0;
    for (int j = 0; j < N; ++j) {
        std::complex<long double> acc = 0;
        for (int k = 0; k < N; ++k) {
            const long double ang = (INV ? 2 : -2) * pi * (long double)((long long)j * k % N) / N;
            acc += std::complex<long double>(in[k].real(), in[k].imag()) *
                   std::complex<long double>(cosl(ang), sinl(ang));
        }
        const std::complex<double> ex((double)acc.real(), (double)acc.imag());
        emax = std::max(emax, std::abs(got[j] - ex));
        scale = std::max(scale, std::abs(ex));
    }
    return emax / scale;
}

template <typename R, int N, int E>
void check(bool ratio) {
    std::mt19937_64 rng(N * 31 + E);
    std::uniform_real_distribution<double> U(-1, 1);
    std::vector<std::complex<double>> in(N);
    for (auto& v : in) v = {U(rng), U(rng)};
    if (std::is_same<R, float>::value)
        for (auto& v : in) v = {double(float(v.real())), double(float(v.imag()))};
    std::vector<C2<R>> tw(N);
    for (int m = 0; m < N; ++m) {
        const long double a = 2 * 3.14159265358979323846264338327950288L * m / N;
        tw[m] = {R(cosl(a)), R(-sinl(a))};
    }
    std::vector<double> rt;
    if (ratio) {
        if constexpr (std::is_same<R, double>::value && E <= 16) {
            rt = ratio_twiddles(N, E);
            size_t need = 0;
            for (int P = 1; P < N;) {
                const int RAD = (P * E <= N) ? E : N / P;
                if (P > 1) need += (size_t)P * ratio_record(RAD);
                P *= RAD;
            }
            if (need != rt.size()) {
                printf("table N %d E %d size %zu expected %zu\n", N, E, rt.size(), need);
                return;
            }
            rt.resize(rt.size() + 64, 1e300);
            const double ef = rel_err<N, false>(in, run_line<R, N, E, false, true>(in, tw, rt));
            const double ei = rel_err<N, true>(in, run_line<R, N, E, true, true>(in, tw, rt));
            printf("ratio64 %d %d 0 %.3e\nratio64 %d %d 1 %.3e\n", N, E, ef, N, E, ei);
        }
        return;
    }
    const auto of = run_line<R, N, E, false, false>(in, tw, rt);
    const auto oi = run_line<R, N, E, true, false>(in, tw, rt);
    const double ef = rel_err<N, false>(in, of);
    const double ei = rel_err<N, true>(in, oi);
    const char* kind = std::is_same<R, double>::value ? "complex64b" : "complex32b";
    printf("%s %d %d 0 %.3e\n%s %d %d 1 %.3e\n", kind, N, E, ef, kind, N, E, ei);
    if constexpr (std::is_same<R, float>::value) {
        const int nrows = tw_rows_elems(N, E, N);
        std::vector<C2<float>> rows(nrows + 64, C2<float>{1e30f, -1e30f});
        build_tw_rows<N, E>(rows.data(), tw.data(), 0, 1);
        const auto rf = run_line<R, N, E, false, false, true>(in, tw, rt, &rows);
        const auto ri = run_line<R, N, E, true, false, true>(in, tw, rt, &rows);
        printf("rows32same %d %d 0 %d\nrows32same %d %d 1 %d\n", N, E, int(rf == of), N, E, int(ri == oi));
    }
}

template <int N>
void check_all() {
    constexpr int E64 = f64_elems_per_thread(N);
    check<double, N, E64>(false);
    check<double, N, E64>(true);
    if constexpr (N >= 32) check<float, N, 16>(false);
    // the other FP32 shapes: 8 values (batch kernel), N / 32 values (small grids)
    if constexpr (N >= 16 && N <= 512) check<float, N, 8>(false);
    if constexpr (N >= 8 && N <= 128) check<float, N, 4>(false);
    if constexpr (N >= 4 && N <= 64) check<float, N, 2>(false);
}

int main() {
    check_all<4>();
    check_all<8>();
    check_all<16>();
    check_all<32>();
    check_all<64>();
    check_all<128>();
    check_all<256>();
    check_all<512>();
    check_all<1024>();
    check_all<2048>();
    check_all<4096>();
    return 0;
}
