// sfac_host.h - host-side FP64 precompute shared by plans and batches.
#pragma once

#include <vector>

namespace sfac {

// The FP64 tables of one axis (Sec. 2.1, Sec. 2.2, Remark 1).
struct AxisHost {
    int n = 0;
    std::vector<double> bcol, cfirst, sfirst, lambda, mu;
    std::vector<double> eC, eS, twist, twid;  // twist, twid: interleaved complex
    std::vector<double> dC, dS;               // expm1 forms for the FP32 increment passes
};

// Zero-padded form of one axis, for any n: e^{t C} and e^{tau S} are symmetric
// Toeplitz matrices, so each is a linear convolution of the line with its
// first column; padded to a power of two L >= 2n - 1 the convolution is
// circular and its multiplier (the DFT of the symmetric padded column) is real.
struct AxisPadded {
    int n = 0, L = 0;
    std::vector<double> mC, mS;    // L real multipliers incl. 1/L: e^{tau/2 C}, e^{tau S}
    std::vector<double> mC1, mS1;  // the same for (e^{tX} - I): increment forms
    std::vector<double> mB;        // L real multipliers incl. 1/L of B itself (diagnostics)
    std::vector<double> twid;      // L complex e^{-2 pi i m / L}, interleaved
};

bool is_pow2(int v);

// Smallest power of two >= 2n - 1 (at least 4).
int padded_length(int n);

// Padded tables of one axis (needs the spectra of compute_axis in T).
void compute_axis_padded(const AxisHost& T, double tau, AxisPadded* P);

// Tables of one axis for Riesz order alpha, interface parameter eps, step tau,
// domain [a, b] and n interior unknowns.
void compute_axis(double alpha, double eps, double tau, double a, double b, int n, AxisHost* T);

// Ratio-twiddle records of the FP64 FFT passes of length N with E values per
// thread (E <= 16; layout in sfac_fft.cuh, FftPassRatio); empty if no pass of
// span > 1 exists.
std::vector<double> ratio_twiddles(int N, int E);

}  // namespace sfac
