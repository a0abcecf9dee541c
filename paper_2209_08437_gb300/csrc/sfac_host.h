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

bool is_pow2(int v);

// Tables of one axis for Riesz order alpha, interface parameter eps, step tau,
// domain [a, b] and n interior unknowns.
void compute_axis(double alpha, double eps, double tau, double a, double b, int n, AxisHost* T);

}  // namespace sfac
