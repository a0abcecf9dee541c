// sfac_host.cu - FP64 precompute of the per-axis tables (host code).
#include <cmath>
#include <utility>

#include "sfac_host.h"

namespace sfac {

namespace {


// ---------------------------------------------------------------------------
// FP64 precompute (Sec. 2.1, Sec. 2.2, Remark 1)
// ---------------------------------------------------------------------------

// cos(pi m / n) and sin(pi m / n) for integer m, reduced exactly to an angle in
// [0, pi/4] first so that every table entry is correctly rounded or nearly so.
void sincospi_frac(long long m, long long n, double* c, double* s) {
    const long long two_n = 2 * n;
    m %= two_n;
    if (m < 0) m += two_n;
    double sc = 1.0, ss = 1.0;
    if (m >= n) {  // theta - pi
        m -= n;
        sc = -sc;
        ss = -ss;
    }
    if (2 * m > n) {  // pi - theta
        m = n - m;
        sc = -sc;
    }
    // theta = pi m / n in [0, pi/2]
    double cv, sv;
    if (4 * m > n) {  // theta = pi/2 - phi, phi = pi (n - 2m) / (2n) in [0, pi/4)
        const double phi = M_PI * (double)(n - 2 * m) / (double)(2 * n);
        cv = std::sin(phi);
        sv = std::cos(phi);
    } else {
        const double th = M_PI * (double)m / (double)n;
        cv = std::cos(th);
        sv = std::sin(th);
    }
    *c = sc * cv;
    *s = ss * sv;
}

// Compensated (Neumaier) summation.
struct KahanSum {
    double s = 0.0, c = 0.0;
    void add(double v) {
        const double t = s + v;
        if (std::fabs(s) >= std::fabs(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
    double value() const { return s + c; }
};

// In-place iterative radix-2 FFT (forward, e^{-2 pi i jk/L}) of L = 2^k complex
// values, FP64, with exactly reduced twiddles.
void fft_pow2(std::vector<double>& re, std::vector<double>& im) {
    const int L = (int)re.size();
    for (int i = 1, j = 0; i < L; ++i) {
        int bit = L >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            std::swap(re[i], re[j]);
            std::swap(im[i], im[j]);
        }
    }
    for (int len = 2; len <= L; len <<= 1) {
        const int half = len >> 1;
        for (int k = 0; k < half; ++k) {
            double c, s;
            sincospi_frac(2LL * k, len, &c, &s);  // angle 2 pi k / len
            const double wr = c, wi = -s;
            for (int i = k; i < L; i += len) {
                const double xr = re[i + half] * wr - im[i + half] * wi;
                const double xi = re[i + half] * wi + im[i + half] * wr;
                re[i + half] = re[i] - xr;
                im[i + half] = im[i] - xi;
                re[i] += xr;
                im[i] += xi;
            }
        }
    }
}

}  // namespace

int padded_length(int n) {
    int L = 4;
    while (L < 2 * n - 1) L <<= 1;
    return L;
}

void compute_axis_padded(const AxisHost& T, double tau, AxisPadded* P) {
    const int n = T.n;
    const int L = padded_length(n);
    P->n = n;
    P->L = L;
    std::vector<double> cs(2 * n), sn(2 * n);
    for (int m = 0; m < 2 * n; ++m) sincospi_frac(m, n, &cs[m], &sn[m]);
    // First columns of e^{t C} - I and e^{tau S} - I from expm1 of the spectra:
    //   g_d = (1/n) sum_j expm1(t lambda_j) cos(2 pi j d / n),     d = 0 .. n-1
    //   h_d = (1/n) sum_j expm1(tau mu_j) cos(pi d (2j - 1) / n),  d = 0 .. n-1 (h_{-d} = h_d)
    // (the identity's share sum_j cos(...) vanishes for d != 0 mod n).
    std::vector<double> xc(n), xs(n), g1(n), h1(n);
    for (int j = 0; j < n; ++j) {
        xc[j] = std::expm1(0.5 * tau * T.lambda[j]);
        xs[j] = std::expm1(tau * T.mu[j]);
    }
    const int two_n = 2 * n;
    for (int d = 0; d < n; ++d) {
        KahanSum sg, sh;
        // indices (2jd) mod 2n and d(2j - 1) mod 2n, stepped in j (stride 2d)
        const int step = (2 * d) % two_n;
        int mg = 0, mh = (two_n - d % two_n) % two_n;
        for (int j = 0; j < n; ++j) {
            sg.add(xc[j] * cs[mg]);
            sh.add(xs[j] * cs[mh]);
            mg += step;
            if (mg >= two_n) mg -= two_n;
            mh += step;
            if (mh >= two_n) mh -= two_n;
        }
        g1[d] = sg.value() / n;
        h1[d] = sh.value() / n;
    }
    // Padded, symmetric columns: offset d in (-n, n) at index d mod L. The
    // circulant part repeats its column with period n (c_d = g_{d mod n}).
    auto spectrum = [&](const std::vector<double>& col, bool circulant, double diag_add, std::vector<double>* out) {
        std::vector<double> re(L, 0.0), im(L, 0.0);
        for (int d = -(n - 1); d <= n - 1; ++d) {
            const int src = circulant ? ((d % n) + n) % n : (d < 0 ? -d : d);
            re[(d % L + L) % L] = col[src];
        }
        re[0] += diag_add;
        fft_pow2(re, im);
        out->resize(L);
        for (int k = 0; k < L; ++k) (*out)[k] = re[k] / (double)L;  // real: the column is symmetric
    };
    spectrum(T.bcol, false, 0.0, &P->mB);
    spectrum(g1, true, 1.0, &P->mC);
    spectrum(h1, false, 1.0, &P->mS);
    spectrum(g1, true, 0.0, &P->mC1);
    spectrum(h1, false, 0.0, &P->mS1);
    P->twid.resize(2 * L);
    for (int k = 0; k < L; ++k) {
        double c, s;
        sincospi_frac(2LL * k, L, &c, &s);
        P->twid[2 * k] = c;
        P->twid[2 * k + 1] = -s;
    }
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Tables of one axis: omega_k by eqs. (g_coe), (omega_coe); b_k by eq. (B);
// c_k, s_k by eqs. (C), (S); spectra by Remark 1; exponentials for tau.
void compute_axis(double alpha, double eps, double tau, double a, double b, int n, AxisHost* T) {
    T->n = n;
    const double h = (b - a) / (double)(n + 1);
    // g_{k+1} = (1 - (alpha+1)/(k+1)) g_k; omega_0 = alpha/2 g_0;
    // omega_{k+1} = alpha/2 g_{k+1} + (2-alpha)/2 g_k
    std::vector<double> g(n + 2), w(n + 2);
    g[0] = 1.0;
    for (int k = 0; k + 1 < n + 2; ++k) g[k + 1] = (1.0 - (alpha + 1.0) / (double)(k + 1)) * g[k];
    w[0] = 0.5 * alpha * g[0];
    for (int k = 0; k + 1 < n + 2; ++k) w[k + 1] = 0.5 * alpha * g[k + 1] + 0.5 * (2.0 - alpha) * g[k];
    // B = r (D + D^T), r = -eps^2 / (2 h^alpha cos(alpha pi / 2)) > 0:
    // b_0 = 2 r omega_1, b_1 = r (omega_0 + omega_2), b_k = r omega_{k+1} (k >= 2).
    const double r = -eps * eps / (2.0 * std::pow(h, alpha) * std::cos(alpha * M_PI / 2.0));
    T->bcol.assign(n, 0.0);
    T->bcol[0] = 2.0 * r * w[1];
    if (n > 1) T->bcol[1] = r * (w[0] + w[2]);
    for (int k = 2; k < n; ++k) T->bcol[k] = r * w[k + 1];
    // B is symmetric, b_{-k} = b_k, so b_{k-m+1} = b_{-(n-k)} = b_{n-k} with n = m-1:
    // c_k = (b_k + b_{n-k}) / 2, s_k = (b_k - b_{n-k}) / 2 (k >= 1), c_0 = s_0 = b_0 / 2.
    T->cfirst.assign(n, 0.0);
    T->sfirst.assign(n, 0.0);
    T->cfirst[0] = 0.5 * T->bcol[0];
    T->sfirst[0] = 0.5 * T->bcol[0];
    for (int k = 1; k < n; ++k) {
        T->cfirst[k] = 0.5 * (T->bcol[k] + T->bcol[n - k]);
        T->sfirst[k] = 0.5 * (T->bcol[k] - T->bcol[n - k]);
    }
    // cos / sin of pi m / n for m in [0, 2n)
    std::vector<double> cs(2 * n), sn(2 * n);
    for (int m = 0; m < 2 * n; ++m) sincospi_frac(m, n, &cs[m], &sn[m]);
    // lambda_j = sum_k c_k e^{-2 pi i jk/n}; mu_j = sum_k s_k e^{i pi k/n} e^{-2 pi i jk/n}
    //         = sum_k s_k e^{-i pi k (2j-1)/n}. Both are real because C and S are
    // symmetric (c_k = c_{n-k}, s_{-k} = -s_{n-k}); the real parts are summed.
    T->lambda.assign(n, 0.0);
    T->mu.assign(n, 0.0);
    // The angle indices (2jk) mod 2n and k(2j - 1) mod 2n advance by fixed
    // strides in k; they are stepped instead of recomputed with a division.
    const int two_n = 2 * n;
    for (int j = 0; j < n; ++j) {
        KahanSum sl, sm;
        const int dl = (2 * j) % two_n;
        const int dm = ((2 * j - 1) % two_n + two_n) % two_n;
        int ml = 0, mm = 0;
        for (int k = 0; k < n; ++k) {
            sl.add(T->cfirst[k] * cs[ml]);
            sm.add(T->sfirst[k] * cs[mm]);
            ml += dl;
            if (ml >= two_n) ml -= two_n;
            mm += dm;
            if (mm >= two_n) mm -= two_n;
        }
        T->lambda[j] = sl.value();
        T->mu[j] = sm.value();
    }
    // Factors with the inverse-FFT normalisation 1/n folded in.
    T->eC.resize(n);
    T->eS.resize(n);
    T->dC.resize(n);
    T->dS.resize(n);
    for (int j = 0; j < n; ++j) {
        T->eC[j] = std::exp(0.5 * tau * T->lambda[j]) / (double)n;
        T->eS[j] = std::exp(tau * T->mu[j]) / (double)n;
        T->dC[j] = std::expm1(0.5 * tau * T->lambda[j]) / (double)n;
        T->dS[j] = std::expm1(tau * T->mu[j]) / (double)n;
    }
    // Twist e^{i pi k/n} and FFT twiddles e^{-2 pi i m/n}.
    T->twist.resize(2 * n);
    T->twid.resize(2 * n);
    for (int k = 0; k < n; ++k) {
        T->twist[2 * k] = cs[k];
        T->twist[2 * k + 1] = sn[k];
        T->twid[2 * k] = cs[(2 * k) % (2 * n)];
        T->twid[2 * k + 1] = -sn[(2 * k) % (2 * n)];
    }
}



// Ratio twiddles (sfac_fft.cuh, FftPassRatio). For pass span P and radix RAD:
// c_r + i s_r = e^{-2 pi i r k / (P RAD)}. A cosine that is exactly 0 (w = -+i)
// is stored as 2^-60 with rho = s / 2^-60 exact: c t then equals s times the
// other part to within 2^-60 of |a|, far below the rounding of the sums.
std::vector<double> ratio_twiddles(int N, int E) {
    std::vector<double> out;
    for (int P = 1; P < N;) {
        const int RAD = (P * E <= N) ? E : N / P;
        if (P > 1) {
            for (int k = 0; k < P; ++k) {
                double c[16] = {}, s[16] = {}, rho[16] = {};
                for (int r = 0; r < RAD; ++r) {
                    double cv, sv;
                    sincospi_frac(2LL * r * k, (long long)P * RAD, &cv, &sv);
                    c[r] = cv == 0.0 ? std::ldexp(1.0, -60) : cv;
                    s[r] = -sv;
                    rho[r] = s[r] / c[r];
                }
                if (RAD == 16) {
                    // DftRatio16 (sfac_fft.cuh): rho_1..rho_15; g(S, R0) = c_{R0+S}/c_R0
                    // (c_0 = 1) at 15 + S - 1 + R0; h = g/sqrt 2 of the nodes (1,0),
                    // (2,0), (2,1); g(1,0) cos(pi/8); padding
                    double rec[36] = {};
                    for (int r = 1; r < 16; ++r) rec[r - 1] = rho[r];
                    for (int S = 1; S <= 8; S *= 2)
                        for (int R0 = 0; R0 < S; ++R0)
                            rec[15 + S - 1 + R0] = (R0 == 0 ? c[S] : c[R0 + S] / c[R0]);
                    const long double rs2 = sqrtl(0.5L), cp8 = cosl(3.14159265358979323846264338327950288L / 8);
                    rec[30] = (double)((long double)rec[15] * rs2);
                    rec[31] = (double)((long double)rec[16] * rs2);
                    rec[32] = (double)((long double)rec[17] * rs2);
                    rec[33] = (double)((long double)rec[15] * cp8);
                    out.insert(out.end(), rec, rec + 36);
                } else if (RAD == 8) {
                    const double rec[16] = {rho[1], rho[2], rho[3], rho[4], rho[5], rho[6], rho[7], c[4],
                                            c[6] / c[2], c[5] / c[1], c[7] / c[3], c[3] / c[1],
                                            c[2], c[1], (double)((long double)c[1] * sqrtl(0.5L)), 0.0};
                    out.insert(out.end(), rec, rec + 16);
                } else if (RAD == 4) {
                    const double rec[8] = {rho[1], rho[2], rho[3], c[2], c[3] / c[1], c[1], 0.0, 0.0};
                    out.insert(out.end(), rec, rec + 8);
                } else {
                    out.push_back(rho[1]);
                    out.push_back(c[1]);
                }
            }
        }
        P *= RAD;
    }
    return out;
}

}  // namespace sfac
