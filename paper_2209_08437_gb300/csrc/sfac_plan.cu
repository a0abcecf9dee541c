// sfac_plan.cu - host side of libsfac: parameter checks, the FP64 precompute of
// the per-axis tables, the device plan and the C ABI declared in sfac.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "sfac.h"
#include "sfac_diag.h"
#include "sfac_host.h"
#include "sfac_internal.h"
#include "sfac_steps.h"

using sfac::AxisHost;
using sfac::compute_axis;
using sfac::is_pow2;

namespace {

thread_local std::string g_last_error;

sfac_status fail(sfac_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

}  // namespace

namespace sfac {
void set_last_error(const std::string& msg) { g_last_error = msg; }

sfac_status abi_exception_status() noexcept {
    const char* what = "host resource error";
    try {
        throw;
    } catch (const std::bad_alloc&) {
        what = "host allocation failed";
    } catch (const std::exception& e) {
        what = e.what();
    } catch (...) {
    }
    try {
        g_last_error = what;
    } catch (...) {
    }
    return SFAC_ENOMEM;
}
}  // namespace sfac

namespace {

sfac_status cuda_fail(cudaError_t err, const char* what) {
    return fail(SFAC_ECUDA, std::string(what) + ": " + cudaGetErrorString(err));
}

sfac_status validate(const sfac_params* p, bool need_supported) {
    if (!p) return fail(SFAC_EINVAL, "params is NULL");
    if (p->dim < 1 || p->dim > 3) return fail(SFAC_EINVAL, "dim must be 1, 2 or 3");
    if (p->reserved != 0) return fail(SFAC_EINVAL, "reserved field must be 0");
    if (p->prec != SFAC_FP64 && p->prec != SFAC_FP32) return fail(SFAC_EINVAL, "prec must be SFAC_FP64 or SFAC_FP32");
    if (!(std::isfinite(p->eps) && p->eps > 0)) return fail(SFAC_EINVAL, "eps must be finite and > 0");
    if (!(std::isfinite(p->tau) && p->tau > 0)) return fail(SFAC_EINVAL, "tau must be finite and > 0");
    if (!(std::isfinite(p->a) && std::isfinite(p->b) && p->b > p->a)) return fail(SFAC_EINVAL, "need finite a < b");
    long long pts = 1;
    for (int l = 0; l < p->dim; ++l) {
        if (p->n[l] < 1) return fail(SFAC_EINVAL, "n[l] must be >= 1");
        if (!(p->alpha[l] > 1.0 && p->alpha[l] < 2.0)) return fail(SFAC_EINVAL, "alpha[l] must lie in (1, 2)");
        if (need_supported && p->n[l] < 2)
            return fail(SFAC_EUNSUPPORTED, "n[l] must be at least 2");
        if (need_supported && !(is_pow2(p->n[l]) && p->n[l] >= 4) && p->n[l] > 2048)
            return fail(SFAC_EUNSUPPORTED, "n[l] must be a power of two <= 4096 or any length <= 2048");
        if (need_supported && is_pow2(p->n[l]) && p->n[l] > 4096)
            return fail(SFAC_EUNSUPPORTED, "n[l] must be a power of two <= 4096 or any length <= 2048");
        pts *= p->n[l];
    }
    if (pts > (1LL << 34)) return fail(SFAC_EUNSUPPORTED, "grid too large");
    return SFAC_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

struct sfac_plan {
    sfac_params p;
    int device = 0;
    long long npts = 0;
    void* dev_tables = nullptr;
    struct Ax {
        const void* eC;
        const void* eS;
        const void* twist;
        const void* twid;
        const void* rtwid;  // FP64 ratio twiddles (CTA passes), else NULL
        int fft_len;  // N of the pass: n, or the padded length L
        bool padded;
        // FP64 diagnostic tables: lambda/N, mu/N, twist, twiddles (padded axes:
        // the multiplier of B, -, -, twiddles)
        const double* dA;
        const double* dB;
        const void* dtwist;
        const void* dtwid;
    } ax[3] = {};
    double3* diag_partial = nullptr;
    double* diag_out = nullptr;
    unsigned int* status = nullptr;       // SFAC_PASS_TIMEOUT bits set by the passes (device)
    unsigned int* bar = nullptr;          // grid barrier of the whole-call launch (device, 2 words)
    unsigned int* status_host = nullptr;  // pinned host copy of it
    long long wait_cycles = 4LL << 30;
    int hold = 0;
    double jq_half_E = 0, jq_half_1mE = 0, jq_full_E = 0, jq_full_1mE = 0;
    void* staging = nullptr;
};

namespace {

size_t real_size(const sfac_plan* P) { return P->p.prec == SFAC_FP64 ? sizeof(double) : sizeof(float); }

// Scoped switch to the plan's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Arguments of one pass along axis `ax` of the field u.
sfac::PassArgs pass_args(const sfac_plan* P, void* u, int ax, int jq_in, int jq_out) {
    long long inner = 1;
    for (int l = 0; l < ax; ++l) inner *= P->p.n[l];
    const int n = P->p.n[ax];
    sfac::PassArgs a;
    a.u = u;
    a.inner = inner;
    a.outer = P->npts / ((long long)n * inner);
    a.clines = (ax == 0) ? (a.outer + 1) / 2 : a.outer * ((inner + 1) / 2);
    a.nmem = n;
    a.eC = P->ax[ax].eC;
    a.eS = P->ax[ax].eS;
    a.twist = P->ax[ax].twist;
    a.twid = P->ax[ax].twid;
    a.rtwid = P->ax[ax].rtwid;
    a.jq_in = jq_in != 0;
    a.jq_in_E = jq_in == 2 ? P->jq_full_E : P->jq_half_E;
    a.jq_in_1mE = jq_in == 2 ? P->jq_full_1mE : P->jq_half_1mE;
    a.jq_out = jq_out != 0;
    a.jq_out_E = jq_out == 2 ? P->jq_full_E : P->jq_half_E;
    a.jq_out_1mE = jq_out == 2 ? P->jq_full_1mE : P->jq_half_1mE;
    a.status = P->status;
    a.wait_cycles = P->wait_cycles;
    a.hold = P->hold;
    return a;
}

// One pass along axis `ax`: in place on u, or (out != NULL, host_io) loading
// from u and storing to out, one of them host memory mapped into the device's
// address space.
sfac_status launch_axis(sfac_plan* P, void* u, int ax, int jq_in, int jq_out, cudaStream_t st,
                        void* out = nullptr, bool host_io = false) {
    sfac::PassArgs a = pass_args(P, u, ax, jq_in, jq_out);
    if (out) a.out_shift = (static_cast<char*>(out) - static_cast<char*>(u)) / (long long)real_size(P);
    a.host_io = host_io ? 1 : 0;
    const int N = P->ax[ax].fft_len;
    cudaError_t err;
    if (P->ax[ax].padded) {
        err = (P->p.prec == SFAC_FP64) ? sfac::launch_pass_padded_f64(N, a, st) : sfac::launch_pass_padded_f32(N, a, st);
    } else if (P->p.prec == SFAC_FP64) {
        err = sfac::launch_pass_f64(N, a, st);
    } else {
        err = sfac::launch_pass_staged_f32(N, a, st);
        if (err == cudaErrorNotSupported) err = sfac::launch_pass_f32(N, a, st);
    }
    if (err != cudaSuccess) return cuda_fail(err, "axis pass launch");
    return SFAC_OK;
}

// Small grids run a whole call of two or more steps in one cooperative launch
// (sfac_steps.cu): every axis a spectral pass of 32..256 points, at most 65536
// unknowns, and a grid that is resident at once on the device.
constexpr long long kStepsMaxPoints = 1LL << 16;

bool steps_shape(const sfac_plan* P) {
    if (P->npts > kStepsMaxPoints) return false;
    for (int ax = 0; ax < P->p.dim; ++ax) {
        const int N = P->ax[ax].fft_len;
        if (P->ax[ax].padded || N < 32 || N > 256) return false;
    }
    return true;
}

sfac::StepsArgs steps_args(const sfac_plan* P, void* u, long long nsteps) {
    sfac::StepsArgs g{};
    for (int ax = 0; ax < P->p.dim; ++ax) {
        g.ax[ax] = pass_args(P, u, ax, 0, 0);
        g.n[ax] = P->ax[ax].fft_len;
    }
    g.dim = P->p.dim;
    g.nsteps = nsteps;
    g.jq_half_E = P->jq_half_E;
    g.jq_half_1mE = P->jq_half_1mE;
    g.jq_full_E = P->jq_full_E;
    g.jq_full_1mE = P->jq_full_1mE;
    g.bar = P->bar;
    g.status = P->status;
    g.wait_cycles = P->wait_cycles;
    g.hold = P->hold;
    return g;
}

bool steps_used(const sfac_plan* P, long long nsteps) {
    return nsteps >= 2 && steps_shape(P) && sfac::steps_fit(P->p.prec, steps_args(P, nullptr, nsteps));
}

// nsteps whole steps on the device field u. host_in / host_out (host buffers
// mapped into the device's address space, same layout as u; nsteps >= 1 and
// the per-pass route): the first pass loads the field from host_in, the last
// one stores the result to host_out; u holds it in between. The passes run the
// same arithmetic on the same lines as in place, so the result is the same bits.
// sfac_step_host's route for the host buffer u_host (SFAC_HOST_*), and in
// *mapped its device address when the route maps it. Pinned host memory is
// mapped into the device's address space (unified addressing; over
// NVLink-C2C on GB300), so a pass can load from it or store to it directly.
// That pays off where the first and the last pass have lines enough to hide
// the link's latency: measured side by side on GB300 (e2e per step, copies vs
// mapped) 3D 128^3 FP64 0.94 -> 0.79 ms, 256^3 FP64 7.56 -> 6.25 ms, 256^3
// FP32 0.89 -> 0.77 ms, 100^3 FP64 1.10 -> 1.02 ms; but 2D 1024^2 FP64
// 0.52 -> 0.54 ms and 64^3 FP64 0.178 -> 0.190 ms (few lines: latency bound).
// Hence at least kHostRouteLines complex lines in both passes. An FP32 last
// pass of more than 512 points writes narrow rows (fewer than 4 lines a CTA;
// 2D 4096^2 FP32 1.38 -> 3.47 ms): the result then goes back by a copy.
constexpr long long kHostRouteLines = 4096;

int host_route(const sfac_plan* P, const void* u_host, long long nsteps, void** mapped) {
    *mapped = nullptr;
    const int d = P->p.dim;
    if (nsteps < 1 || steps_used(P, nsteps) || reinterpret_cast<uintptr_t>(u_host) % 16 != 0) return SFAC_HOST_COPY;
    if (pass_args(P, nullptr, 0, 0, 0).clines < kHostRouteLines ||
        pass_args(P, nullptr, d - 1, 0, 0).clines < kHostRouteLines)
        return SFAC_HOST_COPY;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, u_host) != cudaSuccess) {
        cudaGetLastError();
        return SFAC_HOST_COPY;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer || reinterpret_cast<uintptr_t>(at.devicePointer) % 16 != 0)
        return SFAC_HOST_COPY;
    *mapped = at.devicePointer;
    if (P->p.prec == SFAC_FP32 && P->ax[d - 1].fft_len > 512) return SFAC_HOST_MAPPED_IN;
    return SFAC_HOST_MAPPED;
}

sfac_status run_steps(sfac_plan* P, void* u, long long nsteps, cudaStream_t st, void* host_in = nullptr,
                      void* host_out = nullptr) {
    const int d = P->p.dim;
    if (!host_in && !host_out && steps_used(P, nsteps)) {
        const cudaError_t err = sfac::launch_steps(P->p.prec, steps_args(P, u, nsteps), st);
        if (err != cudaSuccess) return cuda_fail(err, "small-grid launch");
        return SFAC_OK;
    }
    for (long long s = 0; s < nsteps; ++s) {
        // J^Q_{tau/2} opens the first step and closes the last one; between two
        // steps of one call the closing and opening halves act as one J^Q_{tau}.
        const bool last = (s == nsteps - 1);
        for (int ax = 0; ax < d; ++ax) {
            const int jin = (ax == 0 && s == 0) ? 1 : 0;
            const int jout = (ax == d - 1) ? (last ? 1 : 2) : 0;
            const bool from_host = host_in && s == 0 && ax == 0, to_host = host_out && last && ax == d - 1;
            void* src = from_host ? host_in : u;
            void* dst = to_host ? host_out : u;
            const sfac_status r = launch_axis(P, src, ax, jin, jout, st, dst == src ? nullptr : dst,
                                              from_host || to_host);
            if (r != SFAC_OK) return r;
        }
    }
    return SFAC_OK;
}

}  // namespace

extern "C" {

int sfac_version(void) { return 100; }

const char* sfac_last_error(void) { return g_last_error.c_str(); }

sfac_status sfac_plan_tables(const sfac_params* params, int axis, double* lambda, double* mu,
                             double* bcol, double* jq) try {
    sfac_status st = validate(params, false);
    if (st != SFAC_OK) return st;
    if (axis < 0 || axis >= params->dim) return fail(SFAC_EINVAL, "axis out of range");
    AxisHost T;
    try {
        compute_axis(params->alpha[axis], params->eps, params->tau, params->a, params->b, params->n[axis], &T);
    } catch (const std::bad_alloc&) {
        return fail(SFAC_ENOMEM, "host allocation failed");
    }
    const int n = params->n[axis];
    if (lambda) std::memcpy(lambda, T.lambda.data(), sizeof(double) * n);
    if (mu) std::memcpy(mu, T.mu.data(), sizeof(double) * n);
    if (bcol) std::memcpy(bcol, T.bcol.data(), sizeof(double) * n);
    if (jq) {
        jq[0] = std::exp(-params->tau);
        jq[1] = -std::expm1(-params->tau);
        jq[2] = std::exp(-2.0 * params->tau);
        jq[3] = -std::expm1(-2.0 * params->tau);
    }
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_plan_create(const sfac_params* params, void* stream, sfac_plan** out) try {
    if (!out) return fail(SFAC_EINVAL, "out is NULL");
    *out = nullptr;
    sfac_status st = validate(params, true);
    if (st != SFAC_OK) return st;
    sfac_plan* P = new (std::nothrow) sfac_plan();
    if (!P) return fail(SFAC_ENOMEM, "host allocation failed");
    P->p = *params;
    for (int l = params->dim; l < 3; ++l) P->p.n[l] = 1;
    P->npts = 1;
    for (int l = 0; l < params->dim; ++l) P->npts *= params->n[l];
    P->jq_half_E = std::exp(-params->tau);
    P->jq_half_1mE = -std::expm1(-params->tau);
    P->jq_full_E = std::exp(-2.0 * params->tau);
    P->jq_full_1mE = -std::expm1(-2.0 * params->tau);

    AxisHost host[3];
    sfac::AxisPadded pad[3];
    bool padded[3] = {false, false, false};
    try {
        long long inner = 1;
        for (int l = 0; l < params->dim; ++l) {
            compute_axis(params->alpha[l], params->eps, params->tau, params->a, params->b, params->n[l], &host[l]);
            // Zero-padded pass for lengths that are not powers of two >= 4, and for
            // any strided axis (l > 0) whose stride (the product of the earlier
            // extents) is odd: its column pairs are not 2-vector aligned.
            padded[l] = !(is_pow2(params->n[l]) && params->n[l] >= 4) || (l > 0 && (inner & 1));
            if (padded[l]) sfac::compute_axis_padded(host[l], params->tau, &pad[l]);
            inner *= params->n[l];
        }
    } catch (const std::bad_alloc&) {
        delete P;
        return fail(SFAC_ENOMEM, "host allocation failed");
    }
    cudaError_t err = cudaGetDevice(&P->device);
    if (err != cudaSuccess) {
        delete P;
        return cuda_fail(err, "cudaGetDevice");
    }
    // FP64 ratio twiddles of each axis's FFT length.
    std::vector<double> rtw[3];
    if (params->prec == SFAC_FP64) {
        try {
            for (int l = 0; l < params->dim; ++l) {
                const int N = padded[l] ? pad[l].L : params->n[l];
                const int E = sfac::f64_elems_per_thread(N);
                if (E <= 16) rtw[l] = sfac::ratio_twiddles(N, E);
            }
        } catch (const std::bad_alloc&) {
            delete P;
            return fail(SFAC_ENOMEM, "host allocation failed");
        }
    }
    // One device block: per axis eC[n], eS[n], twist[2n], twid[2n] reals, the
    // FP64 diagnostic tables, and the ratio twiddles.
    const size_t rs = real_size(P);
    size_t off[3][9], total = 0;
    long long max_partials = 1;
    {
        long long inner = 1;
        for (int l = 0; l < params->dim; ++l) {
            const size_t n = padded[l] ? (size_t)pad[l].L : (size_t)params->n[l];
            const size_t sz[9] = {n * rs, n * rs, padded[l] ? 0 : 2 * n * rs, 2 * n * rs,
                                  n * 8,  padded[l] ? 0 : n * 8, padded[l] ? 0 : 2 * n * 8, 2 * n * 8,
                                  rtw[l].size() * sizeof(double)};
            for (int q = 0; q < 9; ++q) {
                off[l][q] = total;
                total += align256(sz[q]);
            }
            const long long outer = P->npts / ((long long)params->n[l] * inner);
            const long long clines = l == 0 ? (outer + 1) / 2 : outer * ((inner + 1) / 2);
            max_partials = std::max(max_partials, sfac::diag_partials_needed(clines, (int)n));
            inner *= params->n[l];
        }
    }
    const size_t off_partial = total;
    total += align256(sizeof(double3) * (size_t)max_partials);
    const size_t off_out = total;
    total += align256(4 * sizeof(double));
    const size_t off_status = total;
    total += align256(sizeof(unsigned int));
    const size_t off_bar = total;
    total += align256(2 * sizeof(unsigned int));
    std::vector<unsigned char> blob;
    try {
        blob.assign(total, 0);
    } catch (const std::bad_alloc&) {
        delete P;
        return fail(SFAC_ENOMEM, "host allocation failed");
    }
    for (int l = 0; l < params->dim; ++l) {
        const bool f64 = params->prec == SFAC_FP64;
        const std::vector<double> none;
        const std::vector<double>* src[4] = {f64 ? &host[l].eC : &host[l].dC, f64 ? &host[l].eS : &host[l].dS,
                                             &host[l].twist, &host[l].twid};
        if (padded[l]) {
            src[0] = f64 ? &pad[l].mC : &pad[l].mC1;
            src[1] = f64 ? &pad[l].mS : &pad[l].mS1;
            src[2] = &none;
            src[3] = &pad[l].twid;
        }
        // FP64 diagnostic tables
        std::vector<double> lamN, muN;
        if (!padded[l]) {
            const double inv = 1.0 / (double)params->n[l];
            lamN.resize(params->n[l]);
            muN.resize(params->n[l]);
            for (int j = 0; j < params->n[l]; ++j) {
                lamN[j] = host[l].lambda[j] * inv;
                muN[j] = host[l].mu[j] * inv;
            }
        }
        const std::vector<double>* dsrc[4] = {padded[l] ? &pad[l].mB : &lamN, padded[l] ? &none : &muN,
                                              padded[l] ? &none : &host[l].twist,
                                              padded[l] ? &pad[l].twid : &host[l].twid};
        for (int q = 0; q < 4; ++q)
            if (!dsrc[q]->empty())
                std::memcpy(blob.data() + off[l][4 + q], dsrc[q]->data(), dsrc[q]->size() * sizeof(double));
        if (!rtw[l].empty())
            std::memcpy(blob.data() + off[l][8], rtw[l].data(), rtw[l].size() * sizeof(double));
        for (int q = 0; q < 4; ++q) {
            unsigned char* dst = blob.data() + off[l][q];
            const std::vector<double>& v = *src[q];
            if (rs == sizeof(double)) {
                std::memcpy(dst, v.data(), v.size() * sizeof(double));
            } else {
                float* f = reinterpret_cast<float*>(dst);
                for (size_t i = 0; i < v.size(); ++i) f[i] = (float)v[i];  // rounded once
            }
        }
    }
    err = cudaMalloc(&P->dev_tables, total);
    if (err != cudaSuccess) {
        delete P;
        cudaGetLastError();
        return fail(SFAC_ENOMEM, std::string("cudaMalloc of tables: ") + cudaGetErrorString(err));
    }
    cudaStream_t st_ = static_cast<cudaStream_t>(stream);
    err = cudaMemcpyAsync(P->dev_tables, blob.data(), total, cudaMemcpyHostToDevice, st_);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st_);
    if (err != cudaSuccess) {
        cudaFree(P->dev_tables);
        delete P;
        return cuda_fail(err, "table upload");
    }
    unsigned char* base = static_cast<unsigned char*>(P->dev_tables);
    for (int l = 0; l < params->dim; ++l) {
        P->ax[l].eC = base + off[l][0];
        P->ax[l].eS = base + off[l][1];
        P->ax[l].twist = padded[l] ? nullptr : base + off[l][2];
        P->ax[l].twid = base + off[l][3];
        P->ax[l].rtwid = rtw[l].empty() ? nullptr : base + off[l][8];
        P->ax[l].padded = padded[l];
        P->ax[l].fft_len = padded[l] ? pad[l].L : params->n[l];
        P->ax[l].dA = reinterpret_cast<const double*>(base + off[l][4]);
        P->ax[l].dB = padded[l] ? nullptr : reinterpret_cast<const double*>(base + off[l][5]);
        P->ax[l].dtwist = padded[l] ? nullptr : base + off[l][6];
        P->ax[l].dtwid = base + off[l][7];
    }
    P->diag_partial = reinterpret_cast<double3*>(base + off_partial);
    P->diag_out = reinterpret_cast<double*>(base + off_out);
    P->status = reinterpret_cast<unsigned int*>(base + off_status);
    P->bar = reinterpret_cast<unsigned int*>(base + off_bar);
    err = cudaMallocHost(reinterpret_cast<void**>(&P->status_host), sizeof(unsigned int));
    if (err != cudaSuccess) {
        cudaGetLastError();
        P->status_host = nullptr;
        cudaFree(P->dev_tables);
        delete P;
        return fail(SFAC_ENOMEM, std::string("cudaMallocHost of the status word: ") + cudaGetErrorString(err));
    }
    *P->status_host = 0;
    *out = P;
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_plan_destroy(sfac_plan* plan) try {
    if (!plan) return SFAC_OK;
    sfac_status st = SFAC_OK;
    {
        DeviceGuard g(plan->device);
        cudaError_t err = cudaDeviceSynchronize();
        if (err != cudaSuccess) st = cuda_fail(err, "synchronise before destroy");
        if (plan->dev_tables) cudaFree(plan->dev_tables);
        if (plan->staging) cudaFree(plan->staging);
        if (plan->status_host) cudaFreeHost(plan->status_host);
    }
    delete plan;
    return st;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_step(sfac_plan* plan, void* u_dev, long long nsteps, void* stream) try {
    if (!plan) return fail(SFAC_EINVAL, "plan is NULL");
    if (!u_dev) return fail(SFAC_EINVAL, "u_dev is NULL");
    if (nsteps < 0) return fail(SFAC_EINVAL, "nsteps must be >= 0");
    if (reinterpret_cast<uintptr_t>(u_dev) % 16 != 0) return fail(SFAC_EINVAL, "u_dev must be 16-byte aligned");
    if (nsteps == 0) return SFAC_OK;
    DeviceGuard g(plan->device);
    if (!g.ok) return fail(SFAC_ECUDA, "cannot select the plan's device");
    return run_steps(plan, u_dev, nsteps, static_cast<cudaStream_t>(stream));
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_axis_pass(sfac_plan* plan, void* u_dev, int axis, int jq_in, int jq_out, void* stream) try {
    if (!plan) return fail(SFAC_EINVAL, "plan is NULL");
    if (!u_dev) return fail(SFAC_EINVAL, "u_dev is NULL");
    if (axis < 0 || axis >= plan->p.dim) return fail(SFAC_EINVAL, "axis out of range");
    if (jq_in < 0 || jq_in > 2 || jq_out < 0 || jq_out > 2) return fail(SFAC_EINVAL, "jq mode must be 0, 1 or 2");
    if (reinterpret_cast<uintptr_t>(u_dev) % 16 != 0) return fail(SFAC_EINVAL, "u_dev must be 16-byte aligned");
    DeviceGuard g(plan->device);
    if (!g.ok) return fail(SFAC_ECUDA, "cannot select the plan's device");
    return launch_axis(plan, u_dev, axis, jq_in, jq_out, static_cast<cudaStream_t>(stream));
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_plan_info(const sfac_plan* plan, int axis, int* fft_len, int* padded) try {
    if (!plan || axis < 0 || axis >= plan->p.dim) return fail(SFAC_EINVAL, "bad plan or axis");
    if (fft_len) *fft_len = plan->ax[axis].fft_len;
    if (padded) *padded = plan->ax[axis].padded ? 1 : 0;
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_plan_kernel(const sfac_plan* plan, int axis, const void* u_dev, int* kind) try {
    if (!plan || axis < 0 || axis >= plan->p.dim || !kind) return fail(SFAC_EINVAL, "bad plan, axis or kind");
    long long inner = 1;
    for (int l = 0; l < axis; ++l) inner *= plan->p.n[l];
    const int N = plan->ax[axis].fft_len;
    sfac::PassArgs a;
    a.u = const_cast<void*>(u_dev);
    a.inner = inner;
    a.outer = plan->npts / ((long long)plan->p.n[axis] * inner);
    a.nmem = plan->p.n[axis];
    if (plan->p.prec == SFAC_FP32 && !plan->ax[axis].padded && sfac::staged_pass_eligible(N, a))
        *kind = SFAC_KERNEL_STAGED;
    else if (plan->p.prec == SFAC_FP32 && N >= 32 && N <= 512)
        *kind = SFAC_KERNEL_WARP;
    else
        *kind = SFAC_KERNEL_CTA;
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_plan_step_kernel(const sfac_plan* plan, long long nsteps, int* kind) try {
    if (!plan || !kind || nsteps < 0) return fail(SFAC_EINVAL, "need a plan, kind and nsteps >= 0");
    DeviceGuard g(plan->device);
    if (!g.ok) return fail(SFAC_ECUDA, "cannot select the plan's device");
    *kind = steps_used(plan, nsteps) ? SFAC_STEP_WHOLE : SFAC_STEP_PASSES;
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_plan_host_route(const sfac_plan* plan, const void* u_host, long long nsteps, int* route) try {
    if (!plan || !u_host || !route || nsteps < 0) return fail(SFAC_EINVAL, "need a plan, u_host, route and nsteps >= 0");
    DeviceGuard g(plan->device);
    if (!g.ok) return fail(SFAC_ECUDA, "cannot select the plan's device");
    void* mapped = nullptr;
    *route = host_route(plan, u_host, nsteps, &mapped);
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

// The status word already copied to plan->status_host and the stream
// synchronised: clear a recorded timeout and report it.
static sfac_status status_after_sync(sfac_plan* plan, cudaStream_t st) {
    if (*plan->status_host == 0) return SFAC_OK;
    *plan->status_host = 0;
    cudaError_t err = cudaMemsetAsync(plan->status, 0, sizeof(unsigned int), st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return cuda_fail(err, "status reset");
    return fail(SFAC_ETIMEOUT, "an axis pass gave up waiting for a staged tile copy; the field is not valid");
}

sfac_status sfac_plan_set_wait_limit(sfac_plan* plan, long long wait_cycles, int hold) try {
    if (!plan || wait_cycles < 1) return fail(SFAC_EINVAL, "need a plan and wait_cycles >= 1");
    plan->wait_cycles = wait_cycles;
    plan->hold = hold != 0;
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_plan_check(sfac_plan* plan, void* stream) try {
    if (!plan) return fail(SFAC_EINVAL, "plan is NULL");
    DeviceGuard g(plan->device);
    if (!g.ok) return fail(SFAC_ECUDA, "cannot select the plan's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t err = cudaMemcpyAsync(plan->status_host, plan->status, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return cuda_fail(err, "status read");
    return status_after_sync(plan, st);
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_diagnostics(sfac_plan* plan, const void* u_dev, double* out, void* stream) try {
    if (!plan || !u_dev || !out) return fail(SFAC_EINVAL, "NULL argument");
    if (reinterpret_cast<uintptr_t>(u_dev) % 16 != 0) return fail(SFAC_EINVAL, "u_dev must be 16-byte aligned");
    DeviceGuard g(plan->device);
    if (!g.ok) return fail(SFAC_ECUDA, "cannot select the plan's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t err = cudaMemsetAsync(plan->diag_out, 0, 3 * sizeof(double), st);
    if (err != cudaSuccess) return cuda_fail(err, "diagnostics reset");
    long long inner = 1;
    double hprod = 1.0;
    for (int ax = 0; ax < plan->p.dim; ++ax) {
        const int n = plan->p.n[ax];
        sfac::PassArgs a;
        a.u = const_cast<void*>(u_dev);
        a.inner = inner;
        a.outer = plan->npts / ((long long)n * inner);
        a.clines = (ax == 0) ? (a.outer + 1) / 2 : a.outer * ((inner + 1) / 2);
        a.nmem = n;
        a.eC = a.eS = nullptr;
        a.twist = plan->ax[ax].dtwist;
        a.twid = plan->ax[ax].dtwid;
        a.jq_in = a.jq_out = 0;
        a.jq_in_E = a.jq_in_1mE = a.jq_out_E = a.jq_out_1mE = 0.0;
        err = sfac::launch_diag_axis(plan->p.prec == SFAC_FP64, plan->ax[ax].padded, plan->ax[ax].fft_len, a,
                                     plan->ax[ax].dA, plan->ax[ax].dB, ax == 0, plan->diag_partial,
                                     plan->diag_out, st);
        if (err != cudaSuccess) return cuda_fail(err, "diagnostics launch");
        inner *= n;
        hprod *= (plan->p.b - plan->p.a) / (double)(n + 1);
    }
    double host[3];
    err = cudaMemcpyAsync(host, plan->diag_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return cuda_fail(err, "diagnostics copy");
    out[0] = host[2];                                 // max |u|
    out[1] = hprod * (0.25 * host[1] - 0.5 * host[0]);  // discrete energy
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_solve(sfac_plan* plan, void* u_dev, double T, void* stream) try {
    if (!plan) return fail(SFAC_EINVAL, "plan is NULL");
    if (!(std::isfinite(T) && T >= 0)) return fail(SFAC_EINVAL, "T must be finite and >= 0");
    const double q = T / plan->p.tau;
    const double r = std::nearbyint(q);
    if (std::fabs(q - r) > 1e-9 * std::fmax(1.0, q)) return fail(SFAC_EINVAL, "T is not a whole number of steps");
    return sfac_step(plan, u_dev, (long long)r, stream);
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_step_host(sfac_plan* plan, void* u_host, long long nsteps, void* stream) try {
    if (!plan) return fail(SFAC_EINVAL, "plan is NULL");
    if (!u_host) return fail(SFAC_EINVAL, "u_host is NULL");
    if (nsteps < 0) return fail(SFAC_EINVAL, "nsteps must be >= 0");
    DeviceGuard g(plan->device);
    if (!g.ok) return fail(SFAC_ECUDA, "cannot select the plan's device");
    const size_t bytes = (size_t)plan->npts * real_size(plan);
    cudaError_t err;
    if (!plan->staging) {
        err = cudaMalloc(&plan->staging, bytes);
        if (err != cudaSuccess) {
            plan->staging = nullptr;
            cudaGetLastError();
            return fail(SFAC_ENOMEM, std::string("cudaMalloc of staging buffer: ") + cudaGetErrorString(err));
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* mapped = nullptr;
    const int route = host_route(plan, u_host, nsteps, &mapped);
    if (route != SFAC_HOST_COPY) {
        // the first pass loads the field from the mapped buffer; the last one
        // stores the result there (SFAC_HOST_MAPPED) or into the device buffer
        sfac_status s = run_steps(plan, plan->staging, nsteps, st, mapped,
                                  route == SFAC_HOST_MAPPED ? mapped : nullptr);
        if (s != SFAC_OK) return s;
        if (route == SFAC_HOST_MAPPED_IN) {
            err = cudaMemcpyAsync(u_host, plan->staging, bytes, cudaMemcpyDeviceToHost, st);
            if (err != cudaSuccess) return cuda_fail(err, "device-to-host copy");
        }
    } else {
        err = cudaMemcpyAsync(plan->staging, u_host, bytes, cudaMemcpyHostToDevice, st);
        if (err != cudaSuccess) return cuda_fail(err, "host-to-device copy");
        sfac_status s = run_steps(plan, plan->staging, nsteps, st);
        if (s != SFAC_OK) return s;
        err = cudaMemcpyAsync(u_host, plan->staging, bytes, cudaMemcpyDeviceToHost, st);
        if (err != cudaSuccess) return cuda_fail(err, "device-to-host copy");
    }
    // the status word rides along: one synchronisation for both
    err = cudaMemcpyAsync(plan->status_host, plan->status, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
    if (err != cudaSuccess) return cuda_fail(err, "status read");
    err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return cuda_fail(err, "stream synchronise");
    return status_after_sync(plan, st);
} catch (...) {
    return sfac::abi_exception_status();
}

}  // extern "C"
