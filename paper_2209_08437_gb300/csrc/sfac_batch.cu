// sfac_batch.cu - host side of the batched persistent runner (sfac_batch_* in
// sfac.h): per-instance FP64 tables, the phase schedule, scratch counters, the
// persistent launch and its autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "sfac.h"
#include "sfac_batch_launch.h"
#include "sfac_host.h"
#include "sfac_internal.h"

namespace {

sfac_status bfail(sfac_status st, const std::string& msg) {
    sfac::set_last_error(msg);
    return st;
}

sfac_status bcuda(cudaError_t err, const char* what) {
    return bfail(SFAC_ECUDA, std::string(what) + ": " + cudaGetErrorString(err));
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Kernel shapes the autotuner chooses from: warps per CTA x values per thread
// for N <= 256 (radix-8 or radix-16 passes) x warp-groups per item. Shapes of
// up to 4 warps run a kernel built for three resident CTAs (at most 168
// registers: more warps, some spilling at N >= 256), 8-warp shapes one built
// for one CTA (no register cap).
struct BatchConfig {
    int wpb, es, mult;
};
const BatchConfig kConfigs[] = {
    {4, 16, 1}, {2, 16, 1}, {8, 16, 1}, {8, 16, 4}, {8, 8, 1}, {4, 16, 2},
    {8, 16, 2}, {4, 8, 2},  {8, 8, 2},  {4, 16, 4}, {8, 8, 4},  {2, 16, 2},
};
constexpr int kNumConfigs = sizeof(kConfigs) / sizeof(kConfigs[0]);

// Strided items of 256+ points are staged in shared memory (FP32, 8-warp
// shapes of >= 2 groups, which run one CTA per SM anyway: smaller CTAs would
// lose resident CTAs to the buffers); the launch provides the buffers only if
// some instance has such a pass.
int stage_of(int prec, const BatchConfig& c, bool long_strided) {
    return (prec == SFAC_FP32 && c.wpb == 8 && c.mult >= 2 && long_strided) ? c.mult : 0;
}

cudaError_t setup_batch(int prec, const BatchConfig& c, int stage, int sms, int* grid) {
    return prec == SFAC_FP64 ? sfac::setup_batch_f64(c.wpb, c.es, 0, sms, grid)
                             : sfac::setup_batch_f32(c.wpb, c.es, stage, sms, grid);
}

cudaError_t dispatch_batch(int prec, const BatchConfig& c, int grid, const sfac::BatchSchedule& sc, cudaStream_t s) {
    return prec == SFAC_FP64 ? sfac::launch_batch_f64(c.wpb, c.es, grid, sc, s)
                             : sfac::launch_batch_f32(c.wpb, c.es, grid, sc, s);
}

}  // namespace

struct sfac_batch {
    int count = 0;
    int prec = SFAC_FP32;
    int device = 0;
    int sms = 0;
    std::vector<sfac_params> params;
    void* dev_tables = nullptr;
    void* dev_common = nullptr;  // twiddles and twists per length (make_common_tables)
    std::vector<sfac::BatchInst> inst;  // tables filled at creation; fields and steps at prepare
    void* dev_sched = nullptr;          // instance array + schedule arrays
    size_t sched_cap = 0;
    unsigned long long* dev_scratch = nullptr;  // counter, done[count], error
    int* host_error = nullptr;                  // pinned copy of the error flag
    sfac::BatchSchedule sched{};
    int grid = 0;
    bool prepared = false;
    int config = 0;
    long long spin_limit = 20000000;  // ~2 s of 100 ns polls
    int hold_instance = -1;
    std::vector<void*> fields;
    std::vector<long long> nsteps;
};

namespace {
struct BatchDeleter {
    void operator()(sfac_batch* B) const { sfac_batch_destroy(B); }
};
}  // namespace

namespace {

sfac_status check_params(const sfac_params& p, int prec0) {
    if (p.dim != 2 && p.dim != 3) return bfail(SFAC_EUNSUPPORTED, "batch instances must be 2D or 3D");
    if (p.reserved != 0) return bfail(SFAC_EINVAL, "reserved field must be 0");
    if (p.prec != prec0) return bfail(SFAC_EINVAL, "all batch instances must share one precision");
    if (p.prec != SFAC_FP64 && p.prec != SFAC_FP32) return bfail(SFAC_EINVAL, "bad precision");
    if (!(std::isfinite(p.eps) && p.eps > 0) || !(std::isfinite(p.tau) && p.tau > 0))
        return bfail(SFAC_EINVAL, "eps and tau must be finite and > 0");
    if (!(std::isfinite(p.a) && std::isfinite(p.b) && p.b > p.a)) return bfail(SFAC_EINVAL, "need finite a < b");
    for (int l = 0; l < p.dim; ++l) {
        if (!(p.alpha[l] > 1.0 && p.alpha[l] < 2.0)) return bfail(SFAC_EINVAL, "alpha[l] must lie in (1, 2)");
        if (!sfac::is_pow2(p.n[l]) || p.n[l] < 32 || p.n[l] > 512)
            return bfail(SFAC_EUNSUPPORTED, "batch grid lengths must be powers of two in [32, 512]");
    }
    return SFAC_OK;
}

}  // namespace

namespace sfac {

// Items per pass of every instance for kernel shape `c` (lines per item follow
// from the values per thread the shape uses at that length).
void set_items(BatchInst& I, int es, int mult) {
    long long inner = 1;
    for (int a = 0; a < I.dim; ++a) {
        const int N = I.n[a];
        const long long outer = I.npts / ((long long)N * inner);
        const long long clines = a == 0 ? (outer + 1) / 2 : outer * (inner / 2);
        const int E = N >= 512 ? 16 : es;                     // values per thread
        const long long lpi = (long long)(32 * E / N) * mult;  // complex lines per item
        I.items[a] = (int)((clines + lpi - 1) / lpi);
        inner *= N;
    }
    for (int a = I.dim; a < 3; ++a) I.items[a] = 0;
}

// Build the phase schedule of `inst` into `blob` (the seven arrays below, each
// 256-byte aligned) and record its layout.
void pack_schedule(const std::vector<BatchInst>& inst, std::vector<unsigned char>& blob, ScheduleLayout* lay) {
    const int n_inst = (int)inst.size();
    long long max_steps = 0;
    for (const BatchInst& I : inst) max_steps = std::max<long long>(max_steps, I.steps);
    std::vector<long long> phase_base(1, 0), phase_first(1, 0), slot_cum;
    std::vector<int> phase_step, phase_axis, slot_inst;
    // Within a phase the slots go by line length, longest first (then by
    // instance): the warps running at one time then mostly execute the pass
    // body of one length, instead of all of them at once, which thrashed the
    // instruction cache when sizes were interleaved.
    std::vector<int> order[3];
    for (int a = 0; a < 3; ++a) {
        order[a].resize(n_inst);
        for (int i = 0; i < n_inst; ++i) order[a][i] = i;
        std::stable_sort(order[a].begin(), order[a].end(), [&](int x, int y) {
            const int nx = a < inst[x].dim ? inst[x].n[a] : 0, ny = a < inst[y].dim ? inst[y].n[a] : 0;
            return nx > ny;
        });
    }
    for (long long s = 0; s < max_steps; ++s) {
        for (int a = 0; a < 3; ++a) {
            long long cum = 0;
            for (int q = 0; q < n_inst; ++q) {
                const int i = order[a][q];
                const BatchInst& I = inst[i];
                if (s < I.steps && a < I.dim) {
                    cum += I.items[a];
                    slot_inst.push_back(i);
                    slot_cum.push_back(cum);
                }
            }
            if (cum == 0) continue;
            phase_step.push_back((int)s);
            phase_axis.push_back(a);
            phase_base.push_back(phase_base.back() + cum);
            phase_first.push_back((long long)slot_inst.size());
        }
    }
    // One device block: instances, phase_base, phase_first, slot_cum (8-byte
    // arrays), then phase_step, phase_axis, slot_inst (4-byte arrays).
    const size_t sz_inst = sizeof(BatchInst) * std::max(n_inst, 1);
    const size_t sizes[7] = {sz_inst, 8 * phase_base.size(), 8 * phase_first.size(),
                             8 * std::max<size_t>(slot_cum.size(), 1), 4 * std::max<size_t>(phase_step.size(), 1),
                             4 * std::max<size_t>(phase_axis.size(), 1), 4 * std::max<size_t>(slot_inst.size(), 1)};
    size_t total = 0;
    for (int q = 0; q < 7; ++q) {
        lay->off[q] = total;
        total += align256(sizes[q]);
    }
    lay->total = total;
    lay->nphase = (int)phase_step.size();
    lay->total_items = phase_base.back();
    blob.assign(total, 0);
    const size_t* off = lay->off;
    if (n_inst) std::memcpy(blob.data() + off[0], inst.data(), sizeof(BatchInst) * n_inst);
    std::memcpy(blob.data() + off[1], phase_base.data(), 8 * phase_base.size());
    std::memcpy(blob.data() + off[2], phase_first.data(), 8 * phase_first.size());
    if (!slot_cum.empty()) std::memcpy(blob.data() + off[3], slot_cum.data(), 8 * slot_cum.size());
    if (!phase_step.empty()) std::memcpy(blob.data() + off[4], phase_step.data(), 4 * phase_step.size());
    if (!phase_axis.empty()) std::memcpy(blob.data() + off[5], phase_axis.data(), 4 * phase_axis.size());
    if (!slot_inst.empty()) std::memcpy(blob.data() + off[6], slot_inst.data(), 4 * slot_inst.size());
}

void bind_schedule(const ScheduleLayout& lay, void* dev, int mult, BatchSchedule* sc) {
    unsigned char* base = static_cast<unsigned char*>(dev);
    sc->inst = reinterpret_cast<const BatchInst*>(base + lay.off[0]);
    sc->phase_base = reinterpret_cast<const long long*>(base + lay.off[1]);
    sc->phase_first = reinterpret_cast<const long long*>(base + lay.off[2]);
    sc->slot_cum = reinterpret_cast<const long long*>(base + lay.off[3]);
    sc->phase_step = reinterpret_cast<const int*>(base + lay.off[4]);
    sc->phase_axis = reinterpret_cast<const int*>(base + lay.off[5]);
    sc->slot_inst = reinterpret_cast<const int*>(base + lay.off[6]);
    sc->nphase = lay.nphase;
    sc->mult = mult;
    sc->total_items = lay.total_items;
}

sfac_status upload_schedule(const std::vector<BatchInst>& inst, int mult, void** dev, size_t* cap,
                            BatchSchedule* sc, cudaStream_t st) {
    std::vector<unsigned char> blob;
    ScheduleLayout lay{};
    pack_schedule(inst, blob, &lay);
    const size_t total = lay.total;
    cudaError_t err;
    if (total > *cap) {
        if (*dev) {
            cudaStreamSynchronize(st);
            cudaFree(*dev);
            *dev = nullptr;
            *cap = 0;
        }
        err = cudaMalloc(dev, total);
        if (err != cudaSuccess) {
            cudaGetLastError();
            *dev = nullptr;
            return bfail(SFAC_ENOMEM, "cudaMalloc of the batch schedule failed");
        }
        *cap = total;
    }
    err = cudaMemcpyAsync(*dev, blob.data(), total, cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return bcuda(err, "schedule upload");
    bind_schedule(lay, *dev, mult, sc);
    return SFAC_OK;
}

sfac_status make_common_tables(int prec, void** dev) {
    *dev = nullptr;
    const bool f64 = prec == SFAC_FP64;
    const size_t rs = f64 ? sizeof(double) : sizeof(float);
    std::vector<unsigned char> blob((size_t)BATCH_COMMON_ELEMS * 2 * rs);
    try {
        for (int N = 32; N <= 512; N *= 2) {
            // the same routine as every instance's tables, so the values agree bit for bit
            AxisHost H;
            compute_axis(1.5, 0.1, 0.01, -1.0, 1.0, N, &H);
            const std::vector<double>* src[2] = {&H.twid, &H.twist};
            for (int q = 0; q < 2; ++q) {
                const size_t first = 2 * ((size_t)batch_common_offset(N) + (size_t)q * N);  // reals
                for (size_t k = 0; k < 2 * (size_t)N; ++k) {
                    const double v = (*src[q])[k];
                    if (f64) std::memcpy(blob.data() + (first + k) * rs, &v, rs);
                    else {
                        const float f = (float)v;
                        std::memcpy(blob.data() + (first + k) * rs, &f, rs);
                    }
                }
            }
        }
    } catch (const std::bad_alloc&) {
        return bfail(SFAC_ENOMEM, "host allocation failed");
    }
    cudaError_t err = cudaMalloc(dev, blob.size());
    if (err != cudaSuccess) {
        cudaGetLastError();
        *dev = nullptr;
        return bfail(SFAC_ENOMEM, std::string("cudaMalloc of the common tables: ") + cudaGetErrorString(err));
    }
    err = cudaMemcpy(*dev, blob.data(), blob.size(), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) {
        cudaFree(*dev);
        *dev = nullptr;
        return bcuda(err, "common table upload");
    }
    return SFAC_OK;
}

bool batch_shape(int index, int* wpb, int* es, int* mult) {
    if (index < 0 || index >= kNumConfigs) return false;
    *wpb = kConfigs[index].wpb;
    *es = kConfigs[index].es;
    *mult = kConfigs[index].mult;
    return true;
}

}  // namespace sfac

namespace {

// Build the instance descriptors and the phase schedule for the current fields,
// step counts and kernel config, and upload them.
sfac_status build_schedule(sfac_batch* B, cudaStream_t st) {
    const BatchConfig& c = kConfigs[B->config];
    const int n_inst = B->count;
    for (int i = 0; i < n_inst; ++i) {
        sfac::BatchInst& I = B->inst[i];
        I.u = B->fields[i];
        I.steps = (int)B->nsteps[i];
        sfac::set_items(I, c.es, c.mult);
    }
    sfac_status r = sfac::upload_schedule(B->inst, c.mult, &B->dev_sched, &B->sched_cap, &B->sched, st);
    if (r != SFAC_OK) return r;
    sfac::BatchSchedule& sc = B->sched;
    sc.counter = B->dev_scratch;
    sc.done = B->dev_scratch + 1;
    sc.error = reinterpret_cast<int*>(B->dev_scratch + 1 + n_inst);
    sc.spin_limit = B->spin_limit;
    sc.hold_instance = B->hold_instance;
    sc.common = B->dev_common;
    bool long_strided = false;
    for (const sfac::BatchInst& I : B->inst)
        for (int a = 1; a < I.dim; ++a) long_strided = long_strided || I.n[a] >= 256;
    sc.stage = stage_of(B->prec, c, long_strided);
    cudaError_t err = setup_batch(B->prec, c, sc.stage, B->sms, &B->grid);
    if (err != cudaSuccess) return bcuda(err, "batch kernel setup");
    B->prepared = true;
    return SFAC_OK;
}

sfac_status launch(sfac_batch* B, cudaStream_t st) {
    if (!B->prepared) return bfail(SFAC_EINVAL, "batch is not prepared (call sfac_batch_prepare)");
    const size_t scratch = sizeof(unsigned long long) * (size_t)(B->count + 2);
    cudaError_t err = cudaMemsetAsync(B->dev_scratch, 0, scratch, st);
    if (err != cudaSuccess) return bcuda(err, "scratch reset");
    if (B->sched.total_items > 0) {
        const BatchConfig& c = kConfigs[B->config];
        err = dispatch_batch(B->prec, c, B->grid, B->sched, st);
        if (err != cudaSuccess) return bcuda(err, "batch kernel launch");
    }
    err = cudaMemcpyAsync(B->host_error, B->sched.error, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (err != cudaSuccess) return bcuda(err, "error flag copy");
    return SFAC_OK;
}

}  // namespace

namespace sfac {

// The prepared run of B with its scratch counters at `scratch` (work counter,
// B->count completion counters, status word) instead of B's own; used by
// sfac_batch_launch_noalloc. Clears the counters, launches, copies the status.
sfac_status batch_launch_with_scratch(sfac_batch* B, unsigned long long* scratch, cudaStream_t st) {
    if (!B->prepared) return bfail(SFAC_EINVAL, "batch is not prepared (call sfac_batch_prepare)");
    BatchSchedule sc = B->sched;
    sc.counter = scratch;
    sc.done = scratch + 1;
    sc.error = reinterpret_cast<int*>(scratch + 1 + B->count);
    cudaError_t err = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (size_t)(B->count + 2), st);
    if (err != cudaSuccess) return bcuda(err, "scratch reset");
    if (sc.total_items > 0) {
        err = dispatch_batch(B->prec, kConfigs[B->config], B->grid, sc, st);
        if (err != cudaSuccess) return bcuda(err, "batch kernel launch");
    }
    err = cudaMemcpyAsync(B->host_error, sc.error, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (err != cudaSuccess) return bcuda(err, "error flag copy");
    return SFAC_OK;
}

// Runs fn(w, nth) for every share w in [0, nth): shares 1.. on host threads,
// share 0 and any share whose thread could not be started on the calling
// thread. Every started thread is joined before this returns or throws, and an
// exception thrown by a share is rethrown here (the first one), so no
// exception escapes a thread and no joinable thread is left behind.
template <class F>
void run_shares(unsigned nth, F fn) {
    std::vector<std::exception_ptr> errs(nth);
    auto share = [&](unsigned w) {
        try {
            fn(w, nth);
        } catch (...) {
            errs[w] = std::current_exception();
        }
    };
    std::vector<std::thread> pool;
    unsigned started = 1;
    try {
        pool.reserve(nth);
        for (; started < nth; ++started) pool.emplace_back(share, started);
    } catch (...) {
        // thread creation failed: the shares not started run below
    }
    share(0);
    for (unsigned w = started; w < nth; ++w) share(w);
    for (auto& t : pool) t.join();
    for (const auto& e : errs)
        if (e) std::rethrow_exception(e);
}

int batch_count(const sfac_batch* B) { return B->count; }
int batch_device(const sfac_batch* B) { return B->device; }

}  // namespace sfac

extern "C" {

sfac_status sfac_batch_create(const sfac_params* params, int count, void* stream, sfac_batch** out) try {
    if (!out) return bfail(SFAC_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || count < 1) return bfail(SFAC_EINVAL, "need params and count >= 1");
    for (int i = 0; i < count; ++i) {
        const sfac_status st = check_params(params[i], params[0].prec);
        if (st != SFAC_OK) return bfail(st, "instance " + std::to_string(i) + ": " + sfac_last_error());
    }
    // Owned here until it is handed out: every early return or exception below
    // releases what was allocated so far.
    std::unique_ptr<sfac_batch, BatchDeleter> owner(new (std::nothrow) sfac_batch());
    sfac_batch* B = owner.get();
    if (!B) return bfail(SFAC_ENOMEM, "host allocation failed");
    B->count = count;
    B->prec = params[0].prec;
    B->params.assign(params, params + count);
    cudaGetDevice(&B->device);
    cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, B->device);
    // FP64 precompute of every instance's axes, spread over host threads.
    std::vector<sfac::AxisHost> host((size_t)count * 3);
    sfac::run_shares(std::max(1u, std::min(16u, std::thread::hardware_concurrency())), [&](unsigned w, unsigned nth) {
        for (int i = (int)w; i < count; i += (int)nth) {
            const sfac_params& p = params[i];
            for (int a = 0; a < p.dim; ++a)
                sfac::compute_axis(p.alpha[a], p.eps, p.tau, p.a, p.b, p.n[a], &host[(size_t)i * 3 + a]);
        }
    });
    const bool f64 = B->prec == SFAC_FP64;
    const size_t rs = f64 ? sizeof(double) : sizeof(float);
    // Per instance and axis the two spectral factors; twists and twiddles depend
    // on the length only and live in the common block (make_common_tables).
    std::vector<size_t> off((size_t)count * 6, 0);
    size_t total = 0;
    for (int i = 0; i < count; ++i)
        for (int a = 0; a < params[i].dim; ++a) {
            const size_t n = (size_t)params[i].n[a];
            for (int q = 0; q < 2; ++q) {
                off[((size_t)i * 3 + a) * 2 + q] = total;
                total += align256(n * rs);
            }
        }
    std::vector<unsigned char> blob(total, 0);
    for (int i = 0; i < count; ++i)
        for (int a = 0; a < params[i].dim; ++a) {
            const sfac::AxisHost& H = host[(size_t)i * 3 + a];
            const std::vector<double>* src[2] = {f64 ? &H.eC : &H.dC, f64 ? &H.eS : &H.dS};
            for (int q = 0; q < 2; ++q) {
                unsigned char* dst = blob.data() + off[((size_t)i * 3 + a) * 2 + q];
                if (f64) {
                    std::memcpy(dst, src[q]->data(), src[q]->size() * sizeof(double));
                } else {
                    float* f = reinterpret_cast<float*>(dst);
                    for (size_t k = 0; k < src[q]->size(); ++k) f[k] = (float)(*src[q])[k];
                }
            }
        }
    {
        const sfac_status cs = sfac::make_common_tables(B->prec, &B->dev_common);
        if (cs != SFAC_OK) return cs;
    }
    cudaError_t err = cudaMalloc(&B->dev_tables, total);
    if (err == cudaSuccess)
        err = cudaMalloc(reinterpret_cast<void**>(&B->dev_scratch), sizeof(unsigned long long) * (size_t)(count + 2));
    if (err == cudaSuccess) err = cudaMallocHost(reinterpret_cast<void**>(&B->host_error), sizeof(int));
    if (err != cudaSuccess) {
        cudaGetLastError();
        return bfail(SFAC_ENOMEM, std::string("batch allocation: ") + cudaGetErrorString(err));
    }
    *B->host_error = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    err = cudaMemcpyAsync(B->dev_tables, blob.data(), total, cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return bcuda(err, "batch table upload");
    B->inst.resize(count);
    unsigned char* base = static_cast<unsigned char*>(B->dev_tables);
    for (int i = 0; i < count; ++i) {
        const sfac_params& p = params[i];
        sfac::BatchInst& I = B->inst[i];
        std::memset(&I, 0, sizeof(I));
        I.dim = p.dim;
        I.npts = 1;
        for (int a = 0; a < 3; ++a) {
            I.n[a] = a < p.dim ? p.n[a] : 1;
            I.npts *= I.n[a];
            for (int q = 0; q < 2; ++q) I.tab[a][q] = a < p.dim ? base + off[((size_t)i * 3 + a) * 2 + q] : nullptr;
        }
        I.jq[0] = std::exp(-p.tau);
        I.jq[1] = -std::expm1(-p.tau);
        I.jq[2] = std::exp(-2.0 * p.tau);
        I.jq[3] = -std::expm1(-2.0 * p.tau);
    }
    B->fields.assign(count, nullptr);
    B->nsteps.assign(count, 0);
    *out = owner.release();
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_batch_destroy(sfac_batch* B) try {
    if (!B) return SFAC_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != B->device) cudaSetDevice(B->device);
    cudaDeviceSynchronize();
    if (B->dev_tables) cudaFree(B->dev_tables);
    if (B->dev_common) cudaFree(B->dev_common);
    if (B->dev_sched) cudaFree(B->dev_sched);
    if (B->dev_scratch) cudaFree(B->dev_scratch);
    if (B->host_error) cudaFreeHost(B->host_error);
    if (prev >= 0 && prev != B->device) cudaSetDevice(prev);
    delete B;
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_batch_prepare(sfac_batch* B, void* const* u_dev, const long long* nsteps, void* stream) try {
    if (!B || !u_dev || !nsteps) return bfail(SFAC_EINVAL, "NULL argument");
    for (int i = 0; i < B->count; ++i) {
        if (!u_dev[i]) return bfail(SFAC_EINVAL, "field " + std::to_string(i) + " is NULL");
        if (reinterpret_cast<uintptr_t>(u_dev[i]) % 16 != 0) return bfail(SFAC_EINVAL, "fields must be 16-byte aligned");
        if (nsteps[i] < 0 || nsteps[i] > (1LL << 30)) return bfail(SFAC_EINVAL, "nsteps out of range");
        B->fields[i] = u_dev[i];
        B->nsteps[i] = nsteps[i];
    }
    return build_schedule(B, static_cast<cudaStream_t>(stream));
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_batch_launch(sfac_batch* B, void* stream) try {
    if (!B) return bfail(SFAC_EINVAL, "batch is NULL");
    return launch(B, static_cast<cudaStream_t>(stream));
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_batch_wait(sfac_batch* B, void* stream) try {
    if (!B) return bfail(SFAC_EINVAL, "batch is NULL");
    cudaError_t err = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (err != cudaSuccess) return bcuda(err, "batch synchronise");
    if (*B->host_error == sfac::SFAC_BATCH_TIMEOUT) return bfail(SFAC_ETIMEOUT, "a dependency wait gave up");
    if (*B->host_error != 0) return bfail(SFAC_ECUDA, "batch kernel reported an error");
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_batch_step(sfac_batch* B, void* const* u_dev, const long long* nsteps, void* stream) try {
    sfac_status st = sfac_batch_prepare(B, u_dev, nsteps, stream);
    if (st != SFAC_OK) return st;
    st = sfac_batch_launch(B, stream);
    if (st != SFAC_OK) return st;
    return sfac_batch_wait(B, stream);
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_batch_autotune(sfac_batch* B, int max_steps, void* stream, int* choice) try {
    if (!B || max_steps < 1) return bfail(SFAC_EINVAL, "need a batch and max_steps >= 1");
    if (!B->prepared) return bfail(SFAC_EINVAL, "prepare the batch with its fields first");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Work on copies of the fields, for min(nsteps, max_steps) steps per instance.
    const size_t rs = B->prec == SFAC_FP64 ? 8 : 4;
    std::vector<size_t> off(B->count);
    size_t total = 0;
    for (int i = 0; i < B->count; ++i) {
        off[i] = total;
        total += align256((size_t)B->inst[i].npts * rs);
    }
    void* tmp = nullptr;
    cudaError_t err = cudaMalloc(&tmp, total);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return bfail(SFAC_ENOMEM, "autotune scratch allocation failed");
    }
    const std::vector<void*> saved_fields = B->fields;
    const std::vector<long long> saved_steps = B->nsteps;
    const int saved_config = B->config;
    for (int i = 0; i < B->count; ++i) {
        B->fields[i] = static_cast<unsigned char*>(tmp) + off[i];
        B->nsteps[i] = std::min<long long>(saved_steps[i], max_steps);
        cudaMemcpyAsync(B->fields[i], saved_fields[i], (size_t)B->inst[i].npts * rs, cudaMemcpyDeviceToDevice, st);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_cfg = saved_config;
    sfac_status result = SFAC_OK;
    for (int c = 0; c < kNumConfigs && result == SFAC_OK; ++c) {
        B->config = c;
        result = build_schedule(B, st);
        if (result != SFAC_OK) break;
        result = launch(B, st);  // warm-up
        if (result == SFAC_OK) result = sfac_batch_wait(B, stream);
        if (result != SFAC_OK) break;
        cudaEventRecord(e0, st);
        result = launch(B, st);
        cudaEventRecord(e1, st);
        if (result == SFAC_OK) result = sfac_batch_wait(B, stream);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (result == SFAC_OK && ms < best) {
            best = ms;
            best_cfg = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(tmp);
    B->fields = saved_fields;
    B->nsteps = saved_steps;
    B->config = result == SFAC_OK ? best_cfg : saved_config;
    const sfac_status rebuilt = build_schedule(B, st);
    if (result != SFAC_OK) return result;
    if (choice) *choice = best_cfg;
    return rebuilt;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_batch_set_config(sfac_batch* B, int config) try {
    if (!B || config < 0 || config >= kNumConfigs) return bfail(SFAC_EINVAL, "bad batch or config index");
    B->config = config;
    B->prepared = false;
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_batch_get_config(const sfac_batch* B, int* config, int* warps_per_cta, int* values_per_thread,
                                  int* groups_per_item) try {
    if (!B) return bfail(SFAC_EINVAL, "batch is NULL");
    const BatchConfig& c = kConfigs[B->config];
    if (config) *config = B->config;
    if (warps_per_cta) *warps_per_cta = c.wpb;
    if (values_per_thread) *values_per_thread = c.es;
    if (groups_per_item) *groups_per_item = c.mult;
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

int sfac_batch_num_configs(void) { return kNumConfigs; }

sfac_status sfac_batch_set_wait_limit(sfac_batch* B, long long spin_limit, int hold_instance) try {
    if (!B || spin_limit < 1 || hold_instance < -1 || hold_instance >= B->count)
        return bfail(SFAC_EINVAL, "bad batch, limit or instance");
    B->spin_limit = spin_limit;
    B->hold_instance = hold_instance;
    B->prepared = false;
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

}  // extern "C"
