// sfac_server.cu - continuous batching of SFAC solves (sfac_server_* in sfac.h).
//
// A server owns one device arena. Each admitted request gets a slot: its field
// and its per-axis tables live in the arena until the result is fetched.
// Rounds advance every active slot by up to `chunk` steps in one persistent
// launch of the batch kernel (sfac_batch.cuh), so requests admitted while a
// round runs join a later round and their work overlaps on the device with
// everyone else's. Two rounds may be in flight: the host enqueues round k + 1
// behind round k (each round has its own schedule, scratch counters and status
// word) and collects round k's finished requests while round k + 1 runs, so
// the device does not wait for the host between rounds. Admission and result
// copies use an internal copy stream, so they overlap with the rounds.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "sfac.h"
#include "sfac_batch_launch.h"
#include "sfac_host.h"
#include "sfac_internal.h"

namespace {

sfac_status sfail(sfac_status st, const std::string& msg) {
    sfac::set_last_error(msg);
    return st;
}

sfac_status scuda(cudaError_t err, const char* what) {
    return sfail(SFAC_ECUDA, std::string(what) + ": " + cudaGetErrorString(err));
}

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Slot {
    bool used = false;
    sfac_params p{};
    sfac::BatchInst inst{};
    size_t off = 0, bytes = 0;  // arena allocation
    long long remaining = 0, done = 0;
    long long queued = 0;  // steps of rounds in flight
    bool failed = false;   // a round that advanced it gave up: no result
};

// First-fit allocator over [0, size) with coalescing frees.
struct Arena {
    std::map<size_t, size_t> free_blocks;  // offset -> size
    size_t total = 0, used = 0;
    void init(size_t size) {
        free_blocks.clear();
        free_blocks[0] = size;
        total = size;
        used = 0;
    }
    bool alloc(size_t bytes, size_t* off) {
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t noff = it->first + bytes;
                free_blocks.erase(it);
                if (rest) free_blocks[noff] = rest;
                used += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        auto it = free_blocks.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_blocks.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_blocks.erase(next);
        }
        if (it != free_blocks.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_blocks.erase(it);
            }
        }
        used -= bytes;
    }
    size_t largest_free() const {
        size_t m = 0;
        for (const auto& kv : free_blocks) m = std::max(m, kv.second);
        return m;
    }
};

size_t real_bytes(int prec) { return prec == SFAC_FP64 ? 8 : 4; }

// Arena bytes one request needs: its field and four tables per axis.
size_t request_bytes(const sfac_params& p) {
    const size_t rs = real_bytes(p.prec);
    size_t pts = 1;
    for (int a = 0; a < p.dim; ++a) pts *= (size_t)p.n[a];
    size_t b = al256(pts * rs);
    for (int a = 0; a < p.dim; ++a) b += 2 * al256((size_t)p.n[a] * rs);  // eC, eS per axis
    return b;
}

sfac_status check_request(const sfac_params* p, int prec) {
    if (!p) return sfail(SFAC_EINVAL, "params is NULL");
    if (p->dim != 2 && p->dim != 3) return sfail(SFAC_EUNSUPPORTED, "served problems must be 2D or 3D");
    if (p->reserved != 0) return sfail(SFAC_EINVAL, "reserved field must be 0");
    if (p->prec != prec) return sfail(SFAC_EINVAL, "request precision differs from the server's");
    if (!(std::isfinite(p->eps) && p->eps > 0) || !(std::isfinite(p->tau) && p->tau > 0))
        return sfail(SFAC_EINVAL, "eps and tau must be finite and > 0");
    if (!(std::isfinite(p->a) && std::isfinite(p->b) && p->b > p->a)) return sfail(SFAC_EINVAL, "need finite a < b");
    for (int l = 0; l < p->dim; ++l) {
        if (!(p->alpha[l] > 1.0 && p->alpha[l] < 2.0)) return sfail(SFAC_EINVAL, "alpha[l] must lie in (1, 2)");
        if (!sfac::is_pow2(p->n[l]) || p->n[l] < 32 || p->n[l] > 512)
            return sfail(SFAC_EUNSUPPORTED, "served grid lengths must be powers of two in [32, 512]");
    }
    return SFAC_OK;
}

struct Round {
    bool active = false;
    std::vector<int> slots;          // slots advanced by this round
    std::vector<long long> steps;    // and by how many steps each
    void* dev_sched = nullptr;       // schedule (device)
    size_t sched_cap = 0;
    unsigned char* host_sched = nullptr;  // pinned staging of the schedule upload
    size_t host_cap = 0;
    unsigned long long* scratch = nullptr;  // counter, done[max_slots], error
    int* host_error = nullptr;              // pinned copy of the error word
    cudaEvent_t done = nullptr;             // recorded after the kernel and the error copy
    sfac::BatchSchedule sc{};
};

constexpr int kRounds = 2;

}  // namespace

struct sfac_server {
    int device = 0, sms = 0, prec = SFAC_FP32;
    void* arena_mem = nullptr;
    Arena arena;
    std::vector<Slot> slots;
    cudaStream_t copy_stream = nullptr;
    void* dev_common = nullptr;  // twiddles and twists per length (make_common_tables)
    Round rounds[kRounds];
    long long launched = 0, completed = 0;  // rounds enqueued / waited for; in flight = launched - completed
    long long spin_limit = 20000000;
    int hold_slot = -1;  // test hook (sfac_server_set_wait_limit)
};

namespace {

sfac_status release_round_buffers(Round& R) {
    if (R.dev_sched) cudaFree(R.dev_sched);
    if (R.host_sched) cudaFreeHost(R.host_sched);
    if (R.scratch) cudaFree(R.scratch);
    if (R.host_error) cudaFreeHost(R.host_error);
    if (R.done) cudaEventDestroy(R.done);
    R = Round();
    return SFAC_OK;
}

// Grow the round's schedule buffers to `bytes` (device and pinned host). The
// round is not in flight; freeing the old device buffer may wait for the other
// round, which only happens when a round's schedule outgrows every earlier one.
cudaError_t reserve_schedule(Round& R, size_t bytes) {
    if (bytes <= R.sched_cap && bytes <= R.host_cap) return cudaSuccess;
    const size_t want = std::max(bytes, 2 * std::max(R.sched_cap, R.host_cap));
    if (R.dev_sched) cudaFree(R.dev_sched);
    if (R.host_sched) cudaFreeHost(R.host_sched);
    R.dev_sched = nullptr;
    R.host_sched = nullptr;
    R.sched_cap = R.host_cap = 0;
    cudaError_t err = cudaMalloc(&R.dev_sched, want);
    if (err == cudaSuccess) err = cudaMallocHost(reinterpret_cast<void**>(&R.host_sched), want);
    if (err != cudaSuccess) return err;
    R.sched_cap = R.host_cap = want;
    return cudaSuccess;
}

}  // namespace

extern "C" {

sfac_status sfac_server_create(size_t arena_bytes, int max_slots, int prec, void* stream, sfac_server** out) try {
    (void)stream;
    if (!out) return sfail(SFAC_EINVAL, "out is NULL");
    *out = nullptr;
    if (arena_bytes < 4096 || max_slots < 1 || (prec != SFAC_FP32 && prec != SFAC_FP64))
        return sfail(SFAC_EINVAL, "need arena_bytes >= 4096, max_slots >= 1 and a valid precision");
    sfac_server* S = new (std::nothrow) sfac_server();
    if (!S) return sfail(SFAC_ENOMEM, "host allocation failed");
    S->prec = prec;
    cudaGetDevice(&S->device);
    cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device);
    try {
        S->slots.resize(max_slots);
    } catch (...) {
        sfac_server_destroy(S);
        throw;
    }
    cudaError_t err = cudaMalloc(&S->arena_mem, arena_bytes);
    for (int r = 0; r < kRounds && err == cudaSuccess; ++r) {
        Round& R = S->rounds[r];
        err = cudaMalloc(reinterpret_cast<void**>(&R.scratch), sizeof(unsigned long long) * (size_t)(max_slots + 2));
        if (err == cudaSuccess) err = cudaMallocHost(reinterpret_cast<void**>(&R.host_error), sizeof(int));
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&R.done, cudaEventDisableTiming);
        if (err == cudaSuccess) *R.host_error = 0;
    }
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking);
    if (err != cudaSuccess) {
        cudaGetLastError();
        sfac_server_destroy(S);
        return sfail(SFAC_ENOMEM, std::string("server allocation: ") + cudaGetErrorString(err));
    }
    {
        const sfac_status cs = sfac::make_common_tables(prec, &S->dev_common);
        if (cs != SFAC_OK) {
            sfac_server_destroy(S);
            return cs;
        }
    }
    S->arena.init(arena_bytes);
    *out = S;
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_server_destroy(sfac_server* S) try {
    if (!S) return SFAC_OK;
    cudaDeviceSynchronize();
    if (S->arena_mem) cudaFree(S->arena_mem);
    for (Round& R : S->rounds) release_round_buffers(R);
    if (S->dev_common) cudaFree(S->dev_common);
    if (S->copy_stream) cudaStreamDestroy(S->copy_stream);
    delete S;
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_server_request_bytes(const sfac_params* params, size_t* bytes) try {
    if (!params || !bytes) return sfail(SFAC_EINVAL, "NULL argument");
    const sfac_status st = check_request(params, params->prec);
    if (st != SFAC_OK) return st;
    *bytes = request_bytes(*params);
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_server_admit(sfac_server* S, const sfac_params* params, const void* u0_host, long long nsteps,
                              int* slot_out) try {
    if (!S || !u0_host || !slot_out) return sfail(SFAC_EINVAL, "NULL argument");
    *slot_out = -1;
    sfac_status st = check_request(params, S->prec);
    if (st != SFAC_OK) return st;
    if (nsteps < 0 || nsteps > (1LL << 30)) return sfail(SFAC_EINVAL, "nsteps out of range");
    int slot = -1;
    for (int i = 0; i < (int)S->slots.size(); ++i)
        if (!S->slots[i].used) {
            slot = i;
            break;
        }
    if (slot < 0) return sfail(SFAC_ENOMEM, "no free slot");
    const size_t bytes = request_bytes(*params);
    size_t off = 0;
    if (!S->arena.alloc(bytes, &off)) return sfail(SFAC_ENOMEM, "device arena full");
    // From here on the arena block goes back on every path that does not admit.
    const sfac_params& p = *params;
    const bool f64 = p.prec == SFAC_FP64;
    const size_t rs = real_bytes(p.prec);
    size_t pts = 1;
    for (int a = 0; a < p.dim; ++a) pts *= (size_t)p.n[a];
    Slot s;
    s.inst.dim = p.dim;
    s.inst.npts = (long long)pts;
    unsigned char* base = static_cast<unsigned char*>(S->arena_mem) + off;
    try {
        // FP64 tables on the host, then one copy of field + tables into the arena.
        std::vector<unsigned char> blob(bytes, 0);
        size_t cur = al256(pts * rs);
        std::memcpy(blob.data(), u0_host, pts * rs);
        for (int a = 0; a < 3; ++a) {
            s.inst.n[a] = a < p.dim ? p.n[a] : 1;
            if (a >= p.dim) continue;
            sfac::AxisHost H;
            sfac::compute_axis(p.alpha[a], p.eps, p.tau, p.a, p.b, p.n[a], &H);
            const std::vector<double>* src[2] = {f64 ? &H.eC : &H.dC, f64 ? &H.eS : &H.dS};
            for (int q = 0; q < 2; ++q) {
                unsigned char* dst = blob.data() + cur;
                if (f64) {
                    std::memcpy(dst, src[q]->data(), src[q]->size() * sizeof(double));
                } else {
                    float* f = reinterpret_cast<float*>(dst);
                    for (size_t k = 0; k < src[q]->size(); ++k) f[k] = (float)(*src[q])[k];
                }
                s.inst.tab[a][q] = base + cur;
                cur += al256(src[q]->size() * rs);
            }
        }
        cudaError_t err = cudaMemcpyAsync(base, blob.data(), bytes, cudaMemcpyHostToDevice, S->copy_stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(S->copy_stream);
        if (err != cudaSuccess) {
            S->arena.release(off, bytes);
            return scuda(err, "request upload");
        }
    } catch (...) {
        S->arena.release(off, bytes);
        throw;
    }
    s.inst.u = base;
    s.inst.jq[0] = std::exp(-p.tau);
    s.inst.jq[1] = -std::expm1(-p.tau);
    s.inst.jq[2] = std::exp(-2.0 * p.tau);
    s.inst.jq[3] = -std::expm1(-2.0 * p.tau);
    s.used = true;
    s.p = p;
    s.off = off;
    s.bytes = bytes;
    s.remaining = nsteps;
    s.done = 0;
    S->slots[slot] = s;
    *slot_out = slot;
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_server_round(sfac_server* S, long long chunk, int shape, void* stream, int* launched) try {
    if (launched) *launched = 0;
    if (!S || chunk < 1) return sfail(SFAC_EINVAL, "need a server and chunk >= 1");
    if (S->launched - S->completed >= kRounds)
        return sfail(SFAC_EINVAL, "two rounds are already in flight (call sfac_server_wait)");
    int wpb = 0, es = 0, mult = 0;
    if (!sfac::batch_shape(shape, &wpb, &es, &mult)) return sfail(SFAC_EINVAL, "bad kernel shape index");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Round& R = S->rounds[S->launched % kRounds];
    const bool behind = S->launched > S->completed;  // another round is in flight
    const Round& prev = S->rounds[(S->launched + kRounds - 1) % kRounds];
    std::vector<sfac::BatchInst> inst;
    std::vector<int> rslots;
    std::vector<long long> rsteps;
    int hold = -1;
    for (int i = 0; i < (int)S->slots.size(); ++i) {
        Slot& s = S->slots[i];
        // steps not yet covered by a round in flight
        const long long open = s.remaining - s.queued;
        if (!s.used || s.failed || open <= 0) continue;
        const long long k = std::min(chunk, open);
        sfac::BatchInst I = s.inst;
        I.steps = (int)k;
        sfac::set_items(I, es, mult);
        if (i == S->hold_slot) hold = (int)inst.size();
        inst.push_back(I);
        rslots.push_back(i);
        rsteps.push_back(k);
    }
    if (inst.empty()) return SFAC_OK;  // nothing to do: no round is added
    std::vector<unsigned char> blob;
    sfac::ScheduleLayout lay{};
    sfac::pack_schedule(inst, blob, &lay);
    cudaError_t err = reserve_schedule(R, lay.total);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return sfail(SFAC_ENOMEM, std::string("round schedule allocation: ") + cudaGetErrorString(err));
    }
    // Pinned staging, so that the upload does not wait for the round in flight.
    std::memcpy(R.host_sched, blob.data(), lay.total);
    sfac::BatchSchedule& sc = R.sc;
    sfac::bind_schedule(lay, R.dev_sched, mult, &sc);
    sc.counter = R.scratch;
    sc.done = R.scratch + 1;
    sc.error = reinterpret_cast<int*>(R.scratch + 1 + (long long)S->slots.size());
    sc.spin_limit = S->spin_limit;
    sc.hold_instance = hold;
    sc.common = S->dev_common;
    // strided passes of 256+ points in this round: stage them (see sfac_batch.cuh)
    bool long_strided = false;
    for (const sfac::BatchInst& I : inst)
        for (int a = 1; a < I.dim; ++a) long_strided = long_strided || I.n[a] >= 256;
    sc.stage = (S->prec == SFAC_FP32 && wpb == 8 && mult >= 2 && long_strided) ? mult : 0;
    int grid = 0;
    err = S->prec == SFAC_FP64 ? sfac::setup_batch_f64(wpb, es, 0, S->sms, &grid)
                               : sfac::setup_batch_f32(wpb, es, sc.stage, S->sms, &grid);
    // Fields shared with the round in flight advance in launch order, also when
    // the caller passes another stream.
    if (err == cudaSuccess && behind) err = cudaStreamWaitEvent(st, prev.done, 0);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(R.dev_sched, R.host_sched, lay.total, cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess)
        err = cudaMemsetAsync(R.scratch, 0, sizeof(unsigned long long) * (S->slots.size() + 2), st);
    if (err == cudaSuccess)
        err = S->prec == SFAC_FP64 ? sfac::launch_batch_f64(wpb, es, grid, sc, st)
                                   : sfac::launch_batch_f32(wpb, es, grid, sc, st);
    if (err == cudaSuccess) err = cudaMemcpyAsync(R.host_error, sc.error, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaEventRecord(R.done, st);
    if (err != cudaSuccess) return scuda(err, "round launch");
    R.slots.swap(rslots);
    R.steps.swap(rsteps);
    R.active = true;
    for (size_t k = 0; k < R.slots.size(); ++k) S->slots[R.slots[k]].queued += R.steps[k];
    if (hold >= 0) S->hold_slot = -1;  // the hook acts on one round
    ++S->launched;
    if (launched) *launched = 1;
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_server_wait(sfac_server* S, void* stream, int* finished, int max_finished, int* nfinished) try {
    (void)stream;
    if (!S || !nfinished || (max_finished > 0 && !finished)) return sfail(SFAC_EINVAL, "NULL argument");
    *nfinished = 0;
    if (S->launched == S->completed) return SFAC_OK;
    Round& R = S->rounds[S->completed % kRounds];
    const cudaError_t err = cudaEventSynchronize(R.done);
    R.active = false;
    ++S->completed;
    const bool timed_out = err == cudaSuccess && *R.host_error != 0;
    int nf = 0;
    for (size_t k = 0; k < R.slots.size(); ++k) {
        Slot& s = S->slots[R.slots[k]];
        s.queued -= R.steps[k];
        if (err != cudaSuccess || timed_out) {
            s.failed = true;  // partly advanced: its result is lost
        } else if (!s.failed) {
            s.remaining -= R.steps[k];
            s.done += R.steps[k];
        }
        if (s.queued == 0 && (s.failed || s.remaining == 0)) {
            if (nf < max_finished) finished[nf] = R.slots[k];
            ++nf;
        }
    }
    *nfinished = nf;
    if (err != cudaSuccess) return scuda(err, "round synchronise");
    if (timed_out) return sfail(SFAC_ETIMEOUT, "a dependency wait gave up; the requests of that round failed");
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_server_fetch(sfac_server* S, int slot, void* u_host, int release) try {
    if (!S || slot < 0 || slot >= (int)S->slots.size() || !S->slots[slot].used)
        return sfail(SFAC_EINVAL, "bad server or slot");
    Slot& s = S->slots[slot];
    if (s.queued > 0) return sfail(SFAC_EINVAL, "slot is part of a round in flight");
    const bool failed = s.failed;
    if (u_host && !failed) {
        const size_t bytes = (size_t)s.inst.npts * real_bytes(S->prec);
        cudaError_t err = cudaMemcpyAsync(u_host, s.inst.u, bytes, cudaMemcpyDeviceToHost, S->copy_stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(S->copy_stream);
        if (err != cudaSuccess) return scuda(err, "result copy");
    }
    if (release) {
        S->arena.release(s.off, s.bytes);
        s = Slot();
    }
    if (failed) return sfail(SFAC_ETIMEOUT, "the request's round gave up waiting; it has no result");
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_server_set_wait_limit(sfac_server* S, long long spin_limit, int hold_slot) try {
    if (!S || spin_limit < 1 || hold_slot < -1 || hold_slot >= (int)S->slots.size())
        return sfail(SFAC_EINVAL, "need a server, spin_limit >= 1 and hold_slot in [-1, max_slots)");
    S->spin_limit = spin_limit;
    S->hold_slot = hold_slot;
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

sfac_status sfac_server_info(const sfac_server* S, size_t* free_bytes, size_t* largest_free, int* active,
                             int* capacity) try {
    if (!S) return sfail(SFAC_EINVAL, "server is NULL");
    if (free_bytes) *free_bytes = S->arena.total - S->arena.used;
    if (largest_free) *largest_free = S->arena.largest_free();
    int n = 0;
    for (const Slot& s : S->slots) n += s.used ? 1 : 0;
    if (active) *active = n;
    if (capacity) *capacity = (int)S->slots.size();
    return SFAC_OK;
} catch (...) {
    return sfac::abi_exception_status();
}

}  // extern "C"
