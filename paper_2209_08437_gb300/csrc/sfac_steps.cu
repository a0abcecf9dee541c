// sfac_steps.cu - a whole sfac_step call on a small grid in one launch.
//
// A small grid (a few thousand to 65536 unknowns) has too few lines per axis
// pass to fill the GPU, so a step costs mostly its d kernel launches and the
// latency of one line's chain of six FFTs. Here every line gets a warp of its
// own (one 32-thread CTA per warp-group, N/32 values per thread) and one
// cooperative launch runs all steps of the call: each CTA takes the lines
// g = blockIdx.x + k gridDim.x of the current axis pass, then all CTAs meet
// at a grid-wide barrier before the next pass (the next axis, or the next
// step's first axis). The field stays in global memory (L2: it is small);
// loads bypass L1 (.cg), since other CTAs wrote it during the same launch.
// The pass arithmetic is fused_pass, as in the per-pass kernels, and the
// nonlinear flow is placed as run_steps places it (J^Q_{tau/2} opening the
// first step and closing the last, J^Q_tau between steps).
//
// The barrier is an arrival counter and a generation word. Every wait on it
// is bounded in SM clock cycles (the plan's wait limit): a CTA whose wait runs
// out records SFAC_PASS_TIMEOUT in the plan's status word and returns, so the
// call ends (its field is then not valid) and sfac_plan_check reports it. The
// test hook `hold` sends the first wait of every CTA to a generation that never
// comes. The launch is cooperative, which guarantees that all CTAs are
// resident at once; the grid never exceeds that capacity.
#include <cuda_runtime.h>

#include <atomic>

#include "sfac_pass.cuh"
#include "sfac_steps.h"

namespace sfac {

namespace {

// Values per thread of a small-grid line of N points: 32 threads a line.
template <int N>
__host__ __device__ constexpr int steps_elems() {
    return N / 32 >= 2 ? N / 32 : 2;
}

// Exchange region of the one warp of a CTA: the largest (32/T)(N + N/E) over
// N = 32 .. 256 with E = steps_elems<N>().
constexpr int STEPS_REGION = 288;

template <typename R, int N, bool STRIDED>
__device__ __noinline__ void steps_group(const PassArgs& a, long long first, C2<R>* region, int lane) {
    constexpr int E = steps_elems<N>(), T = N / E;
    using Ex = WarpExchange<R, N, E>;
    static_assert((32 / T) * Ex::LINE_ELEMS <= STEPS_REGION, "exchange region");
    const int j = lane / T, t = lane % T;
    const LineRef<R, N, STRIDED> line(a, first + j);
    const Ex ex{region + j * Ex::LINE_ELEMS};
    C2<R> x[E];
    line.template load<E, true>(x, t);
    // FP64 ratio-twiddle records exist for the default values per thread only
    fused_pass<R, N, E, false, (sizeof(R) == 8 && E == f64_elems_per_thread(N))>(x, t, a, ex);
    line.template store<E>(x, t);
}

template <typename R, int N>
__device__ __forceinline__ void steps_axis(const PassArgs& a, bool strided, C2<R>* region, int lane) {
    constexpr int E = steps_elems<N>(), T = N / E, LPW = 32 / T;
    const long long groups = (a.clines + LPW - 1) / LPW;
    for (long long g = blockIdx.x; g < groups; g += gridDim.x) {
        if (strided) steps_group<R, N, true>(a, g * LPW, region, lane);
        else steps_group<R, N, false>(a, g * LPW, region, lane);
        __syncwarp();
    }
}

// Grid-wide barrier of the cooperative launch (one warp per CTA): false if
// this CTA's wait ran out (recorded in the status word).
__device__ __forceinline__ bool steps_barrier(const StepsArgs& g, bool held, int lane) {
    int ok = 1;
    __syncwarp();
    if (lane == 0) {
        volatile unsigned int* gen = g.bar + 1;
        const unsigned int mine = *gen;
        __threadfence();  // this CTA's stores of the pass before its arrival
        if (atomicAdd(g.bar, 1u) == gridDim.x - 1) {
            atomicExch(g.bar, 0u);  // reset before the release: nobody arrives at the next barrier earlier
            __threadfence();
            atomicAdd(const_cast<unsigned int*>(gen), 1u);
        } else {
            const unsigned int want = held ? mine + 2u : mine + 1u;  // the hook: a generation that never comes
            const long long t0 = clock64();
            while ((int)(*gen - want) < 0) {
                if (clock64() - t0 > g.wait_cycles) {
                    atomicOr(g.status, SFAC_PASS_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();  // loads of the next pass after the release
    }
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

template <typename R>
__global__ void __launch_bounds__(32) steps_kernel(const StepsArgs g) {
    __shared__ __align__(16) C2<R> region[STEPS_REGION];
    const int lane = threadIdx.x;
    for (long long s = 0; s < g.nsteps; ++s) {
        const bool last = s == g.nsteps - 1;
        for (int ax = 0; ax < g.dim; ++ax) {
            PassArgs a = g.ax[ax];
            // J^Q_{tau/2} opens the first step and closes the last one; between
            // two steps the closing and opening halves act as one J^Q_tau
            a.jq_in = (ax == 0 && s == 0);
            a.jq_in_E = g.jq_half_E;
            a.jq_in_1mE = g.jq_half_1mE;
            a.jq_out = (ax == g.dim - 1);
            a.jq_out_E = last ? g.jq_half_E : g.jq_full_E;
            a.jq_out_1mE = last ? g.jq_half_1mE : g.jq_full_1mE;
            switch (g.n[ax]) {
                case 32: steps_axis<R, 32>(a, ax > 0, region, lane); break;
                case 64: steps_axis<R, 64>(a, ax > 0, region, lane); break;
                case 128: steps_axis<R, 128>(a, ax > 0, region, lane); break;
                default: steps_axis<R, 256>(a, ax > 0, region, lane); break;
            }
            if (last && ax == g.dim - 1) break;
            if (!steps_barrier(g, g.hold != 0 && s == 0 && ax == 0, lane)) return;
        }
    }
}

// CTAs of one launch that are resident at once on the current device
// (cooperative-launch capacity), cached per device.
template <typename R>
int steps_capacity() {
    static std::atomic<int> cache[LaunchSetup::kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= LaunchSetup::kMaxDevices) {
        cudaGetLastError();
        return 0;
    }
    int c = cache[dev].load();
    if (c != 0) return c;
    int sms = 0, per_sm = 0, coop = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, steps_kernel<R>, 32, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    c = coop ? per_sm * sms : -1;
    cache[dev].store(c);
    return c;
}

}  // namespace

long long steps_grid(const StepsArgs& g) {
    long long grid = 0;
    for (int ax = 0; ax < g.dim; ++ax) {
        const int N = g.n[ax];
        const int E = N / 32 >= 2 ? N / 32 : 2, LPW = 32 / (N / E);
        const long long groups = (g.ax[ax].clines + LPW - 1) / LPW;
        grid = groups > grid ? groups : grid;
    }
    return grid;
}

bool steps_fit(int prec, const StepsArgs& g) {
    const long long grid = steps_grid(g);
    const int cap = prec == SFAC_FP64 ? steps_capacity<double>() : steps_capacity<float>();
    return grid >= 1 && cap > 0 && grid <= cap;
}

cudaError_t launch_steps(int prec, const StepsArgs& g, cudaStream_t s) {
    const long long grid = steps_grid(g);
    if (!steps_fit(prec, g)) return cudaErrorNotSupported;
    cudaError_t err = cudaMemsetAsync(g.bar, 0, 2 * sizeof(unsigned int), s);
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(32);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return prec == SFAC_FP64 ? cudaLaunchKernelEx(&cfg, steps_kernel<double>, g)
                             : cudaLaunchKernelEx(&cfg, steps_kernel<float>, g);
}

}  // namespace sfac
