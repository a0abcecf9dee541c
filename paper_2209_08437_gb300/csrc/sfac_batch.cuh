// sfac_batch.cuh - one persistent launch that advances many independent SFAC
// problems of uneven sizes, orders and step counts.
//
// Work is cut into items: an item is `mult` warp-groups of lines of one
// instance's axis pass at one step (a warp-group is the 32/T lines one warp
// holds, see warp_pass_lines). Items are numbered phase by phase, a phase being
// (step s, axis a) over every instance still active there, so the numbering is
// a topological order of the dependencies: a pass may start once every item of
// the same instance's previous pass has finished (the previous axis of the same
// step, or the last axis of step s-1: eq. (finalstrang) applies the axes one
// after another and J^Q between steps).
//
// Each warp claims the next item from a global counter, waits until the
// instance's completion counter reaches the number of items of its earlier
// passes, runs the fused pass on its lines and adds one to that counter. Items
// are claimed in increasing order, so the item a warp waits on was claimed
// earlier by a running warp: the scheme cannot deadlock. Every wait is bounded:
// past `spin_limit` polls the warp records an error and leaves, and every other
// warp leaves at its next poll.
#pragma once

#include "sfac_batch_launch.h"
#include "sfac_pass.cuh"

namespace sfac {

// Shared memory per warp: the largest (32/T) * (N + N/E) over the supported
// lengths, 544 complex values (32 <= N <= 512, E <= 16).
constexpr int BATCH_REGION = 544;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// First index j in [lo, hi) with arr[j] > key (hi if none); arr ascending.
// The 32 lanes probe evenly spaced positions each round.
__device__ __forceinline__ long long warp_upper_bound(const long long* arr, long long lo, long long hi,
                                                      long long key, int lane) {
    while (hi - lo > 32) {
        const long long step = (hi - lo + 31) / 32;
        const long long idx = lo + lane * step;
        const bool gt = idx < hi ? (__ldg(arr + idx) > key) : true;
        const unsigned m = __ballot_sync(0xffffffffu, gt);
        if (m == 0) {
            lo = lo + 31 * step + 1;
            continue;
        }
        const int f = __ffs(m) - 1;
        const long long nhi = lo + f * step < hi ? lo + f * step : hi;
        if (f > 0) lo = lo + (f - 1) * step + 1;
        hi = nhi;
    }
    const long long idx = lo + lane;
    const bool gt = idx < hi ? (__ldg(arr + idx) > key) : true;
    const unsigned m = __ballot_sync(0xffffffffu, gt);
    return m ? lo + (__ffs(m) - 1) : hi;
}

// Lines per warp-group for length N with ES values per thread below N = 512.
template <int ES>
__host__ __device__ constexpr int batch_elems(int N) {
    return N >= 512 ? 16 : ES;
}

// FP32: the twiddle rows of TwRows<N, batch_elems<ES>(N)> for every length
// N = 32 .. 512, one after another in shared memory behind the common tables;
// complex values before those of length N, and in all.
template <int ES>
__host__ __device__ constexpr int batch_rows_offset(int N) {
    int off = 0;
    for (int M = 32; M < N; M *= 2) off += tw_rows_elems(M, batch_elems<ES>(M), M);
    return off;
}
template <int ES>
__host__ __device__ constexpr int batch_rows_elems() {
    return batch_rows_offset<ES>(1024);
}

// One warp-group of lines (32/T lines, see warp_pass_lines) of either axis
// kind; kept out of line so that each (R, N, E) body is compiled once per
// kernel and shared by both axis kinds.
template <typename R, int N, int E>
__device__ __noinline__ void batch_lines(const PassArgs& pa, bool strided, long long first, C2<R>* region,
                                         int lane) {
    constexpr int T = N / E;
    using Ex = WarpExchange<R, N, E>;
    const int j = lane / T, t = lane % T;
    const LineRefAny<R, N> line(pa, first + j, strided);
    const Ex ex{region + j * Ex::LINE_ELEMS};
    C2<R> x[E];
    line.template load<E>(x, t);
    fused_pass<R, N, E, false, false, (sizeof(R) == 4)>(x, t, pa, ex);
    line.template store<E>(x, t);
}

// One warp-group of a staged strided item: its lines sit line by line in the
// warp's staging buffer `stage` (line stride S complex values), group m.
template <typename R, int N, int E>
__device__ __noinline__ void batch_lines_staged(const PassArgs& pa, C2<R>* stage, int S, int m, C2<R>* region,
                                                int lane) {
    constexpr int T = N / E;
    constexpr int LPW = 32 / T;
    using Ex = WarpExchange<R, N, E>;
    const int j = lane / T, t = lane % T;
    C2<R>* line = stage + (m * LPW + j) * S;
    const Ex ex{region + j * Ex::LINE_ELEMS};
    C2<R> x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = line[t + e * T];
    fused_pass<R, N, E, false, false, (sizeof(R) == 4)>(x, t, pa, ex);
#pragma unroll
    for (int e = 0; e < E; ++e) line[t + e * T] = x[e];
}

// Complex values of the twiddle rows of one launch (FP32 only).
template <typename R, int ES>
__host__ __device__ constexpr int batch_rows_of() {
    return sizeof(R) == 4 ? batch_rows_elems<ES>() : 0;
}

// Bytes of dynamic shared memory of one launch.
template <typename R, int ES>
__host__ __device__ constexpr size_t batch_smem_bytes(int wpb, int stage) {
    return sizeof(C2<R>) * ((size_t)wpb * BATCH_REGION + BATCH_COMMON_ELEMS + batch_rows_of<R, ES>() +
                            (stage > 0 ? (size_t)wpb * batch_stage_elems(stage) : 0));
}

// Launched with blockDim.x = 32 * (warps per CTA) <= MAXT and dynamic shared
// memory for BATCH_REGION complex values per warp plus BATCH_COMMON_ELEMS;
// MINB CTAs per SM must fit the register allocation.
template <typename R, int ES, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
batch_kernel(const BatchSchedule b) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C2<R>* region = reinterpret_cast<C2<R>*>(smem_raw) + warp * BATCH_REGION;
    // Twiddles and twists of every length, shared by all instances, read from
    // shared memory instead of each instance's global copy.
    C2<R>* common = reinterpret_cast<C2<R>*>(smem_raw) + (blockDim.x >> 5) * BATCH_REGION;
    const C2<R>* gcommon = static_cast<const C2<R>*>(b.common);
    for (int i = threadIdx.x; i < BATCH_COMMON_ELEMS; i += blockDim.x) common[i] = gcommon[i];
    // FP32: the twiddle rows of every length, from the global twiddle tables.
    C2<R>* rows = common + BATCH_COMMON_ELEMS;
    if constexpr (sizeof(R) == 4) {
        C2<float>* r = reinterpret_cast<C2<float>*>(rows);
        const C2<float>* g = reinterpret_cast<const C2<float>*>(gcommon);
        build_tw_rows<32, batch_elems<ES>(32)>(r + batch_rows_offset<ES>(32), g + batch_common_offset(32), threadIdx.x, blockDim.x);
        build_tw_rows<64, batch_elems<ES>(64)>(r + batch_rows_offset<ES>(64), g + batch_common_offset(64), threadIdx.x, blockDim.x);
        build_tw_rows<128, batch_elems<ES>(128)>(r + batch_rows_offset<ES>(128), g + batch_common_offset(128), threadIdx.x, blockDim.x);
        build_tw_rows<256, batch_elems<ES>(256)>(r + batch_rows_offset<ES>(256), g + batch_common_offset(256), threadIdx.x, blockDim.x);
        build_tw_rows<512, 16>(r + batch_rows_offset<ES>(512), g + batch_common_offset(512), threadIdx.x, blockDim.x);
    }
    __syncthreads();
    // This warp's staging buffer for strided items (b.stage > 0, FP32).
    C2<R>* stage = rows + batch_rows_of<R, ES>() + (b.stage > 0 ? warp * batch_stage_elems(b.stage) : 0);
    int p = 0;  // phase of the last item: claimed items increase, so p only moves forward
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(b.counter, 1ULL);
        item = __shfl_sync(0xffffffffu, item, 0);
        if ((long long)item >= b.total_items) break;
        while (__ldg(b.phase_base + p + 1) <= (long long)item) ++p;
        const long long local = (long long)item - __ldg(b.phase_base + p);
        const long long f0 = __ldg(b.phase_first + p), f1 = __ldg(b.phase_first + p + 1);
        const long long slot = warp_upper_bound(b.slot_cum, f0, f1, local, lane);
        const int ii = __ldg(b.slot_inst + slot);
        const long long g = local - (slot > f0 ? __ldg(b.slot_cum + slot - 1) : 0);
        const int s = __ldg(b.phase_step + p), a = __ldg(b.phase_axis + p);
        const BatchInst& I = b.inst[ii];

        // Wait for every item of this instance's earlier passes.
        long long target = 0;
        for (int l = 0; l < I.dim; ++l) target += (long long)I.items[l];
        target *= s;
        for (int l = 0; l < a; ++l) target += I.items[l];
        if (ii == b.hold_instance && (s > 0 || a > 0)) target += 1;  // never satisfied
        int ok = 1;
        if (lane == 0) {
            long long polls = 0;
            while ((long long)ld_acquire_u64(b.done + ii) < target) {
                if (ld_volatile_i32(b.error) != 0) { ok = 0; break; }
                if (++polls > b.spin_limit) {
                    atomicCAS(b.error, 0, SFAC_BATCH_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        __syncwarp();

        // The pass this item belongs to.
        const int N = I.n[a];
        long long inner = 1;
        for (int l = 0; l < a; ++l) inner *= I.n[l];
        PassArgs pa;
        pa.u = I.u;
        pa.inner = inner;
        pa.outer = I.npts / ((long long)N * inner);
        pa.clines = (a == 0) ? (pa.outer + 1) / 2 : pa.outer * (inner / 2);
        pa.nmem = N;
        pa.eC = I.tab[a][0];
        pa.eS = I.tab[a][1];
        pa.twid = common + batch_common_offset(N);
        pa.twrows = rows + batch_rows_offset<ES>(N);
        pa.twist = common + batch_common_offset(N) + N;
        // J^Q_{tau/2} opens step 0 and closes the last step; inner steps merge
        // the closing and opening halves into J^Q_tau.
        pa.jq_in = (a == 0 && s == 0);
        pa.jq_in_E = I.jq[0];
        pa.jq_in_1mE = I.jq[1];
        pa.jq_out = (a == I.dim - 1);
        const bool last = (s == I.steps - 1);
        pa.jq_out_E = last ? I.jq[0] : I.jq[2];
        pa.jq_out_1mE = last ? I.jq[1] : I.jq[3];

        const int lpw = 32 * batch_elems<ES>(N) / N;
        const bool strided = a > 0;
        // Staged strided item: its L = mult * lpw lines are adjacent column
        // pairs of one slab (the slab's pair count is a multiple of L, so no
        // item straddles slabs or is partial). The warp copies the N rows of
        // those 2L columns into its staging buffer with 16-byte loads, runs
        // each warp-group from there and writes the block back with 16-byte
        // stores: one L2 round trip per item, in whole 32-byte sectors, instead
        // of one per group at 8 or 16 bytes a row.
        bool staged = false;
        if constexpr (sizeof(R) == 4) {
            const int L = b.mult * lpw;
            const long long pairs = inner / 2;
            // Only lines of 256+ points: their groups read 8 or 16 bytes a row;
            // shorter lines already read whole sectors and gain nothing.
            staged = b.stage > 0 && strided && N >= 256 && b.mult == b.stage && pairs % L == 0;
            if (staged) {
                const int S = N + BATCH_STAGE_PAD;
                const long long first = g * L;                  // first line of the item
                const long long o = first / pairs;
                R* base = static_cast<R*>(I.u) + o * (long long)N * inner + 2 * (first - o * pairs);
                const int q4 = L / 2;                           // 16-byte pieces per row (a power of two)
                const int qs = __ffs(q4) - 1;
                for (int f = lane; f < N * q4; f += 32) {
                    const int k = f >> qs, q = f & (q4 - 1);
                    const float4 v = __ldcg(reinterpret_cast<const float4*>(base + (long long)k * inner) + q);
                    stage[(2 * q) * S + k] = C2<R>{R(v.x), R(v.y)};
                    stage[(2 * q + 1) * S + k] = C2<R>{R(v.z), R(v.w)};
                }
                __syncwarp();
                for (int m = 0; m < b.mult; ++m) {
                    switch (N) {
                        case 32: batch_lines_staged<R, 32, ES>(pa, stage, S, m, region, lane); break;
                        case 64: batch_lines_staged<R, 64, ES>(pa, stage, S, m, region, lane); break;
                        case 128: batch_lines_staged<R, 128, ES>(pa, stage, S, m, region, lane); break;
                        case 256: batch_lines_staged<R, 256, ES>(pa, stage, S, m, region, lane); break;
                        default: batch_lines_staged<R, 512, 16>(pa, stage, S, m, region, lane); break;
                    }
                    __syncwarp();
                }
                for (int f = lane; f < N * q4; f += 32) {
                    const int k = f >> qs, q = f & (q4 - 1);
                    const C2<R> lo = stage[(2 * q) * S + k], hi = stage[(2 * q + 1) * S + k];
                    reinterpret_cast<float4*>(base + (long long)k * inner)[q] =
                        make_float4(float(lo.x), float(lo.y), float(hi.x), float(hi.y));
                }
                __syncwarp();
            }
        }
        if (!staged) {
        for (int m = 0; m < b.mult; ++m) {
            const long long first = (g * b.mult + m) * lpw;
            if (first >= pa.clines) break;
            switch (N) {
                case 32: batch_lines<R, 32, ES>(pa, strided, first, region, lane); break;
                case 64: batch_lines<R, 64, ES>(pa, strided, first, region, lane); break;
                case 128: batch_lines<R, 128, ES>(pa, strided, first, region, lane); break;
                case 256: batch_lines<R, 256, ES>(pa, strided, first, region, lane); break;
                default: batch_lines<R, 512, 16>(pa, strided, first, region, lane); break;
            }
            __syncwarp();
        }
        }
        // Publish: the stores above happen before the count is raised.
        if (lane == 0) {
            __threadfence();
            atomicAdd(b.done + ii, 1ULL);
        }
    }
}

}  // namespace sfac

namespace sfac {

// Set the kernel's shared-memory limit and return its persistent grid (one CTA
// per resident slot on every SM). Called when a run is prepared, outside any
// stream capture.
// Kernels of up to 4 warps are compiled for three resident CTAs per SM
// (FP32; at most 168 registers a thread), 8-warp ones for one.
template <typename R>
constexpr int batch_small_minb() {
    return sizeof(R) == 4 ? 3 : 2;
}

template <typename R, int ES>
cudaError_t setup_batch(int wpb, int stage, int sms, int* grid) {
    if (wpb < 1 || wpb > 8 || stage < 0 || stage > 4) return cudaErrorInvalidValue;
    auto kern = wpb <= 4 ? batch_kernel<R, ES, 128, batch_small_minb<R>()> : batch_kernel<R, ES, 256, 1>;
    const size_t smem = batch_smem_bytes<R, ES>(wpb, stage);
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem);
    if (err != cudaSuccess) return err;
    *grid = (per_sm < 1 ? 1 : per_sm) * sms;
    return cudaSuccess;
}

// Enqueue only (no attribute calls, no allocation): safe inside a graph capture.
template <typename R, int ES>
cudaError_t launch_batch(int wpb, int grid, const BatchSchedule& sc, cudaStream_t s) {
    if (wpb < 1 || wpb > 8 || grid < 1) return cudaErrorInvalidValue;
    const size_t smem = batch_smem_bytes<R, ES>(wpb, sc.stage);
    if (wpb <= 4)
        batch_kernel<R, ES, 128, batch_small_minb<R>()><<<grid, wpb * 32, smem, s>>>(sc);
    else
        batch_kernel<R, ES, 256, 1><<<grid, wpb * 32, smem, s>>>(sc);
    return cudaGetLastError();
}

}  // namespace sfac
