// sfac_pass_staged_f32.cu - the FP32 strided axis pass with TMA-staged tiles.
//
// In a strided pass (axis l > 0) complex line c of an outer slab is the column
// pair (2c, 2c + 1): each row of a line is 8 bytes, one row apart per element.
// Loading such lines thread by thread touches a new 32-byte sector for every
// 8 or 16 useful bytes and keeps the L1 busy. Here a CTA instead moves a whole
// tile, BW consecutive columns (BW/2 complex lines) by all N rows of one slab,
// with one TMA box copy per 256 rows: every row of the tile is BW * 4 = 64 or
// 128 contiguous bytes, and no thread issues the copy but one. The tile lands
// in shared memory with the 128-byte (64-byte) swizzle, under which the reads
// of each warp's lines are free of bank conflicts at N = 128 and, with the
// lanes interleaved (StagedShape::INTERLEAVE), at N = 256; the fused pass
// (sfac_pass.cuh) runs on them unchanged, the results go back into the same
// tile and one TMA store writes it out.
//
// The CTA is persistent over the tiles g = blockIdx.x + k * gridDim.x with a
// ring of three stage buffers: the load of tile k + 2 is issued when tile k is
// stored, after the store of tile k - 1 has finished reading its buffer, so a
// tile's copy overlaps the computation of the tile before it. Tiles may run
// past the last column (inner % BW != 0): the load fills zeros there and the
// store skips them.
//
// Every wait on a load is bounded (a.wait_cycles). A CTA whose wait runs out
// records SFAC_PASS_TIMEOUT in a.status, stops taking tiles, waits (bounded)
// for its loads still in flight and for its stores, and returns. The test hook
// a.hold sends the first wait of every CTA to a barrier nothing completes.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "sfac_pass.cuh"
#include "sfac_tma.cuh"

namespace sfac {

namespace {

template <int N>
struct StagedShape {
    static constexpr int E = 16;
    static constexpr int T = N / E;
    static constexpr int LPW = 32 / T;                       // complex lines per warp
    static constexpr int WPB = N >= 256 ? 4 * (N / 256) : 16 / LPW;  // warps per CTA
    static constexpr int BW = 2 * WPB * LPW;                 // tile width in floats: 32, or 16 from N = 256
    static constexpr int ROWS = N < 256 ? N : 256;           // rows per TMA box (the box limit is 256)
    static constexpr int BOXES = N / ROWS;
    static constexpr int STAGE_BYTES = N * BW * 4;
    static constexpr int STAGES = 3;
    // CTAs per SM the register allocation must allow: three CTAs of at most
    // four warps (168 registers a thread at N = 256, no spills; their shared
    // memory fits three times too); one 8-warp CTA at N = 512.
    static constexpr int MINB = WPB <= 4 ? 3 : 1;
    // Lane layout. Default: lane = j T + t (line j, thread t of the line).
    // With 64-byte tile rows and two lines per warp (N = 256) each half-warp
    // would read 16 consecutive rows of one line, and under the 64-byte
    // swizzle those rows cover only 8 of the 16 eight-byte bank slots (a 2-way
    // conflict on every tile read and write). There the lanes interleave the
    // lines instead, lane = t LPW + j: a half-warp reads 8 rows of both lines,
    // which fill all 16 slots. The exchange regions of the two lines are then
    // 8 values apart modulo 16 (LE = N + N/E + 8), so that the exchanges stay
    // free of conflicts too.
    static constexpr bool INTERLEAVE = (BW == 16 && LPW == 2);
    static constexpr int LE = N + N / E + (INTERLEAVE ? 8 : 0);
    using Ex = WarpExchange<float, N, E, LE>;
    static constexpr int XCH_ELEMS = WPB * LPW * LE;
    static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE_BYTES + SmemTables<float, N, E, false>::BYTES +
                                   sizeof(C2<float>) * XCH_ELEMS + 8 * (STAGES + 1);
    static_assert(BW == 32 || BW == 16, "tile rows are 64 or 128 bytes");
    static_assert(STAGE_BYTES % 1024 == 0, "stage buffers keep the swizzle atom alignment");
};

// Complex line `col / 2` of a staged tile: element k is the float pair at row
// k, columns col and col + 1, at the address the TMA swizzle gives it (16-byte
// chunk index XOR row bits; the buffer is 1024-byte aligned).
template <int N, int E, int BW>
struct StagedLine {
    unsigned char* buf;
    int col;

    __device__ __forceinline__ float2* at(int k) const {
        int off = (k * BW + col) * 4;
        off ^= (BW == 32) ? (((off >> 7) & 7) << 4) : (((off >> 7) & 3) << 4);
        return reinterpret_cast<float2*>(buf + off);
    }
    __device__ __forceinline__ void load(C2<float> (&x)[E], int t) const {
        constexpr int T = N / E;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float2 v = *at(t + e * T);
            x[e] = {v.x, v.y};
        }
    }
    __device__ __forceinline__ void store(const C2<float> (&x)[E], int t) const {
        constexpr int T = N / E;
#pragma unroll
        for (int e = 0; e < E; ++e) *at(t + e * T) = make_float2(x[e].x, x[e].y);
    }
};


template <int N>
__global__ void __launch_bounds__(StagedShape<N>::WPB * 32, StagedShape<N>::MINB)
axis_pass_staged_kernel(const __grid_constant__ CUtensorMap tmap, const PassArgs a0, long long tiles_per_outer,
                        long long ntiles) {
    using Sh = StagedShape<N>;
    constexpr int E = Sh::E, T = Sh::T, LPW = Sh::LPW, BW = Sh::BW, S = Sh::STAGES;
    using Ex = typename Sh::Ex;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* stage0 = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* tabs = stage0 + S * Sh::STAGE_BYTES;
    C2<float>* xch = reinterpret_cast<C2<float>*>(tabs + SmemTables<float, N, E, false>::BYTES);
    uint64_t* full = reinterpret_cast<uint64_t*>(xch + Sh::XCH_ELEMS);
    uint64_t* never = full + S;  // no arrival ever completes it (the hold test hook)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool leader = threadIdx.x == 0;
    if (leader) {
        prefetch_tensormap(&tmap);
        for (int s = 0; s < S + 1; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    PassArgs a = a0;
    SmemTables<float, N, E, false>::load(a, tabs);  // ends with __syncthreads

    const long long first = blockIdx.x, step = gridDim.x;
    const long long mine = first < ntiles ? (ntiles - 1 - first) / step + 1 : 0;
    // Tile k of this CTA: slab o, first column c.
    auto coords = [&](long long k, int& c, int& o) {
        const long long g = first + k * step;
        const long long ob = g / tiles_per_outer;
        o = (int)ob;
        c = (int)((g - ob * tiles_per_outer) * BW);
    };
    auto issue = [&](long long k) {
        int c, o;
        coords(k, c, o);
        const int s = (int)(k % S);
        unsigned char* dst = stage0 + s * Sh::STAGE_BYTES;
        mbar_expect_tx(&full[s], Sh::STAGE_BYTES);
#pragma unroll
        for (int b = 0; b < Sh::BOXES; ++b) tma_load_3d(dst + b * Sh::ROWS * BW * 4, &tmap, &full[s], c, b * Sh::ROWS, o);
    };
    long long issued = 0;  // loads issued (leader only)
    if (leader)
        for (; issued < S - 1 && issued < mine; ++issued) issue(issued);

    const int j = Sh::INTERLEAVE ? lane % LPW : lane / T;
    const int t = Sh::INTERLEAVE ? lane / LPW : lane % T;
    const Ex ex{xch + (warp * LPW + j) * Ex::LINE_ELEMS};
    long long k = 0;
    bool failed = false;
    for (; k < mine; ++k) {
        const int s = (int)(k % S);
        unsigned char* buf = stage0 + s * Sh::STAGE_BYTES;
        const bool held = a0.hold != 0 && k == 0;
        const bool ok = mbar_wait_bounded(held ? never : &full[s], held ? 0u : (unsigned)((k / S) & 1), a0.wait_cycles);
        const StagedLine<N, E, BW> line{buf, 2 * (warp * LPW + j)};
        C2<float> x[E];
        if (ok) {
            line.load(x, t);
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) x[e] = {0.f, 0.f};
        }
        fused_pass<float, N, E, false, false, true>(x, t, a, ex);
        if (ok) line.store(x, t);
        fence_proxy_async_smem();
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (leader) {
            int c, o;
            coords(k, c, o);
#pragma unroll
            for (int b = 0; b < Sh::BOXES; ++b) tma_store_3d(&tmap, buf + b * Sh::ROWS * BW * 4, c, b * Sh::ROWS, o);
            bulk_commit();
            if (issued < mine) {
                bulk_wait_read<1>();  // the store of tile k - 1 has left buffer (k - 1) % S
                issue(issued++);
            }
        }
    }
    if (leader) {
        if (failed) {
            if (a0.status) atomicOr(a0.status, SFAC_PASS_TIMEOUT);
            for (long long q = k; q < issued; ++q)
                mbar_wait_bounded(&full[q % S], (unsigned)((q / S) & 1), a0.wait_cycles);
        }
        bulk_wait<0>();
    }
}

// cuTensorMapEncodeTiled, looked up through the runtime (no link against the
// driver library).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static const EncodeTiled fn = []() -> EncodeTiled {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<EncodeTiled>(p);
    }();
    return fn;
}

int tile_width(int N) {
    switch (N) {
        case 32: return StagedShape<32>::BW;
        case 64: return StagedShape<64>::BW;
        case 128: return StagedShape<128>::BW;
        case 256: return StagedShape<256>::BW;
        case 512: return StagedShape<512>::BW;
        default: return 0;
    }
}

template <int N>
cudaError_t launch_staged(const PassArgs& a, cudaStream_t s) {
    using Sh = StagedShape<N>;
    // The field as a 3D tensor [outer][N][inner] of floats, boxes of BW x ROWS x 1.
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)a.inner, (cuuint64_t)N, (cuuint64_t)a.outer};
    const cuuint64_t strides[2] = {(cuuint64_t)a.inner * 4, (cuuint64_t)a.inner * 4 * N};
    const cuuint32_t box[3] = {(cuuint32_t)Sh::BW, (cuuint32_t)Sh::ROWS, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encoder()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.u, dims, strides, box, estr,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE,
                                 Sh::BW == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorNotSupported;

    auto kern = axis_pass_staged_kernel<N>;
    static LaunchSetup setup;
    int dev = 0, resident = 0;
    cudaError_t err = set_smem(kern, Sh::SMEM, setup, &dev);
    if (err == cudaSuccess) err = resident_grid(kern, Sh::WPB * 32, Sh::SMEM, setup, dev, &resident);
    if (err != cudaSuccess) return err;
    const long long tiles_per_outer = (a.inner + Sh::BW - 1) / Sh::BW;
    const long long ntiles = a.outer * tiles_per_outer;
    if (ntiles <= 0) return cudaSuccess;
    const long long grid = ntiles < resident ? ntiles : resident;
    kern<<<(unsigned)grid, Sh::WPB * 32, Sh::SMEM, s>>>(map, a, tiles_per_outer, ntiles);
    return cudaGetLastError();
}

// SMs of the current device (cached per device).
int sm_count() {
    static std::atomic<int> cache[LaunchSetup::kMaxDevices] = {};
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= LaunchSetup::kMaxDevices) {
        cudaGetLastError();
        return 0;
    }
    if ((sms = cache[dev].load()) != 0) return sms;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cache[dev].store(sms);
    return sms;
}

}  // namespace

bool staged_pass_eligible(int N, const PassArgs& a) {
    const int bw = tile_width(N);
    if (bw == 0 || a.nmem != N || a.inner <= 1 || a.host_io || a.out_shift != 0) return false;
    if (a.inner % 4 != 0 || a.inner < bw) return false;
    if (a.inner > 0x7fffffffLL || a.outer > 0x7fffffffLL) return false;
    if (reinterpret_cast<uintptr_t>(a.u) % 16 != 0) return false;
    // Fewer tiles than SMs would leave SMs idle that the warp kernel (a few
    // lines per CTA) keeps busy.
    const long long ntiles = a.outer * ((a.inner + bw - 1) / bw);
    if (ntiles < sm_count()) return false;
    return encoder() != nullptr;
}

cudaError_t launch_pass_staged_f32(int N, const PassArgs& a, cudaStream_t s) {
    if (!staged_pass_eligible(N, a)) return cudaErrorNotSupported;
    switch (N) {
        case 32: return launch_staged<32>(a, s);
        case 64: return launch_staged<64>(a, s);
        case 128: return launch_staged<128>(a, s);
        case 256: return launch_staged<256>(a, s);
        case 512: return launch_staged<512>(a, s);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace sfac
