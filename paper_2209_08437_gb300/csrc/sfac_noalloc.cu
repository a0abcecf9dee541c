// sfac_noalloc.cu - sfac_batch_launch_noalloc: the batched launch with its
// scratch counters in a fixed, library-wide device array instead of memory the
// batch allocated.
//
// Why: some callers may not allocate device memory at the point where they
// launch work. Examples: code running under an allocator that owns the whole
// device and forbids raw cudaMalloc, real-time loops where cudaMalloc and
// cudaFree would add unpredictable latency or implicit synchronisation, and
// embedders that budget every byte of device memory up front. This entry point
// allocates nothing: the work counter, the per-instance completion counters and
// the status flag of the persistent batch kernel live in `g_noalloc_scratch`
// below, which exists once per device for as long as the library is loaded.
//
// Limits and rules:
//  - at most SFAC_NOALLOC_MAX_INSTANCES instances per batch (larger batches are
//    rejected with SFAC_EINVAL before anything is enqueued);
//  - every call on a device shares the one array and leaves its counters in it;
//    each call clears them first (cudaMemsetAsync), so calls that overlap on
//    the GPU (another stream, another thread, another batch) race and must be
//    serialised by the caller;
//  - the first call on each device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current; make that first call
//    before capturing any stream. The address is kept per device together
//    with the device's current context: after a context reset (for example
//    cudaDeviceReset) the array lives in a new context, so the next call finds
//    a different context and looks the address up again (again before any
//    capture);
//  - the batch must already be prepared (sfac_batch_prepare), which is where
//    its tables and schedule were allocated.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "sfac.h"
#include "sfac_batch_launch.h"
#include "sfac_internal.h"

namespace {

// Work counter, SFAC_NOALLOC_MAX_INSTANCES completion counters and a status
// word: (8192 + 2) * 8 bytes = 64 KiB per device.
constexpr int kMaxInstances = SFAC_NOALLOC_MAX_INSTANCES;
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kMaxInstances + 2];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Per device: the context the address was looked up in, and the address.
CUcontext g_scratch_ctx[kMaxDevices] = {};
unsigned long long* g_scratch_addr[kMaxDevices] = {};

sfac_status nfail(sfac_status st, const std::string& msg) {
    sfac::set_last_error(msg);
    return st;
}

// cuCtxGetCurrent, looked up through the runtime (no link against the driver
// library); NULL if the driver does not provide it.
using CtxGetCurrent = CUresult (*)(CUcontext*);
CtxGetCurrent ctx_get_current() {
    static const CtxGetCurrent fn = []() -> CtxGetCurrent {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<CtxGetCurrent>(p);
    }();
    return fn;
}

// The calling thread's current context (NULL if none or unknown).
CUcontext current_context() {
    CUcontext c = nullptr;
    const CtxGetCurrent fn = ctx_get_current();
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

// Device address of g_noalloc_scratch on the current device: looked up once
// per device and context (set-up), with that device current.
sfac_status scratch_address(int dev, unsigned long long** out) {
    if (dev < 0 || dev >= kMaxDevices) return nfail(SFAC_EUNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lock(g_mu);
    const CUcontext ctx = current_context();
    if (!g_scratch_addr[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
        void* ptr = nullptr;
        const cudaError_t err = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (err != cudaSuccess)
            return nfail(SFAC_ECUDA, std::string("cudaGetSymbolAddress of the static scratch: ") +
                                         cudaGetErrorString(err));
        g_scratch_addr[dev] = static_cast<unsigned long long*>(ptr);
        g_scratch_ctx[dev] = current_context();  // the lookup made the device's context current
    }
    *out = g_scratch_addr[dev];
    return SFAC_OK;
}

}  // namespace

namespace sfac {
// Implemented in sfac_batch.cu: the prepared run of `batch` with its three
// scratch pointers redirected to `scratch` (counter, done[], status word).
sfac_status batch_launch_with_scratch(sfac_batch* batch, unsigned long long* scratch, cudaStream_t stream);
int batch_count(const sfac_batch* batch);
int batch_device(const sfac_batch* batch);
}  // namespace sfac

extern "C" {

sfac_status sfac_batch_launch_noalloc(sfac_batch* batch, void* stream) try {
    if (!batch) return nfail(SFAC_EINVAL, "batch is NULL");
    const int count = sfac::batch_count(batch);
    if (count > kMaxInstances)
        return nfail(SFAC_EINVAL, "sfac_batch_launch_noalloc takes at most " + std::to_string(kMaxInstances) +
                                      " instances; this batch has " + std::to_string(count));
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return nfail(SFAC_ECUDA, "cudaGetDevice failed");
    const int dev = sfac::batch_device(batch);
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return nfail(SFAC_ECUDA, "cannot select the batch's device");
    unsigned long long* scratch = nullptr;
    sfac_status st = scratch_address(dev, &scratch);
    if (st == SFAC_OK) st = sfac::batch_launch_with_scratch(batch, scratch, static_cast<cudaStream_t>(stream));
    if (prev != dev) cudaSetDevice(prev);
    return st;
} catch (...) {
    return sfac::abi_exception_status();
}

}  // extern "C"
