// pslr_apply_noalloc: the preconditioner apply for callers that cannot
// allocate device memory at the time they apply it.
//
// pslr_apply keeps its scratch (series iterates, accumulator, per-subdomain
// partial sums, grid-barrier and error words) in buffers the context
// allocated at set-up.  Some callers cannot have device memory allocated for
// them - for instance code that hands all device memory to its own pool
// allocator and forbids cudaMalloc/cudaFree (or any allocating library call)
// outside it, or code paths that must not trigger the implicit
// synchronisation a cudaFree implies.  For them this entry point runs the
// same kernel on a scratch array that lives in the library itself: a
// file-scope __device__ array of fixed size, which every GPU that loads the
// library holds until the process exits.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "pslr.h"
#include "pslr_internal.h"

namespace pslr {
pslr_status apply_with_scratch(pslr_ctx *c, const void *b, void *z, int prec, int dir, cudaStream_t st,
                               void *scratch, size_t scratch_bytes);
pslr_status report(pslr_ctx *c, pslr_status st, const char *msg);
}  // namespace pslr

namespace {

// 16 MiB: enough for interface sizes q up to about 690,000 in FP64 (the
// 128^3 convection-diffusion problem has q = 511,640).
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array, looked up once per device (with that device
// current) and kept for the life of the process.  In host code the array's
// name is only a host-side stand-in: a kernel given &g_noalloc_scratch would
// address the wrong memory.  The lookup takes the lock only to fill an empty
// entry; later calls read the entry without it.  A cudaDeviceReset ends the
// context the address belongs to, so the cached address must not be used
// across one (documented in the header).
constexpr int kMaxDevices = 64;
std::atomic<void *> g_scratch_addr[kMaxDevices];
std::mutex g_scratch_lock;

cudaError_t scratch_of_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    void *p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lock(g_scratch_lock);
        p = g_scratch_addr[dev].load(std::memory_order_relaxed);
        if (!p) {
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return e;
            g_scratch_addr[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" pslr_status pslr_apply_noalloc(pslr_ctx *c, const void *b_dev, void *z_dev, pslr_prec prec,
                                          int32_t transpose, void *stream) {
    if (!c) return PSLR_ERR_ARG;
    void *scratch = nullptr;
    cudaError_t e = scratch_of_current_device(&scratch);
    if (e != cudaSuccess) return pslr::report(c, PSLR_ERR_CUDA, cudaGetErrorString(e));
    return pslr::apply_with_scratch(c, b_dev, z_dev, (int)prec, transpose ? 1 : 0,
                                    static_cast<cudaStream_t>(stream), scratch, kNoAllocScratchBytes);
}
