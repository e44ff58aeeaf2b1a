// train_noalloc.cu -- apsm_train_noalloc: training whose scratch memory belongs to the library.
//
// apsm_train asks its caller for a device workspace.  Some callers cannot provide one: a
// real-time receive loop that must not allocate device memory once it is running (an
// allocation can block the loop and fragment memory), or a plug-in hosted by a framework that
// owns the device memory and hands its plug-ins no allocator.  For them this entry point runs
// the same training with its scratch in a fixed array that is part of the loaded library image
// (APSM_NOALLOC_SCRATCH_BYTES on every device that loads the library, held until the process
// exits).  It calls no cudaMalloc, no cudaFree and no allocating library routine.
//
// The scratch array's name, used in host code, is only a host-side stand-in for the device
// array: its device address is looked up with cudaGetSymbolAddress while the device is current,
// and that address is what the kernels receive.  The address belongs to the CUDA context the
// module was loaded into, so it is cached per context (by the driver's unique context id), not
// per device: after cudaDeviceReset, or when a primary context is released and created again,
// the new context gets its own lookup and a stale address is never used.
#include <cuda.h>

#include <mutex>

#include "apsm_common.cuh"

namespace {

constexpr size_t kScratchBytes = APSM_NOALLOC_SCRATCH_BYTES;

// The library-owned scratch.  Every call on a device shares it and it keeps whatever the last
// call left in it; the training kernels write every scratch word before they read it, so no
// part of it has to be cleared between calls.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

constexpr int kCacheSlots = 16;
struct CacheSlot {
    unsigned long long ctx_id;  // 0: empty
    void *addr;
};
std::mutex g_mu;
CacheSlot g_cache[kCacheSlots] = {};
int g_next_slot = 0;
CtxGetCurrentFn g_get_current = nullptr;
CtxGetIdFn g_get_id = nullptr;

// Unique id of the current context (made current first by a runtime call), or 0 on failure.
unsigned long long current_context_id() {
    if (!g_get_current || !g_get_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            cudaGetLastError();
            return 0;
        }
        g_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        g_get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr || g_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_noalloc_scratch in the current context (looked up on its first use).
apsm_status scratch_address(void **out) {
    // cudaSetDevice on the current device makes its primary context current (creating it if
    // needed) so that the driver can name it.
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        return APSM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long id = current_context_id();
    if (id == 0) return APSM_ERR_CUDA;
    for (const CacheSlot &s : g_cache)
        if (s.ctx_id == id) {
            *out = s.addr;
            return APSM_OK;
        }
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
        cudaGetLastError();
        return APSM_ERR_CUDA;
    }
    g_cache[g_next_slot] = CacheSlot{id, ptr};  // oldest slot reused: contexts are not recycled
    g_next_slot = (g_next_slot + 1) % kCacheSlots;
    *out = ptr;
    return APSM_OK;
}

}  // namespace

extern "C" apsm_status apsm_train_noalloc(const apsm_params *p, const float *rx_pilot, const float *sym_pilot,
                                          int32_t P, const float *clin0, const apsm_state *st, int8_t *case_log,
                                          void *stream) {
    size_t need = 0;
    apsm_status s = apsm_train_workspace_bytes(p, P, &need);
    if (s != APSM_OK) return s;
    if (!st || !st->dict || !st->dict_norm || !st->gamma || !st->clin || !st->meta) return APSM_ERR_INVALID_ARG;
    if (P > 0 && (!rx_pilot || !sym_pilot)) return APSM_ERR_INVALID_ARG;
    if (need > kScratchBytes) return APSM_ERR_WORKSPACE;  // more scratch than the fixed array holds
    void *scratch = nullptr;
    if ((s = scratch_address(&scratch)) != APSM_OK) return s;
    return apsm_train(p, rx_pilot, sym_pilot, P, clin0, st, scratch, kScratchBytes, case_log, stream);
}
