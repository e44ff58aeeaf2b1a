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
// array: its device address is looked up once per device with cudaGetSymbolAddress while that
// device is current, and that address is what the kernels receive.
#include <mutex>

#include "apsm_common.cuh"

namespace {

constexpr size_t kScratchBytes = APSM_NOALLOC_SCRATCH_BYTES;

// The library-owned scratch.  Every call on a device shares it and it keeps whatever the last
// call left in it; the training kernels write every scratch word before they read it, so no
// part of it has to be cleared between calls.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up on first use).
apsm_status scratch_address(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return APSM_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return APSM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return APSM_ERR_CUDA;
        }
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
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
