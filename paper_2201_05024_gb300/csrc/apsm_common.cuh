// apsm_common.cuh -- device helpers shared by the sm_103a APSM kernels.
//
// Inline PTX for the bulk-copy engine (cp.async.bulk global -> shared, completion counted on
// an mbarrier), bounded mbarrier waits, and the MUFU base-2 exponential.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/apsm.h"

namespace apsm {

// Entries per dictionary tile staged into shared memory; the state's slot count is a multiple
// of it so that whole tiles can always be copied.
constexpr int kTileEntries = 32;

// A bounded wait gives up after this many SM clock cycles (about two seconds at 2 GHz),
// writes APSM_ERR_TIMEOUT to the status word and lets the kernel return.
constexpr long long kWaitCycles = 4000000000LL;

// log2(e): exp(-d / (2 sigma^2)) = 2^(-d * log2(e) / (2 sigma^2)).
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make mbarrier initialisation visible to the async (bulk-copy) proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete; false after kWaitCycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}

// The same wait for a thread whose wait is not on the critical path (a producer that runs a
// tile or more ahead): it sleeps between polls so that its spinning takes no issue slots from
// the warps that share its scheduler.
__device__ __forceinline__ bool mbar_wait_sleepy(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        __nanosleep(200);
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}

// 1-D bulk copy global -> shared; both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *smem_dst, const void *gmem_src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// MUFU base-2 exponential (flush-to-zero); the argument is always <= 0 here.
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Gray square QAM of apsm_params.modulation, one axis: L = 2^half levels (2i - (L-1)) a.  The
// level is the number of decision boundaries (2b - L) a, b = 1..L-1, at or below y (QPSK: the
// sign, 0 counting as non-negative); the axis label is the Gray code of L - 1 - level.
__device__ __forceinline__ int pam_level(float y, int half, float a) {
    const int L = 1 << half;
    int lev = 0;
    for (int b = 1; b < L; ++b) lev += (y >= (float)(2 * b - L) * a) ? 1 : 0;
    return lev;
}

// The decided amplitude of one axis.
__device__ __forceinline__ float pam_value(int lev, int half, float a) {
    return (float)(2 * lev - ((1 << half) - 1)) * a;
}

__device__ __forceinline__ uint32_t pam_gray(int lev, int half) {
    const uint32_t u = (uint32_t)((1 << half) - 1 - lev);
    return u ^ (u >> 1);
}

// Label of the complex decision: real axis in the low `half` bits, imaginary axis above.
__device__ __forceinline__ uint8_t qam_label(float y1, float y2, int half, float a) {
    if (half == 1) return (uint8_t)((y1 < 0.f ? 1 : 0) | (y2 < 0.f ? 2 : 0));
    return (uint8_t)(pam_gray(pam_level(y1, half, a), half) | (pam_gray(pam_level(y2, half, a), half) << half));
}

__device__ __forceinline__ void report(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Programmatic dependent launch.  A kernel launched by launch_pdl may become resident while its
// predecessor in the stream is still running (its launch and shared-memory setup overlap the
// predecessor); before touching any memory it waits for the predecessor to complete, then lets
// its own successor begin launching.  Launched without the attribute, both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// Since every kernel triggers its successor only after its own wait, a kernel that starts early
// may already rely on everything two launches back having completed.
__device__ __forceinline__ void pdl_enter() {
    pdl_wait();
    pdl_trigger();
}

// Reads of what another kernel of this library wrote (the state, training tables, carried
// values, partial sums, soft outputs) go through L2: __ldcg or bulk copies, never the L1 /
// read-only path.  A kernel launched this way can become resident on an SM beside the previous
// kernel's CTAs, and an L1 line cached there before the previous kernel's other CTAs wrote the
// data was observed to be read after the wait (the FMA detection engine behind training read a
// stale linear filter and entry count until its loads went through L2).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*fn)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, args...);
}

}  // namespace apsm
