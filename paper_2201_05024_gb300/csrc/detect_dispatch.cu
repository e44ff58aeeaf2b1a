// detect_dispatch.cu -- maps (M, K) to the FP32 detection kernels (and adjoint) instantiated for it.
#include <atomic>

#include "detect_bwd.cuh"
#include "detect_f32.cuh"
#include "detect_tc.cuh"
#include "detect_tc_batch.cuh"
#include "detect_tma.cuh"
#include "detect_tcc.cuh"

namespace apsm {

DetectLauncher detect_f32_launcher_m2(int K);
DetectLauncher detect_f32_launcher_m4(int K);
DetectLauncher detect_f32_launcher_m8(int K);
DetectLauncher detect_f32_launcher_m16(int K);
DetectLauncher detect_f32_launcher_m32(int K);
DetectLauncher detect_f32_launcher_m64(int K);

DetectBwdLauncher detect_bwd_launcher_m2(int K);
DetectBwdLauncher detect_bwd_launcher_m4(int K);
DetectBwdLauncher detect_bwd_launcher_m8(int K);
DetectBwdLauncher detect_bwd_launcher_m16(int K);
DetectBwdLauncher detect_bwd_launcher_m32(int K);
DetectBwdLauncher detect_bwd_launcher_m64(int K);

TcLauncher detect_tc_launcher_m2(int kb, int prec);
TcLauncher detect_tc_launcher_m4(int kb, int prec);
TcLauncher detect_tc_launcher_m8(int kb, int prec);
TcLauncher detect_tc_launcher_m16(int kb, int prec);
TcLauncher detect_tc_launcher_m32(int kb, int prec);
TcLauncher detect_tc_launcher_m64(int kb, int prec);

TccLauncher detect_tcc_launcher_m16(int kb);
TccLauncher detect_tcc_launcher_m32(int kb);
TccLauncher detect_tcc_launcher_m64(int kb);
size_t detect_tcc_workspace_m16(int kb, int D);
size_t detect_tcc_workspace_m32(int kb, int D);
size_t detect_tcc_workspace_m64(int kb, int D);

TcBatchLauncher detect_tc_batch_launcher_m2(int kb, int *ctas_per_sm);
TcBatchLauncher detect_tc_batch_launcher_m4(int kb, int *ctas_per_sm);
TcBatchLauncher detect_tc_batch_launcher_m8(int kb, int *ctas_per_sm);
TcBatchLauncher detect_tc_batch_launcher_m16(int kb, int *ctas_per_sm);
TcBatchLauncher detect_tc_batch_launcher_m32(int kb, int *ctas_per_sm);
TcBatchLauncher detect_tc_batch_launcher_m64(int kb, int *ctas_per_sm);

TmaLauncher detect_tma_launcher_m4(int K);
TmaLauncher detect_tma_launcher_m8(int K);
TmaLauncher detect_tma_launcher_m16(int K);

TmaEncodeFn tma_encode_fn() {
    static std::atomic<TmaEncodeFn> fn{nullptr};
    static std::atomic<int> tried{0};
    TmaEncodeFn f = fn.load();
    if (f || tried.load()) return f;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess && p) {
        f = reinterpret_cast<TmaEncodeFn>(p);
        fn.store(f);
    } else {
        cudaGetLastError();
    }
    tried.store(1);
    return f;
}

// TMA-staged FP32 detection for (M, K); nullptr where no instantiation exists.
TmaLauncher detect_tma_launcher(int M, int K) {
    switch (M) {
        case 4: return detect_tma_launcher_m4(K);
        case 8: return detect_tma_launcher_m8(K);
        case 16: return detect_tma_launcher_m16(K);
        default: return nullptr;
    }
}

// Smallest supported user bucket >= K for the tensor-core kernels (0 if none).
int tc_user_bucket(int K) {
    static const int kB[] = {2, 4, 6, 8, 12, 16};
    for (int b : kB)
        if (b >= K) return b;
    return 0;
}

TcLauncher detect_tc_launcher(int M, int K, int prec) {
    const int kb = tc_user_bucket(K);
    if (!kb) return nullptr;
    switch (M) {
        case 2: return detect_tc_launcher_m2(kb, prec);
        case 4: return detect_tc_launcher_m4(kb, prec);
        case 8: return detect_tc_launcher_m8(kb, prec);
        case 16: return detect_tc_launcher_m16(kb, prec);
        case 32: return detect_tc_launcher_m32(kb, prec);
        case 64: return detect_tc_launcher_m64(kb, prec);
        default: return nullptr;
    }
}

// BF16/FP16 detection with the coefficient sums on the tensor cores; nullptr if none.
TccLauncher detect_tcc_launcher(int M, int K) {
    const int kb = tc_user_bucket(K);
    if (!kb) return nullptr;
    switch (M) {
        case 16: return detect_tcc_launcher_m16(kb);
        case 32: return detect_tcc_launcher_m32(kb);
        case 64: return detect_tcc_launcher_m64(kb);
        default: return nullptr;
    }
}
size_t detect_tcc_workspace(int M, int K, int D) {
    const int kb = tc_user_bucket(K);
    if (!kb) return 0;
    switch (M) {
        case 16: return detect_tcc_workspace_m16(kb, D);
        case 32: return detect_tcc_workspace_m32(kb, D);
        case 64: return detect_tcc_workspace_m64(kb, D);
        default: return 0;
    }
}

// Batched persistent detection (FP32 accuracy) for class (M, user bucket of K); nullptr if none.
TcBatchLauncher detect_tc_batch_launcher(int M, int K, int *ctas_per_sm) {
    const int kb = tc_user_bucket(K);
    if (!kb) return nullptr;
    switch (M) {
        case 2: return detect_tc_batch_launcher_m2(kb, ctas_per_sm);
        case 4: return detect_tc_batch_launcher_m4(kb, ctas_per_sm);
        case 8: return detect_tc_batch_launcher_m8(kb, ctas_per_sm);
        case 16: return detect_tc_batch_launcher_m16(kb, ctas_per_sm);
        case 32: return detect_tc_batch_launcher_m32(kb, ctas_per_sm);
        case 64: return detect_tc_batch_launcher_m64(kb, ctas_per_sm);
        default: return nullptr;
    }
}

DetectBwdLauncher detect_bwd_launcher(int M, int K) {
    switch (M) {
        case 2: return detect_bwd_launcher_m2(K);
        case 4: return detect_bwd_launcher_m4(K);
        case 8: return detect_bwd_launcher_m8(K);
        case 16: return detect_bwd_launcher_m16(K);
        case 32: return detect_bwd_launcher_m32(K);
        case 64: return detect_bwd_launcher_m64(K);
        default: return nullptr;
    }
}

DetectLauncher detect_f32_launcher(int M, int K) {
    switch (M) {
        case 2: return detect_f32_launcher_m2(K);
        case 4: return detect_f32_launcher_m4(K);
        case 8: return detect_f32_launcher_m8(K);
        case 16: return detect_f32_launcher_m16(K);
        case 32: return detect_f32_launcher_m32(K);
        case 64: return detect_f32_launcher_m64(K);
        default: return nullptr;
    }
}

}  // namespace apsm
