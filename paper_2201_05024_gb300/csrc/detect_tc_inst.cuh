// detect_tc_inst.cuh -- instantiates the tensor-core detection kernel for one antenna count
// (APSM_TC_M) and every user-count bucket, in both precisions where supported.
#pragma once

#include "detect_tc.cuh"
#include "detect_tc_batch.cuh"
#include "detect_tcc.cuh"

#define APSM_TC_CAT2(a, b) a##b
#define APSM_TC_CAT(a, b) APSM_TC_CAT2(a, b)

namespace apsm {

// kb: user bucket (2, 4, 6, 8, 12, 16); prec: kTF32x3 or kHalf.
TcLauncher APSM_TC_CAT(detect_tc_launcher_m, APSM_TC_M)(int kb, int prec) {
    constexpr int M = APSM_TC_M;
    if (prec == kTF32x3) {
        if constexpr (M <= 32) {
            switch (kb) {
                case 2: return launch_detect_tc<M, 2, kTF32x3>;
                case 4: return launch_detect_tc<M, 4, kTF32x3>;
                case 6: return launch_detect_tc<M, 6, kTF32x3>;
                case 8: return launch_detect_tc<M, 8, kTF32x3>;
                case 12: return launch_detect_tc<M, 12, kTF32x3>;
                case 16: return launch_detect_tc<M, 16, kTF32x3>;
            }
        }
        return nullptr;
    }
    switch (kb) {
        case 2: return launch_detect_tc<M, 2, kHalf>;
        case 4: return launch_detect_tc<M, 4, kHalf>;
        case 6: return launch_detect_tc<M, 6, kHalf>;
        case 8: return launch_detect_tc<M, 8, kHalf>;
        case 12: return launch_detect_tc<M, 12, kHalf>;
        case 16: return launch_detect_tc<M, 16, kHalf>;
        default: return nullptr;
    }
}

// BF16/FP16 Gram with the coefficient sums on the tensor cores, antenna counts 16 to 64:
// launcher and workspace bytes for D dictionary slots (0: no such form).
TccLauncher APSM_TC_CAT(detect_tcc_launcher_m, APSM_TC_M)(int kb) {
    constexpr int M = APSM_TC_M;
    if constexpr (M >= 16) {
        switch (kb) {
            case 2: return launch_detect_tcc<M, 2>;
            case 4: return launch_detect_tcc<M, 4>;
            case 6: return launch_detect_tcc<M, 6>;
            case 8: return launch_detect_tcc<M, 8>;
            case 12: return launch_detect_tcc<M, 12>;
            case 16: return launch_detect_tcc<M, 16>;
        }
    }
    (void)kb;
    return nullptr;
}
size_t APSM_TC_CAT(detect_tcc_workspace_m, APSM_TC_M)(int kb, int D) {
    constexpr int M = APSM_TC_M;
    if constexpr (M >= 16) {
        switch (kb) {
            case 2: return tcc_workspace_bytes<M, 2>(D);
            case 4: return tcc_workspace_bytes<M, 4>(D);
            case 6: return tcc_workspace_bytes<M, 6>(D);
            case 8: return tcc_workspace_bytes<M, 8>(D);
            case 12: return tcc_workspace_bytes<M, 12>(D);
            case 16: return tcc_workspace_bytes<M, 16>(D);
        }
    }
    (void)kb;
    (void)D;
    return 0;
}

// Batched (persistent) form, FP32 accuracy (TF32 x3), antenna counts up to 32: launcher and
// resident CTAs per SM for user bucket kb.
TcBatchLauncher APSM_TC_CAT(detect_tc_batch_launcher_m, APSM_TC_M)(int kb, int *ctas_per_sm) {
    constexpr int M = APSM_TC_M;
    if constexpr (M <= 32) {
        switch (kb) {
            case 2: *ctas_per_sm = tc_batch_ctas_per_sm<M, 2, kTF32x3>(); return launch_detect_tc_batch<M, 2, kTF32x3>;
            case 4: *ctas_per_sm = tc_batch_ctas_per_sm<M, 4, kTF32x3>(); return launch_detect_tc_batch<M, 4, kTF32x3>;
            case 6: *ctas_per_sm = tc_batch_ctas_per_sm<M, 6, kTF32x3>(); return launch_detect_tc_batch<M, 6, kTF32x3>;
            case 8: *ctas_per_sm = tc_batch_ctas_per_sm<M, 8, kTF32x3>(); return launch_detect_tc_batch<M, 8, kTF32x3>;
            case 12: *ctas_per_sm = tc_batch_ctas_per_sm<M, 12, kTF32x3>(); return launch_detect_tc_batch<M, 12, kTF32x3>;
            case 16: *ctas_per_sm = tc_batch_ctas_per_sm<M, 16, kTF32x3>(); return launch_detect_tc_batch<M, 16, kTF32x3>;
        }
    }
    (void)ctas_per_sm;
    return nullptr;
}

}  // namespace apsm
