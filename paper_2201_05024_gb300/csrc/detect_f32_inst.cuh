// detect_f32_inst.cuh -- instantiates the FP32 detection kernel for one antenna count
// (APSM_DETECT_M) and every supported user count K = 1..16, with its adjoint.
#pragma once

#include "detect_bwd.cuh"
#include "detect_f32.cuh"

#define APSM_CAT2(a, b) a##b
#define APSM_CAT(a, b) APSM_CAT2(a, b)

namespace apsm {

DetectLauncher APSM_CAT(detect_f32_launcher_m, APSM_DETECT_M)(int K) {
    constexpr int M = APSM_DETECT_M;
    switch (K) {
        case 1: return launch_detect_f32<M, 1>;
        case 2: return launch_detect_f32<M, 2>;
        case 3: return launch_detect_f32<M, 3>;
        case 4: return launch_detect_f32<M, 4>;
        case 5: return launch_detect_f32<M, 5>;
        case 6: return launch_detect_f32<M, 6>;
        case 7: return launch_detect_f32<M, 7>;
        case 8: return launch_detect_f32<M, 8>;
        case 9: return launch_detect_f32<M, 9>;
        case 10: return launch_detect_f32<M, 10>;
        case 11: return launch_detect_f32<M, 11>;
        case 12: return launch_detect_f32<M, 12>;
        case 13: return launch_detect_f32<M, 13>;
        case 14: return launch_detect_f32<M, 14>;
        case 15: return launch_detect_f32<M, 15>;
        case 16: return launch_detect_f32<M, 16>;
        default: return nullptr;
    }
}

DetectBwdLauncher APSM_CAT(detect_bwd_launcher_m, APSM_DETECT_M)(int K) {
    constexpr int M = APSM_DETECT_M;
    switch (K) {
        case 1: return launch_detect_bwd<M, 1>;
        case 2: return launch_detect_bwd<M, 2>;
        case 3: return launch_detect_bwd<M, 3>;
        case 4: return launch_detect_bwd<M, 4>;
        case 5: return launch_detect_bwd<M, 5>;
        case 6: return launch_detect_bwd<M, 6>;
        case 7: return launch_detect_bwd<M, 7>;
        case 8: return launch_detect_bwd<M, 8>;
        case 9: return launch_detect_bwd<M, 9>;
        case 10: return launch_detect_bwd<M, 10>;
        case 11: return launch_detect_bwd<M, 11>;
        case 12: return launch_detect_bwd<M, 12>;
        case 13: return launch_detect_bwd<M, 13>;
        case 14: return launch_detect_bwd<M, 14>;
        case 15: return launch_detect_bwd<M, 15>;
        case 16: return launch_detect_bwd<M, 16>;
        default: return nullptr;
    }
}

}  // namespace apsm
