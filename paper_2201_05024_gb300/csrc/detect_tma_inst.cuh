// detect_tma_inst.cuh -- instantiates the TMA-staged detection kernel for one antenna count
// (APSM_TMA_M) and every even user count that is its own bucket.
#pragma once

#include "detect_tma.cuh"

#define APSM_TMA_CAT2(a, b) a##b
#define APSM_TMA_CAT(a, b) APSM_TMA_CAT2(a, b)

namespace apsm {

TmaLauncher APSM_TMA_CAT(detect_tma_launcher_m, APSM_TMA_M)(int K) {
    constexpr int M = APSM_TMA_M;
    switch (K) {
        case 2: return launch_detect_tma<M, 2>;
        case 4: return launch_detect_tma<M, 4>;
        case 6: return launch_detect_tma<M, 6>;
        case 8: return launch_detect_tma<M, 8>;
        case 12: return launch_detect_tma<M, 12>;
        case 16: return launch_detect_tma<M, 16>;
        default: return nullptr;
    }
}

}  // namespace apsm
