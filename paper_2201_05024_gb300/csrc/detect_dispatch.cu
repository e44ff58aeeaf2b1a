// detect_dispatch.cu -- maps (M, K) to the FP32 detection kernels (and adjoint) instantiated for it.
#include "detect_bwd.cuh"
#include "detect_f32.cuh"

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
