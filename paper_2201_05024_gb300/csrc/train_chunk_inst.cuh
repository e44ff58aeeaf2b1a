// train_chunk_inst.cuh -- instantiates the phase-B training kernel for one live-range warp count
// (APSM_CHUNK_S) and every padded window it supports, with its launcher table.
#pragma once

#include "train_f32.cuh"

#define APSM_CHUNK_CAT2(a, b) a##b
#define APSM_CHUNK_CAT(a, b) APSM_CHUNK_CAT2(a, b)

namespace apsm {

using ChunkLauncher = cudaError_t (*)(const ChunkArgs &, int, cudaStream_t);

template <int S, int WP, bool kExt>
cudaError_t launch_chunk_sw(const ChunkArgs &a, int smem, cudaStream_t stream) {
    auto fn = train_chunk_kernel<S, WP, kExt>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = launch_pdl(fn, dim3(a.g.K), dim3(32 * S), smem, stream, a);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <bool kExt>
ChunkLauncher chunk_table(int WP) {
    constexpr int S = APSM_CHUNK_S;
    switch (WP) {
        case 4: return launch_chunk_sw<S, 4, kExt>;
        case 8: return launch_chunk_sw<S, 8, kExt>;
        case 12: return launch_chunk_sw<S, 12, kExt>;
        case 16: return launch_chunk_sw<S, 16, kExt>;
        case 20: return launch_chunk_sw<S, 20, kExt>;
        case 24: return launch_chunk_sw<S, 24, kExt>;
        case 32: return launch_chunk_sw<S, 32, kExt>;
        default: break;
    }
    if constexpr (S >= 2) {
        if (WP == 48) return launch_chunk_sw<S, 48, kExt>;
        if (WP == 64) return launch_chunk_sw<S, 64, kExt>;
    }
    if constexpr (S >= 3) {
        if (WP == 96) return launch_chunk_sw<S, 96, kExt>;
    }
    if constexpr (S >= 4) {
        if (WP == 128) return launch_chunk_sw<S, 128, kExt>;
    }
    return nullptr;
}

// One launcher table per translation unit: live-range warp count APSM_CHUNK_S, plain or extended
// instantiations (APSM_CHUNK_EXT); padded windows per S: S = 1 holds up to 32 live-range samples
// (windows <= 32), S = 2 up to 64, and so on.
ChunkLauncher APSM_CHUNK_CAT(APSM_CHUNK_CAT(chunk_launcher_s, APSM_CHUNK_S), APSM_CHUNK_CAT(_x, APSM_CHUNK_EXT))(int WP) {
    return chunk_table<APSM_CHUNK_EXT != 0>(WP);
}

}  // namespace apsm
