// train_chunk.cu -- instantiations of the phase-B training kernel for every supported
// (live-range registers S, padded window WP) pair, and the host-side launcher table.
#include "train_f32.cuh"

namespace apsm {

__global__ void train_gram_kernel(const float2 *__restrict__ rx, TrainGeom g, float k2, float wL, float wG,
                                  float *__restrict__ kmat, float *__restrict__ gev) {
    pdl_enter();
    const int c = blockIdx.y;
    int t0, Tc, s0, s1, l0;
    chunk_range(g, c, t0, Tc, s0, s1, l0);
    const int R = s1 - l0;
    const int RS = g.RS;
    const int n_k = RS * RS, n_e = g.T * 2 * RS;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n_k + n_e; idx += gridDim.x * blockDim.x) {
        if (idx < n_k) {
            const int u = idx / RS, v = idx % RS;
            float val = 0.f;
            if (u < R && v < R) {
                const int mu_ = l0 + u, mv = l0 + v;
                float dot, d2;
                sample_pair(rx + (size_t)(mu_ >> 1) * g.M, rx + (size_t)(mv >> 1) * g.M, g.M, mu_ & 1, mv & 1, dot,
                            d2);
                val = fmaf(wL, dot, wG * ex2(-k2 * d2));  // kappa = w_L kappa_L + w_G kappa_G (Fact 1)
            }
            kmat[(size_t)c * n_k + idx] = val;
        } else {
            const int j = idx - n_k;
            const int e = j / (2 * RS), l = (j / RS) & 1, v = j % RS;
            const int t = t0 + e;
            float val = 0.f;
            if (e < Tc && t >= g.D && v < R) {
                const int mv = l0 + v;
                float dot, d2;
                sample_pair(rx + (size_t)(t - g.D) * g.M, rx + (size_t)(mv >> 1) * g.M, g.M, l, mv & 1, dot, d2);
                val = ex2(-k2 * d2);
            }
            gev[(size_t)c * n_e + j] = val;
        }
    }
}

cudaError_t launch_train_gram(const float2 *rx, const TrainGeom &g, float k2, float wL, float wG, float *kmat,
                              float *gev, cudaStream_t stream) {
    const int per_chunk = g.RS * g.RS + g.T * 2 * g.RS;
    dim3 grid((per_chunk + 255) / 256, g.n_chunks);
    cudaError_t e = launch_pdl(train_gram_kernel, grid, dim3(256), 0, stream, rx, g, k2, wL, wG, kmat, gev);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <int S, int WP>
cudaError_t launch_chunk_sw(const ChunkArgs &a, int smem, cudaStream_t stream) {
    auto fn = train_chunk_kernel<S, WP>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = launch_pdl(fn, dim3(a.g.K), dim3(32 * S), smem, stream, a);
    return e != cudaSuccess ? e : cudaGetLastError();
}

using ChunkLauncher = cudaError_t (*)(const ChunkArgs &, int, cudaStream_t);

// Smallest supported padded window >= W (0 if W is too large).
int padded_window(int W) {
    static const int kWP[] = {4, 8, 12, 16, 20, 24, 32, 48, 64, 96, 128};
    for (int wp : kWP)
        if (wp >= W) return wp;
    return 0;
}

ChunkLauncher chunk_launcher(int S, int WP) {
    switch (S * 1000 + WP) {
        case 1004: return launch_chunk_sw<1, 4>;
        case 1008: return launch_chunk_sw<1, 8>;
        case 1012: return launch_chunk_sw<1, 12>;
        case 1016: return launch_chunk_sw<1, 16>;
        case 1020: return launch_chunk_sw<1, 20>;
        case 1024: return launch_chunk_sw<1, 24>;
        case 1032: return launch_chunk_sw<1, 32>;
        case 2004: return launch_chunk_sw<2, 4>;
        case 2008: return launch_chunk_sw<2, 8>;
        case 2012: return launch_chunk_sw<2, 12>;
        case 2016: return launch_chunk_sw<2, 16>;
        case 2020: return launch_chunk_sw<2, 20>;
        case 2024: return launch_chunk_sw<2, 24>;
        case 2032: return launch_chunk_sw<2, 32>;
        case 2048: return launch_chunk_sw<2, 48>;
        case 2064: return launch_chunk_sw<2, 64>;
        case 3004: return launch_chunk_sw<3, 4>;
        case 3008: return launch_chunk_sw<3, 8>;
        case 3012: return launch_chunk_sw<3, 12>;
        case 3016: return launch_chunk_sw<3, 16>;
        case 3020: return launch_chunk_sw<3, 20>;
        case 3024: return launch_chunk_sw<3, 24>;
        case 3032: return launch_chunk_sw<3, 32>;
        case 3048: return launch_chunk_sw<3, 48>;
        case 3064: return launch_chunk_sw<3, 64>;
        case 3096: return launch_chunk_sw<3, 96>;
        case 4004: return launch_chunk_sw<4, 4>;
        case 4008: return launch_chunk_sw<4, 8>;
        case 4012: return launch_chunk_sw<4, 12>;
        case 4016: return launch_chunk_sw<4, 16>;
        case 4020: return launch_chunk_sw<4, 20>;
        case 4024: return launch_chunk_sw<4, 24>;
        case 4032: return launch_chunk_sw<4, 32>;
        case 4048: return launch_chunk_sw<4, 48>;
        case 4064: return launch_chunk_sw<4, 64>;
        case 4096: return launch_chunk_sw<4, 96>;
        case 4128: return launch_chunk_sw<4, 128>;
        case 5004: return launch_chunk_sw<5, 4>;
        case 5008: return launch_chunk_sw<5, 8>;
        case 5012: return launch_chunk_sw<5, 12>;
        case 5016: return launch_chunk_sw<5, 16>;
        case 5020: return launch_chunk_sw<5, 20>;
        case 5024: return launch_chunk_sw<5, 24>;
        case 5032: return launch_chunk_sw<5, 32>;
        case 5048: return launch_chunk_sw<5, 48>;
        case 5064: return launch_chunk_sw<5, 64>;
        case 5096: return launch_chunk_sw<5, 96>;
        case 5128: return launch_chunk_sw<5, 128>;
        default: return nullptr;
    }
}

}  // namespace apsm
