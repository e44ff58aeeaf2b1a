// train_chunk.cu -- instantiations of the phase-B training kernel for every supported
// (live-range registers S, padded window WP) pair, and the host-side launcher table.
#include "train_f32.cuh"

namespace apsm {

// One CTA per (chunk, 32 x 32 sample tile of one table).  The tile's 16 row and 16 column pilots
// are staged in shared memory with their norms; each thread takes one pilot pair, whose complex
// inner product z = r_a^H r_b gives all four real-split sample pairs:
//   r1(a).r1(b) = r2(a).r2(b) = Re z,  r1(a).r2(b) = Im z,  r2(a).r1(b) = -Im z,
//   ||x_a - x_b||^2 = ||r_a||^2 + ||r_b||^2 - 2 x_a.x_b.
// Tables: 0 = kmat (live range x live range, sum kernel), 1 = gev (dropped entries x live range,
// Gaussian), 2 = kx (live range x next chunk's samples, sum kernel).
__global__ void __launch_bounds__(256) train_gram_kernel(const float2 *__restrict__ rx, TrainGeom g, float k2, float wL,
                                                         float wG, float *__restrict__ kmat, float *__restrict__ gev,
                                                         float *__restrict__ kx) {
    extern __shared__ __align__(16) float2 s_gram[];
    pdl_enter();
    const int c = blockIdx.y;
    int t0, Tc, s0, s1, l0;
    chunk_range(g, c, t0, Tc, s0, s1, l0);
    const int M = g.M, MS = g.M + 1;  // padded row of a staged pilot (bank spread)
    float2 *s_row = s_gram, *s_col = s_gram + 16 * MS;
    float *s_nrm = reinterpret_cast<float *>(s_gram + 32 * MS);  // [0,16) rows, [16,32) columns
    const int RT = g.RS / 32, ET = (2 * g.T + 31) / 32, XT = g.KXS / 32;
    const int n_ev = g.P > g.D ? ET * RT : 0;
    const int n_next = c + 1 < g.n_chunks ? 2 * min(g.T, g.P - t0 - Tc) : 0;
    int job = blockIdx.x, table, rt, ct;
    if (job < RT * RT) {
        table = 0; rt = job / RT; ct = job % RT;
    } else if ((job -= RT * RT) < n_ev) {
        table = 1; rt = job / RT; ct = job % RT;
    } else {
        job -= n_ev;
        if (!g.track || job >= RT * XT) return;
        table = 2; rt = job / XT; ct = job % XT;
    }
    // pilot of staged row / column i (-1: outside the table's valid range)
    auto row_pilot = [&](int i) {
        if (table == 1) {
            const int e = 16 * rt + i;
            return (e < Tc && t0 + e >= g.D) ? t0 + e - g.D : -1;
        }
        const int smp = l0 + 32 * rt + 2 * i;
        return smp < s1 ? smp >> 1 : -1;
    };
    auto col_pilot = [&](int j) {
        if (table == 2) {
            const int v = 32 * ct + 2 * j;
            return v < n_next ? t0 + Tc + (v >> 1) : -1;
        }
        const int smp = l0 + 32 * ct + 2 * j;
        return smp < s1 ? smp >> 1 : -1;
    };
    for (int idx = threadIdx.x; idx < 32 * M; idx += blockDim.x) {
        const int i = idx / M, mm = idx % M;
        const int pr = i < 16 ? row_pilot(i) : col_pilot(i - 16);
        const float2 v = pr >= 0 ? __ldg(rx + (size_t)pr * M + mm) : make_float2(0.f, 0.f);
        (i < 16 ? s_row + i * MS : s_col + (i - 16) * MS)[mm] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const float2 *r = threadIdx.x < 16 ? s_row + threadIdx.x * MS : s_col + (threadIdx.x - 16) * MS;
        float n = 0.f;
        for (int mm = 0; mm < M; ++mm) n = fmaf(r[mm].x, r[mm].x, fmaf(r[mm].y, r[mm].y, n));
        s_nrm[threadIdx.x] = n;
    }
    __syncthreads();
    const int i = threadIdx.x >> 4, j = threadIdx.x & 15;
    const bool ok = row_pilot(i) >= 0 && col_pilot(j) >= 0;
    const float2 *ra = s_row + i * MS, *rb = s_col + j * MS;
    float zr = 0.f, zi = 0.f;
    for (int mm = 0; mm < M; ++mm) {
        const float2 x = ra[mm], y = rb[mm];
        zr = fmaf(x.x, y.x, fmaf(x.y, y.y, zr));
        zi = fmaf(x.x, y.y, fmaf(-x.y, y.x, zi));
    }
    const float nn = s_nrm[i] + s_nrm[16 + j];
    float out[2][2];
#pragma unroll
    for (int la = 0; la < 2; ++la)
#pragma unroll
        for (int lb = 0; lb < 2; ++lb) {
            const float dot = (la == lb) ? zr : (la == 0 ? zi : -zi);
            const float ge = ex2(-k2 * fmaxf(nn - 2.f * dot, 0.f));
            const float val = table == 1 ? ge : fmaf(wL, dot, wG * ge);  // sum kernel (Fact 1)
            out[la][lb] = ok ? val : 0.f;
        }
    const int row0 = 32 * rt + 2 * i, col = 32 * ct + 2 * j;
#pragma unroll
    for (int la = 0; la < 2; ++la) {
        const float2 v = make_float2(out[la][0], out[la][1]);
        if (table == 0) {
            reinterpret_cast<float2 *>(kmat + ((size_t)c * g.RS + row0 + la) * g.RS + col)[0] = v;
        } else if (table == 1) {
            if (row0 + la < 2 * g.T)
                reinterpret_cast<float2 *>(gev + ((size_t)c * 2 * g.T + row0 + la) * g.RS + col)[0] = v;
        } else {
            reinterpret_cast<float2 *>(kx + ((size_t)c * g.RS + row0 + la) * g.KXS + col)[0] = v;
        }
    }
}

cudaError_t launch_train_gram(const float2 *rx, const TrainGeom &g, float k2, float wL, float wG, float *kmat,
                              float *gev, float *kx, cudaStream_t stream) {
    const int RT = g.RS / 32, ET = (2 * g.T + 31) / 32, XT = g.KXS / 32;
    const int jobs = RT * RT + (g.P > g.D ? ET * RT : 0) + (g.track ? RT * XT : 0);
    const size_t smem = (size_t)32 * (g.M + 1) * sizeof(float2) + 32 * sizeof(float);
    cudaError_t e = launch_pdl(train_gram_kernel, dim3(jobs, g.n_chunks), dim3(256), smem, stream, rx, g, k2, wL,
                               wG, kmat, gev, kx);
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
