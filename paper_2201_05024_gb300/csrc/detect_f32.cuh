// detect_f32.cuh -- fused FP32 detection kernel (Sec. III-B detection, Sec. III-C inner products).
//
// For every complex data vector r_s and user k it evaluates
//   y1 = f^k(r1(s)) = w_L Re(c_k^H r_s) + w_G sum_t [g1_t E_A + g2_t E_C]
//   y2 = f^k(r2(s)) = w_L Im(c_k^H r_s) + w_G sum_t [g1_t E_B + g2_t E_A]
// over the dictionary entries t, where (z = r_t^H r_s, n = ||r||^2, 2 sigma^2 = s2)
//   E_A = exp(-(n_t + n_s - 2 Re z)/s2)   centre r1(t) vs r1(s)  (= r2(t) vs r2(s))
//   E_B = exp(-(n_t + n_s - 2 Im z)/s2)   centre r1(t) vs r2(s)
//   E_C = exp(-(n_t + n_s + 2 Im z)/s2)   centre r2(t) vs r1(s)
// One complex inner product per (query, entry) pair yields all four real-split Gaussian kernel
// values of Sec. II-A (r2 is r1 rotated, so distances between like halves coincide).
//
// Layout and schedule (GB300):
//  - each thread keeps QPT query vectors in registers and streams the whole dictionary past
//    them, so accumulators never leave the thread and no reduction is needed;
//  - dictionary tiles (entries, norms, coefficients; contiguous in the state) are staged into a
//    two-stage shared-memory ring by the bulk-copy engine (cp.async.bulk + mbarrier), issued by
//    one thread one tile ahead of the compute; all threads read a tile entry by broadcast;
//  - exponentials run on MUFU (ex2.approx); the norm-expansion distance is clamped at 0.
//  - partial mode (training, phase A): the grid's y dimension splits the entries into slices;
//    each slice writes its raw Gaussian sums [slice][query][2K] without the linear part.
#pragma once

#include "apsm_common.cuh"

namespace apsm {

struct DetectArgs {
    const float2 *rx;          // [N][M] queries
    int N;
    const float2 *dict;        // [A][M]
    const float *dict_norm;    // [A]
    const float *gamma;        // [A][2][K]
    const float2 *clin;        // [M][K]
    const int *meta;           // device entry count (meta[0]); nullable
    int n_entries;             // host upper bound on entries
    int slice_entries;         // entries per grid.y slice (multiple of kTileEntries)
    float k2;                  // log2(e) / (2 sigma^2)
    float wL, wG;
    float2 *soft;              // [N][K] full mode
    uint8_t *hard;             // [N][K] nullable
    float *partial;            // [gridDim.y][N][2K] partial mode (full mode: nullptr)
    int *status;               // device status word
};

template <int M, int K>
struct DetectSmem {
    static constexpr int kDictBytes = kTileEntries * M * 8;
    static constexpr int kNormBytes = kTileEntries * 4;
    static constexpr int kGamBytes = kTileEntries * 2 * K * 4;
    static constexpr int kStageBytes = round_up(kDictBytes + kNormBytes + kGamBytes, 128);
    static constexpr int kClinOffset = 128 + 2 * kStageBytes;
    static constexpr int kBytes = kClinOffset + M * K * 8;
};

template <int M, int K, int QPT>
__global__ void __launch_bounds__(256) detect_f32_kernel(const DetectArgs a) {
    using S = DetectSmem<M, K>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    unsigned char *stage0 = smem + 128;
    float2 *s_clin = reinterpret_cast<float2 *>(smem + S::kClinOffset);

    int n_ent = a.n_entries;
    if (a.meta) n_ent = min(n_ent, max(__ldg(a.meta), 0));
    const int e_begin = blockIdx.y * a.slice_entries;
    const int e_end = min(n_ent, e_begin + a.slice_entries);
    const int n_tiles = e_end > e_begin ? (e_end - e_begin + kTileEntries - 1) / kTileEntries : 0;

    auto issue = [&](int tile) {
        unsigned char *st = stage0 + (tile & 1) * S::kStageBytes;
        const int e0 = e_begin + tile * kTileEntries;
        mbar_arrive_expect_tx(&bar[tile & 1], S::kDictBytes + S::kNormBytes + S::kGamBytes);
        bulk_g2s(st, a.dict + (size_t)e0 * M, S::kDictBytes, &bar[tile & 1]);
        bulk_g2s(st + S::kDictBytes, a.dict_norm + e0, S::kNormBytes, &bar[tile & 1]);
        bulk_g2s(st + S::kDictBytes + S::kNormBytes, a.gamma + (size_t)e0 * 2 * K, S::kGamBytes, &bar[tile & 1]);
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    if (a.partial == nullptr)
        for (int i = threadIdx.x; i < M * K; i += blockDim.x) s_clin[i] = a.clin[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        if (n_tiles > 0) issue(0);
        if (n_tiles > 1) issue(1);
    }

    // Queries of this thread, in registers.
    const int q_base = blockIdx.x * blockDim.x * QPT + threadIdx.x;
    float2 r[QPT][M];
    float hq[QPT];  // -k2 * n_s
#pragma unroll
    for (int i = 0; i < QPT; ++i) {
        const int q = q_base + i * blockDim.x;
        float n = 0.f;
        if (q < a.N) {
            const float4 *src = reinterpret_cast<const float4 *>(a.rx + (size_t)q * M);
#pragma unroll
            for (int m = 0; m < M / 2; ++m) {
                const float4 v = __ldg(src + m);
                r[i][2 * m] = make_float2(v.x, v.y);
                r[i][2 * m + 1] = make_float2(v.z, v.w);
            }
        } else {
#pragma unroll
            for (int m = 0; m < M; ++m) r[i][m] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int m = 0; m < M; ++m) n = fmaf(r[i][m].x, r[i][m].x, fmaf(r[i][m].y, r[i][m].y, n));
        hq[i] = -a.k2 * n;
    }

    float acc1[QPT][K], acc2[QPT][K];
#pragma unroll
    for (int i = 0; i < QPT; ++i)
#pragma unroll
        for (int k = 0; k < K; ++k) acc1[i][k] = acc2[i][k] = 0.f;

    const float g2 = 2.f * a.k2;
    for (int tile = 0; tile < n_tiles; ++tile) {
        const bool ok = mbar_wait_bounded(&bar[tile & 1], (tile >> 1) & 1);
        if (ok) {
            const unsigned char *st = stage0 + (tile & 1) * S::kStageBytes;
            const float2 *sd = reinterpret_cast<const float2 *>(st);
            const float *sn = reinterpret_cast<const float *>(st + S::kDictBytes);
            const float *sg = reinterpret_cast<const float *>(st + S::kDictBytes + S::kNormBytes);
            const int cnt = min(kTileEntries, e_end - (e_begin + tile * kTileEntries));
#pragma unroll 1
            for (int t = 0; t < cnt; ++t) {
                // complex inner product z = r_t^H r_s for every query of the thread
                float zr0[QPT], zi0[QPT], zr1[QPT], zi1[QPT];
#pragma unroll
                for (int i = 0; i < QPT; ++i) zr0[i] = zi0[i] = zr1[i] = zi1[i] = 0.f;
                const float4 *d4 = reinterpret_cast<const float4 *>(sd + t * M);
#pragma unroll
                for (int m = 0; m < M / 2; ++m) {
                    const float4 d = d4[m];
#pragma unroll
                    for (int i = 0; i < QPT; ++i) {
                        const float2 x0 = r[i][2 * m], x1 = r[i][2 * m + 1];
                        zr0[i] = fmaf(d.x, x0.x, zr0[i]);
                        zr0[i] = fmaf(d.y, x0.y, zr0[i]);
                        zi0[i] = fmaf(d.x, x0.y, zi0[i]);
                        zi0[i] = fmaf(-d.y, x0.x, zi0[i]);
                        zr1[i] = fmaf(d.z, x1.x, zr1[i]);
                        zr1[i] = fmaf(d.w, x1.y, zr1[i]);
                        zi1[i] = fmaf(d.z, x1.y, zi1[i]);
                        zi1[i] = fmaf(-d.w, x1.x, zi1[i]);
                    }
                }
                const float ht = -a.k2 * sn[t];
                float gm1[K], gm2[K];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    gm1[k] = sg[t * 2 * K + k];
                    gm2[k] = sg[t * 2 * K + K + k];
                }
#pragma unroll
                for (int i = 0; i < QPT; ++i) {
                    const float zr = zr0[i] + zr1[i], zi = zi0[i] + zi1[i];
                    const float h = hq[i] + ht;  // -k2 (n_s + n_t)
                    const float eA = ex2(fminf(fmaf(g2, zr, h), 0.f));
                    const float eB = ex2(fminf(fmaf(g2, zi, h), 0.f));
                    const float eC = ex2(fminf(fmaf(-g2, zi, h), 0.f));
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        acc1[i][k] = fmaf(gm1[k], eA, fmaf(gm2[k], eC, acc1[i][k]));
                        acc2[i][k] = fmaf(gm1[k], eB, fmaf(gm2[k], eA, acc2[i][k]));
                    }
                }
            }
        }
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) report(a.status, APSM_ERR_TIMEOUT);
            return;
        }
        if (threadIdx.x == 0 && tile + 2 < n_tiles) issue(tile + 2);
    }

#pragma unroll
    for (int i = 0; i < QPT; ++i) {
        const int q = q_base + i * blockDim.x;
        if (q >= a.N) continue;
        if (a.partial != nullptr) {
            float *dst = a.partial + ((size_t)blockIdx.y * a.N + q) * 2 * K;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                dst[k] = acc1[i][k];
                dst[K + k] = acc2[i][k];
            }
            continue;
        }
        unsigned char hbits[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float l1 = 0.f, l2 = 0.f;  // c_k^H r = sum_m conj(c[m][k]) r[m]
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const float2 c = s_clin[m * K + k];
                l1 = fmaf(c.x, r[i][m].x, fmaf(c.y, r[i][m].y, l1));
                l2 = fmaf(c.x, r[i][m].y, fmaf(-c.y, r[i][m].x, l2));
            }
            const float y1 = fmaf(a.wL, l1, a.wG * acc1[i][k]);
            const float y2 = fmaf(a.wL, l2, a.wG * acc2[i][k]);
            a.soft[(size_t)q * K + k] = make_float2(y1, y2);
            hbits[k] = (unsigned char)((y1 < 0.f ? 1 : 0) | (y2 < 0.f ? 2 : 0));
        }
        if (a.hard) {
#pragma unroll
            for (int k = 0; k < K; ++k) a.hard[(size_t)q * K + k] = hbits[k];
        }
    }
}

// Host-side launcher for one (M, K) instantiation.
template <int M, int K>
cudaError_t launch_detect_f32(const DetectArgs &a, int grid_y, int threads, int qpt, cudaStream_t stream) {
    using S = DetectSmem<M, K>;
    const int per_cta = threads * qpt;
    const int gx = (a.N + per_cta - 1) / per_cta;
    if (gx == 0 || grid_y == 0) return cudaSuccess;
    dim3 grid(gx, grid_y);
    if constexpr (M <= 16) {
        if (qpt == 2) {
            auto fn = detect_f32_kernel<M, K, 2>;
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
            if (e != cudaSuccess) return e;
            fn<<<grid, threads, S::kBytes, stream>>>(a);
            return cudaGetLastError();
        }
    }
    {
        auto fn = detect_f32_kernel<M, K, 1>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
        if (e != cudaSuccess) return e;
        fn<<<grid, threads, S::kBytes, stream>>>(a);
    }
    return cudaGetLastError();
}

using DetectLauncher = cudaError_t (*)(const DetectArgs &, int, int, int, cudaStream_t);

}  // namespace apsm
