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
// With k2 = log2(e)/s2 the exponentials factor as
//   E_A = 2^(-k2 n_s) * 2^(-k2 n_t) * 2^(2 k2 Re z)      (likewise E_B, E_C with +-Im z),
// so the query factor is applied once after the sum, the entry factor is folded into the
// entry's coefficients once per tile, and a pair costs its inner product, three MUFU ex2 and
// the coefficient FMAs -- no per-pair adds.  The factored form is exact in real arithmetic and
// keeps every factor inside the FP32 range while k2 n <= kFactorLimit for all queries and
// entries involved (then |2 k2 z| <= k2 (n_s + n_t) <= 2 kFactorLimit); a tile or a CTA outside
// that range takes a guarded form that forms each squared distance by direct differences.
// Inside the range the norm expansion costs at most ~2 kFactorLimit FP32 roundings of absolute
// error in the exponent (a relative error of a few 1e-5 in E at the range's edge, ~1e-6 for
// unit-energy inputs); outside it the guarded form has no cancellation at all.
//
// Layout and schedule (GB300):
//  - each thread keeps QPT query vectors in registers and streams the whole dictionary past
//    them, so accumulators never leave the thread and no reduction is needed;
//  - dictionary tiles (entries, norms, coefficients; contiguous in the state) are staged into a
//    two-stage shared-memory ring by the bulk-copy engine (cp.async.bulk + mbarrier), issued by
//    one thread one tile ahead of the compute; all threads read a tile entry by broadcast;
//  - the CTA's threadIdx.y groups take alternate entries of every staged tile for the same
//    queries (more resident warps without more shared-memory traffic) and merge their partial
//    sums in a fixed order at the end, so results are deterministic;
//  - exponentials run on MUFU (ex2.approx);
//  - partial mode (training, phase A): the grid's y dimension splits the entries into slices;
//    each slice writes its raw Gaussian sums [slice][query][2K] without the linear part.
#pragma once

#include "apsm_common.cuh"

namespace apsm {

constexpr float kFactorLimit = 60.f;

#ifndef APSM_DETECT_UNROLL
#define APSM_DETECT_UNROLL 2
#endif
constexpr int kDetectUnroll = APSM_DETECT_UNROLL;

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
    // Optional slot segments (partial mode): when seg0_hi or seg1_hi is nonzero, grid.y slices
    // [0, seg_slices) cover slots [seg0_lo, seg0_hi) and the rest cover [seg1_lo, seg1_hi), each
    // segment sliced from its first 32-slot tile boundary; slots below a segment start are masked.
    int seg_slices, seg0_lo, seg0_hi, seg1_lo, seg1_hi;
    // Launched beside a training chunk whose own wait has already covered everything this launch
    // reads: let the successor launch at once, skip the wait at the start, and wait for the
    // predecessor (that chunk) only before exiting, so that completion still orders the stream.
    int pdl_late;
};

template <int M, int K>
struct DetectSmem {
    static constexpr int kDictBytes = kTileEntries * M * 8;
    static constexpr int kNormBytes = kTileEntries * 4;
    static constexpr int kGamBytes = kTileEntries * 2 * K * 4;
    static constexpr int kStageBytes = round_up(kDictBytes + kNormBytes + kGamBytes, 128);
    static constexpr int kScaledOffset = 128 + 2 * kStageBytes;          // coefficients x entry factor
    static constexpr int kFlagOffset = kScaledOffset + kGamBytes;        // tile in factor range
    static constexpr int kClinOffset = round_up(kFlagOffset + 16, 16);
    static constexpr int kReduceOffset = round_up(kClinOffset + M * K * 8, 16);  // entry-split merge
    // total for a CTA of `threads` x `split` threads with `qpt` queries per thread
    static constexpr int bytes(int threads, int split, int qpt) {
        return kReduceOffset + (split > 1 ? (split - 1) * threads * qpt * 2 * K * 4 : 0);
    }
};

// 2K consecutive floats from shared memory with the widest aligned vector loads.
template <int K>
__device__ __forceinline__ void load_coef(const float *src, float (&g1)[K], float (&g2)[K]) {
    float v[2 * K];
    if constexpr ((2 * K) % 4 == 0) {
#pragma unroll
        for (int j = 0; j < 2 * K; j += 4) {
            const float4 x = *reinterpret_cast<const float4 *>(src + j);
            v[j] = x.x; v[j + 1] = x.y; v[j + 2] = x.z; v[j + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 2 * K; j += 2) {
            const float2 x = *reinterpret_cast<const float2 *>(src + j);
            v[j] = x.x; v[j + 1] = x.y;
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        g1[k] = v[k];
        g2[k] = v[K + k];
    }
}

// Packed FP32 pair FMA (Blackwell): (d0, d1) = (a0 * b + d0, a1 * b + d1), each lane an IEEE
// fma with one rounding, so results equal two fmaf calls bit for bit in half the instructions.
__device__ __forceinline__ void fma2_pair(float &d0, float &d1, float a0, float a1, float b) {
    asm("{\n\t.reg .b64 d, a, b;\n\t"
        "mov.b64 d, {%0, %1};\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %4};\n\t"
        "fma.rn.f32x2 d, a, b, d;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "+f"(d0), "+f"(d1)
        : "f"(a0), "f"(a1), "f"(b));
}

// Lanes per query vector: from 64 antennas on, the query (2M floats) would not fit the register
// file beside the accumulators, so two adjacent lanes share a query, each holding half of its
// antennas and accumulating half of the users; their partial inner products meet by one shuffle.
template <int M>
constexpr int query_lanes() { return M >= 64 ? 2 : 1; }

// The KH coefficients (both halves) of the users part * KH + j that a lane of a shared query
// accumulates; a user index past K (odd K, second lane) reads a duplicate that is never stored.
template <int K, int KH>
__device__ __forceinline__ void load_coef_part(const float *src, int part, float (&g1)[KH], float (&g2)[KH]) {
    if constexpr (KH == K) {
        load_coef<K>(src, g1, g2);
    } else if constexpr (KH % 4 == 0 && K % 4 == 0) {
        const float *s1 = src + part * KH, *s2 = src + K + part * KH;
#pragma unroll
        for (int j = 0; j < KH; j += 4) {
            const float4 x = *reinterpret_cast<const float4 *>(s1 + j);
            const float4 y = *reinterpret_cast<const float4 *>(s2 + j);
            g1[j] = x.x; g1[j + 1] = x.y; g1[j + 2] = x.z; g1[j + 3] = x.w;
            g2[j] = y.x; g2[j + 1] = y.y; g2[j + 2] = y.z; g2[j + 3] = y.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < KH; ++j) {
            const int k = min(part * KH + j, K - 1);
            g1[j] = src[k];
            g2[j] = src[K + k];
        }
    }
}

template <int M, int K, int QPT>
__global__ void __launch_bounds__(256) detect_f32_kernel(const DetectArgs a) {
    constexpr int QS = query_lanes<M>();               // lanes per query
    constexpr int MH = M / QS, KH = (K + QS - 1) / QS;  // antennas and users per lane
    using S = DetectSmem<M, K>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    unsigned char *stage0 = smem + 128;
    float *s_gs = reinterpret_cast<float *>(smem + S::kScaledOffset);
    int *s_flag = reinterpret_cast<int *>(smem + S::kFlagOffset);
    float2 *s_clin = reinterpret_cast<float2 *>(smem + S::kClinOffset);
    float *s_red = reinterpret_cast<float *>(smem + S::kReduceOffset);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nthreads = blockDim.x * blockDim.y;
    if (a.pdl_late) pdl_trigger();
    else pdl_enter();

    int n_ent = a.n_entries;
    if (a.meta) n_ent = min(n_ent, max(__ldcg(a.meta), 0));
    int e_begin, e_end, e_lo = 0;
    if (a.seg0_hi > 0 || a.seg1_hi > 0) {
        const bool second = (int)blockIdx.y >= a.seg_slices;
        const int lo = second ? a.seg1_lo : a.seg0_lo, hi = second ? a.seg1_hi : a.seg0_hi;
        const int sl = second ? (int)blockIdx.y - a.seg_slices : (int)blockIdx.y;
        e_begin = lo / kTileEntries * kTileEntries + sl * a.slice_entries;
        e_end = min(hi, e_begin + a.slice_entries);
        e_lo = lo;
    } else {
        e_begin = blockIdx.y * a.slice_entries;
        e_end = min(n_ent, e_begin + a.slice_entries);
    }
    const int n_tiles = e_end > e_begin ? (e_end - e_begin + kTileEntries - 1) / kTileEntries : 0;

    auto issue = [&](int tile) {
        unsigned char *st = stage0 + (tile & 1) * S::kStageBytes;
        const int e0 = e_begin + tile * kTileEntries;
        mbar_arrive_expect_tx(&bar[tile & 1], S::kDictBytes + S::kNormBytes + S::kGamBytes);
        bulk_g2s(st, a.dict + (size_t)e0 * M, S::kDictBytes, &bar[tile & 1]);
        bulk_g2s(st + S::kDictBytes, a.dict_norm + e0, S::kNormBytes, &bar[tile & 1]);
        bulk_g2s(st + S::kDictBytes + S::kNormBytes, a.gamma + (size_t)e0 * 2 * K, S::kGamBytes, &bar[tile & 1]);
    };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    if (a.partial == nullptr)
        for (int i = tid; i < M * K; i += nthreads) s_clin[i] = __ldcg(a.clin + i);
    __syncthreads();
    if (tid == 0) {
        if (n_tiles > 0) issue(0);
        if (n_tiles > 1) issue(1);
    }

    // Queries of this thread, in registers, pre-scaled by g2 = 2 k2 so that the inner product
    // directly gives the exponent 2 k2 z of the factored form.
    const float g2 = 2.f * a.k2;
    const int part = QS > 1 ? (int)threadIdx.x % QS : 0;  // which half of the antennas / users
    const int qlanes = blockDim.x / QS;                    // queries per entry group and QPT step
    const int q_base = blockIdx.x * qlanes * QPT + threadIdx.x / QS;
    float2 r[QPT][MH];
    float hq[QPT];  // -k2 * n_s
    bool q_in_range = true;
#pragma unroll
    for (int i = 0; i < QPT; ++i) {
        const int q = q_base + i * qlanes;
        float n = 0.f;
        if (q < a.N) {
            const float4 *src = reinterpret_cast<const float4 *>(a.rx + (size_t)q * M + part * MH);
#pragma unroll
            for (int m = 0; m < MH / 2; ++m) {
                const float4 v = __ldcg(src + m);
                r[i][2 * m] = make_float2(v.x, v.y);
                r[i][2 * m + 1] = make_float2(v.z, v.w);
            }
        } else {
#pragma unroll
            for (int m = 0; m < MH; ++m) r[i][m] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int m = 0; m < MH; ++m) n = fmaf(r[i][m].x, r[i][m].x, fmaf(r[i][m].y, r[i][m].y, n));
        if constexpr (QS > 1) n += __shfl_xor_sync(0xffffffffu, n, 1);
        hq[i] = -a.k2 * n;
        q_in_range = q_in_range && (a.k2 * n <= kFactorLimit);
#pragma unroll
        for (int m = 0; m < MH; ++m) r[i][m] = make_float2(g2 * r[i][m].x, g2 * r[i][m].y);
    }
    const bool cta_in_range = __syncthreads_and(q_in_range);
    // The query factor 2^(-k2 n_s) multiplies the sum at the end when the CTA is in range; the
    // direct form then pre-multiplies its terms by the inverse factor (at most 2^kFactorLimit).
    float qs[QPT];
#pragma unroll
    for (int i = 0; i < QPT; ++i) qs[i] = cta_in_range ? ex2(-hq[i]) : 1.f;

    float acc1[QPT][KH], acc2[QPT][KH];
#pragma unroll
    for (int i = 0; i < QPT; ++i)
#pragma unroll
        for (int k = 0; k < KH; ++k) acc1[i][k] = acc2[i][k] = 0.f;

    for (int tile = 0; tile < n_tiles; ++tile) {
        const bool ok = mbar_wait_bounded(&bar[tile & 1], (tile >> 1) & 1);
        const unsigned char *st = stage0 + (tile & 1) * S::kStageBytes;
        const float2 *sd = reinterpret_cast<const float2 *>(st);
        const float *sn = reinterpret_cast<const float *>(st + S::kDictBytes);
        const float *sg = reinterpret_cast<const float *>(st + S::kDictBytes + S::kNormBytes);
        const int e0 = e_begin + tile * kTileEntries;
        const int cnt = min(kTileEntries, e_end - e0);
        // fold the entry factor 2^(-k2 n_t) into the tile's coefficients
        if (tid == 0) *s_flag = 1;
        __syncthreads();
        if (ok) {
            for (int i = tid; i < cnt * 2 * K; i += nthreads) {
                const float ht = a.k2 * sn[i / (2 * K)];
                if (ht > kFactorLimit) *s_flag = 0;
                s_gs[i] = e0 + i / (2 * K) >= e_lo ? sg[i] * ex2(-ht) : 0.f;  // masked below the segment
            }
        }
        if (!__syncthreads_and(ok)) {
            if (tid == 0) report(a.status, APSM_ERR_TIMEOUT);
            if (a.pdl_late) pdl_wait();
            return;
        }
        if (cta_in_range && *s_flag) {
            // factored form: E = ex2(2 k2 z) against coefficients already scaled by 2^(-k2 n_t)
#pragma unroll kDetectUnroll
            for (int t = threadIdx.y; t < cnt; t += blockDim.y) {
                float zr[QPT], zi[QPT];
#pragma unroll
                for (int i = 0; i < QPT; ++i) zr[i] = zi[i] = 0.f;
                const float4 *d4 = reinterpret_cast<const float4 *>(sd + t * M + part * MH);
#pragma unroll
                for (int m = 0; m < MH / 2; ++m) {
                    const float4 d = d4[m];
#pragma unroll
                    for (int i = 0; i < QPT; ++i) {
                        const float2 x0 = r[i][2 * m], x1 = r[i][2 * m + 1];
                        zr[i] = fmaf(d.x, x0.x, zr[i]);
                        zi[i] = fmaf(d.x, x0.y, zi[i]);
                        zr[i] = fmaf(d.y, x0.y, zr[i]);
                        zi[i] = fmaf(-d.y, x0.x, zi[i]);
                        zr[i] = fmaf(d.z, x1.x, zr[i]);
                        zi[i] = fmaf(d.z, x1.y, zi[i]);
                        zr[i] = fmaf(d.w, x1.y, zr[i]);
                        zi[i] = fmaf(-d.w, x1.x, zi[i]);
                    }
                }
                if constexpr (QS > 1) {
#pragma unroll
                    for (int i = 0; i < QPT; ++i) {
                        zr[i] += __shfl_xor_sync(0xffffffffu, zr[i], 1);
                        zi[i] += __shfl_xor_sync(0xffffffffu, zi[i], 1);
                    }
                }
                float gm1[KH], gm2[KH];
                load_coef_part<K, KH>(s_gs + t * 2 * K, part, gm1, gm2);
#pragma unroll
                for (int i = 0; i < QPT; ++i) {
                    const float eA = ex2(zr[i]), eB = ex2(zi[i]), eC = ex2(-zi[i]);
                    // users in pairs with packed FMAs (same operations and order as the scalar tail)
#pragma unroll
                    for (int k = 0; k + 1 < KH; k += 2) {
                        fma2_pair(acc1[i][k], acc1[i][k + 1], gm2[k], gm2[k + 1], eC);
                        fma2_pair(acc1[i][k], acc1[i][k + 1], gm1[k], gm1[k + 1], eA);
                        fma2_pair(acc2[i][k], acc2[i][k + 1], gm2[k], gm2[k + 1], eA);
                        fma2_pair(acc2[i][k], acc2[i][k + 1], gm1[k], gm1[k + 1], eB);
                    }
                    if constexpr (KH % 2) {
                        acc1[i][KH - 1] = fmaf(gm1[KH - 1], eA, fmaf(gm2[KH - 1], eC, acc1[i][KH - 1]));
                        acc2[i][KH - 1] = fmaf(gm1[KH - 1], eB, fmaf(gm2[KH - 1], eA, acc2[i][KH - 1]));
                    }
                }
            }
        } else {
            // guarded form for norms outside the factor range: the three squared distances by
            // direct differences (no norm expansion, so no cancellation when ||r||^2 dominates):
            //   A = ||r_t - r_s||^2,  B = ||r_t + i r_s||^2 (= ||r1(t) - r2(s)||^2),
            //   C = ||r_t - i r_s||^2 (= ||r2(t) - r1(s)||^2)
            const float inv_g2 = 1.f / g2;
#pragma unroll 1
            for (int t = threadIdx.y; t < cnt; t += blockDim.y) {
                if (e0 + t < e_lo) continue;
                float dA[QPT], dB[QPT], dC[QPT];
#pragma unroll
                for (int i = 0; i < QPT; ++i) dA[i] = dB[i] = dC[i] = 0.f;
#pragma unroll
                for (int m = 0; m < MH; ++m) {
                    const float2 d = sd[t * M + part * MH + m];
#pragma unroll
                    for (int i = 0; i < QPT; ++i) {
                        const float sx = r[i][m].x * inv_g2, sy = r[i][m].y * inv_g2;
                        const float ax = d.x - sx, ay = d.y - sy;
                        const float bx = d.x - sy, by = d.y + sx;
                        const float cx = d.x + sy, cy = d.y - sx;
                        dA[i] = fmaf(ax, ax, fmaf(ay, ay, dA[i]));
                        dB[i] = fmaf(bx, bx, fmaf(by, by, dB[i]));
                        dC[i] = fmaf(cx, cx, fmaf(cy, cy, dC[i]));
                    }
                }
                if constexpr (QS > 1) {
#pragma unroll
                    for (int i = 0; i < QPT; ++i) {
                        dA[i] += __shfl_xor_sync(0xffffffffu, dA[i], 1);
                        dB[i] += __shfl_xor_sync(0xffffffffu, dB[i], 1);
                        dC[i] += __shfl_xor_sync(0xffffffffu, dC[i], 1);
                    }
                }
                float gm1[KH], gm2[KH];
                load_coef_part<K, KH>(sg + t * 2 * K, part, gm1, gm2);
#pragma unroll
                for (int i = 0; i < QPT; ++i) {
                    const float eA = ex2(-a.k2 * dA[i]), eB = ex2(-a.k2 * dB[i]), eC = ex2(-a.k2 * dC[i]);
#pragma unroll
                    for (int k = 0; k < KH; ++k) {
                        acc1[i][k] = fmaf(gm1[k] * qs[i], eA, fmaf(gm2[k] * qs[i], eC, acc1[i][k]));
                        acc2[i][k] = fmaf(gm1[k] * qs[i], eB, fmaf(gm2[k] * qs[i], eA, acc2[i][k]));
                    }
                }
            }
        }
        if (!__syncthreads_and(ok)) {
            if (tid == 0) report(a.status, APSM_ERR_TIMEOUT);
            if (a.pdl_late) pdl_wait();
            return;
        }
        if (tid == 0 && tile + 2 < n_tiles) issue(tile + 2);
    }

    // merge the entry groups' partial sums in group order (group 0 keeps and finishes them)
    if (blockDim.y > 1) {
        if (threadIdx.y > 0) {
            float *dst = s_red + ((size_t)(threadIdx.y - 1) * blockDim.x + threadIdx.x) * QPT * 2 * KH;
#pragma unroll
            for (int i = 0; i < QPT; ++i)
#pragma unroll
                for (int k = 0; k < KH; ++k) {
                    dst[(i * 2 + 0) * KH + k] = acc1[i][k];
                    dst[(i * 2 + 1) * KH + k] = acc2[i][k];
                }
        }
        __syncthreads();
        if (threadIdx.y > 0) return;
        for (int y = 1; y < (int)blockDim.y; ++y) {
            const float *src = s_red + ((size_t)(y - 1) * blockDim.x + threadIdx.x) * QPT * 2 * KH;
#pragma unroll
            for (int i = 0; i < QPT; ++i)
#pragma unroll
                for (int k = 0; k < KH; ++k) {
                    acc1[i][k] += src[(i * 2 + 0) * KH + k];
                    acc2[i][k] += src[(i * 2 + 1) * KH + k];
                }
        }
    }

    const float inv_g2 = 1.f / g2;
#pragma unroll
    for (int i = 0; i < QPT; ++i) {
        const int q = q_base + i * qlanes;
        const bool live = q < a.N;  // the same for both lanes of a shared query
        if (QS == 1 && !live) continue;  // (a shared query's lanes still meet at the shuffles)
        const float fq = cta_in_range ? ex2(hq[i]) : 1.f;  // query factor 2^(-k2 n_s)
        if (a.partial != nullptr) {
            if (!live) continue;
            float *dst = a.partial + ((size_t)blockIdx.y * a.N + q) * 2 * K;
#pragma unroll
            for (int j = 0; j < KH; ++j) {
                const int k = part * KH + j;
                if (QS == 1 || k < K) {
                    dst[k] = fq * acc1[i][j];
                    dst[K + k] = fq * acc2[i][j];
                }
            }
            continue;
        }
        unsigned char hbits[KH];
#pragma unroll
        for (int j = 0; j < KH; ++j) {
            // c_k^H r = sum_m conj(c[m][k]) r[m]  (r held as g2 r); with a shared query each lane
            // sums its own antennas for its own user and for the partner's user of the same j,
            // and the partner's sum for this lane's user arrives by shuffle (all lanes take part).
            const int k = min(part * KH + j, K - 1);
            float l1 = 0.f, l2 = 0.f;
#pragma unroll
            for (int m = 0; m < MH; ++m) {
                const float2 c = s_clin[(part * MH + m) * K + k];
                l1 = fmaf(c.x, r[i][m].x, fmaf(c.y, r[i][m].y, l1));
                l2 = fmaf(c.x, r[i][m].y, fmaf(-c.y, r[i][m].x, l2));
            }
            if constexpr (QS > 1) {
                const int ko = min((1 - part) * KH + j, K - 1);
                float o1 = 0.f, o2 = 0.f;
#pragma unroll
                for (int m = 0; m < MH; ++m) {
                    const float2 c = s_clin[(part * MH + m) * K + ko];
                    o1 = fmaf(c.x, r[i][m].x, fmaf(c.y, r[i][m].y, o1));
                    o2 = fmaf(c.x, r[i][m].y, fmaf(-c.y, r[i][m].x, o2));
                }
                l1 += __shfl_xor_sync(0xffffffffu, o1, 1);
                l2 += __shfl_xor_sync(0xffffffffu, o2, 1);
            }
            const float y1 = fmaf(a.wL * inv_g2, l1, a.wG * fq * acc1[i][j]);
            const float y2 = fmaf(a.wL * inv_g2, l2, a.wG * fq * acc2[i][j]);
            if (live && (QS == 1 || part * KH + j < K)) a.soft[(size_t)q * K + k] = make_float2(y1, y2);
            hbits[j] = (unsigned char)((y1 < 0.f ? 1 : 0) | (y2 < 0.f ? 2 : 0));  // QPSK (QAM: separate pass)
        }
        if (a.hard && live) {
#pragma unroll
            for (int j = 0; j < KH; ++j)
                if (QS == 1 || part * KH + j < K) a.hard[(size_t)q * K + part * KH + j] = hbits[j];
        }
    }
    if (a.pdl_late) pdl_wait();
}

// Host-side launcher for one (M, K) instantiation.
// Launch shape: `threads` query lanes x `split` entry groups per CTA, `qpt` queries per lane.
struct DetectShape {
    int threads, split, qpt;
};

template <int M, int K>
cudaError_t launch_detect_f32(const DetectArgs &a, int grid_y, DetectShape sh, cudaStream_t stream) {
    using S = DetectSmem<M, K>;
    if constexpr (M > 16) sh.qpt = 1;
    const int per_cta = sh.threads / query_lanes<M>() * sh.qpt;
    const int gx = (a.N + per_cta - 1) / per_cta;
    if (gx == 0 || grid_y == 0) return cudaSuccess;
    const dim3 grid(gx, grid_y), block(sh.threads, sh.split);
    const int smem = S::bytes(sh.threads, sh.split, sh.qpt);
    if constexpr (M <= 16) {
        if (sh.qpt == 2) {
            auto fn = detect_f32_kernel<M, K, 2>;
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            e = launch_pdl(fn, grid, block, smem, stream, a);
            return e != cudaSuccess ? e : cudaGetLastError();
        }
    }
    {
        auto fn = detect_f32_kernel<M, K, 1>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        e = launch_pdl(fn, grid, block, smem, stream, a);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

using DetectLauncher = cudaError_t (*)(const DetectArgs &, int, DetectShape, cudaStream_t);

}  // namespace apsm
