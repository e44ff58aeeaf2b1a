// detect_tcc.cuh -- reduced-precision detection with both contractions on the tensor cores
// (Sec. III-B detection; the BF16/FP16 form of detect_tc.cuh).
//
// The dist-Gram is the BF16 or FP16 GEMM of detect_tc.cuh (query operand 2 k2 [Re r_s; Im r_s],
// two rows per entry, accumulators in TMEM).  The coefficient sums
//   acc1_k = sum_t g1_tk E_A + g2_tk E_C,   acc2_k = sum_t g1_tk E_B + g2_tk E_A
// (E_A, E_B, E_C the three exponentials of a pair, g1, g2 the entry's two real-split
// coefficients) are a second GEMM Y[s][n] = sum_j X[s][j] G[n][j] over j = (exponential kind c,
// entry t): X = the exponentials in BF16, written by the epilogue threads into shared memory a
// chunk of 16 entries at a time, and G the coefficients arranged per output column (n = k:
// g1 against E_A, g2 against E_C; n = KB + k: g2 against E_A, g1 against E_B) as a BF16 hi + lo
// pair, so that their rounding does not count.  Y (128 rows x NY columns, FP32) accumulates in
// TMEM over the whole dictionary; the FP32 pipe then only forms the exponent arguments.
// Pairs flagged by the cancellation guard (theta = 2^-4, see detect_tc.cuh) enter X as zero
// and are recomputed by direct differences into FP32 register sums.
//
// Both operands that depend on the dictionary alone -- the Gram's entry operand and G -- are
// packed once per call by tcc_pack_kernel into the caller's workspace, one contiguous block per
// 64-entry tile [Gram entry operand | G hi | G lo | -k2 n_t] in exactly the shared-memory layout
// the MMAs read; the detection CTAs then fetch each tile with one bulk copy.
//
// Roles (192 threads): warps 0-3 epilogue (query row = thread), warp 4 lane 0 issues the tile
// copies and the Gram MMAs, warp 5 lane 0 the coefficient MMAs (each as soon as all four
// epilogue warps have written an exponential chunk).  Two tile stages, two Gram accumulators,
// two exponential buffers.  All waits are bounded.
#pragma once

#include "detect_tc.cuh"

namespace apsm {

constexpr int kTccChunk = 16;     // entries per exponential chunk
constexpr int kTccXBuf = 2;       // exponential buffers
constexpr int kTccThreads = 192;

// Shared-memory matrix descriptor, K-major, no swizzle, with an explicit leading byte offset
// (bytes between k-adjacent core matrices) and stride byte offset (between 8-row groups).
__device__ __forceinline__ uint64_t umma_sdesc_lbo(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

template <int M, int KB>
struct TccSmem {
    using Sh = TcShape<M, kHalf>;
    static constexpr int E = kTcEntries;
    static constexpr int NY = round_up(2 * KB, 16);               // coefficient GEMM N
    static constexpr int KX = 3 * kTccChunk;                      // its K per chunk (48)
    static constexpr int kXBytes = kTcRows * KX * 2;              // one exponential buffer
    static constexpr int kGBytes = NY * 3 * E * 2;                // one copy of G for a tile
    // a packed tile (the same layout in the workspace and in a shared-memory stage)
    static constexpr int kOG = Sh::kBytesB;                       // G hi, then G lo
    static constexpr int kOH = kOG + 2 * kGBytes;                 // -k2 n_t [E]
    static constexpr int kTile = round_up(kOH + E * 4, 1024);
    static constexpr int kA = 0;
    static constexpr int kS = round_up(Sh::kBytesA, 1024);        // 2 tile stages
    static constexpr int kX = kS + 2 * kTile;                     // exponential buffers
    static constexpr int kBar = kX + kTccXBuf * kXBytes;          // mbarriers
    static constexpr int kTmem = kBar + 16 * 8;
    static constexpr int kBytes = kTmem + 16;
    static_assert(kBytes <= 227 * 1024, "one CTA per SM");
    static_assert(Sh::kBytesB % 16 == 0 && kGBytes % 16 == 0, "bulk-copy granules");
};

// Workspace of the packed form: one kTile block per 64-entry tile of the dictionary capacity.
template <int M, int KB>
constexpr size_t tcc_workspace_bytes(int D) {
    return (size_t)((D + kTcEntries - 1) / kTcEntries) * TccSmem<M, KB>::kTile;
}

// One block per tile: the Gram entry operand (rows 2e: [Re r_t; Im r_t], 2e+1: [-Im r_t; Re r_t],
// in BF16 or FP16), G in BF16 hi + lo, and -k2 n_t; zeros past the held entries.
template <int M, int KB>
__global__ void __launch_bounds__(128) tcc_pack_kernel(const TcArgs a, unsigned char *packed) {
    using Sh = TcShape<M, kHalf>;
    using L = TccSmem<M, KB>;
    constexpr int E = kTcEntries, NY = L::NY, CE = kTccChunk;
    __shared__ float s_coef[E * 2 * KB];
    const int tile = blockIdx.x, ct = threadIdx.x, e0 = tile * E;
    int n_ent = a.n_entries;
    if (a.meta) n_ent = min(n_ent, max(__ldg(a.meta), 0));
    unsigned char *blk = packed + (size_t)tile * L::kTile;
    if constexpr (tc_core_rows<M, kHalf>()) {
        using Rows = EntryRows<M, kHalf>;
        for (int i = 0; i < Rows::P; ++i) {
            int e, h, p;
            Rows::task(ct, i, e, h, p);
            float4 v[Rows::V];
            Rows::load(a.dict, e0 + e, n_ent, p, v);
            Rows::put(blk, e, h, p, v, a.half_fmt);
        }
    } else {
        const int t = e0 + (ct >> 1), h = ct & 1;
        const float2 *rt = a.dict + (size_t)t * M;
        for (int m = 0; m < M; ++m) {
            const float2 v = t < n_ent ? __ldg(rt + m) : make_float2(0.f, 0.f);
            put_elem<kHalf>(blk, Sh::kBytesB, Sh::off(ct, m), h ? -v.y : v.x, a.half_fmt);
            put_elem<kHalf>(blk, Sh::kBytesB, Sh::off(ct, M + m), h ? v.x : v.y, a.half_fmt);
        }
        for (int k = 2 * M; k < Sh::KD; ++k) put_elem<kHalf>(blk, Sh::kBytesB, Sh::off(ct, k), 0.f, a.half_fmt);
    }
    for (int i = ct; i < E * 2 * KB; i += 128) {
        const int e = i / (2 * KB), j = i % (2 * KB), l = j / KB, k = j % KB, t = e0 + e;
        s_coef[i] = (t < n_ent && k < a.K) ? __ldg(a.gamma + ((size_t)t * 2 + l) * a.K + k) : 0.f;
    }
    if (ct < E) {
        const int t = e0 + ct;
        reinterpret_cast<float *>(blk + L::kOH)[ct] = t < n_ent ? -a.k2 * __ldg(a.dict_norm + t) : 0.f;
    }
    __syncthreads();
    // G: row n, k = (chunk c, kind, entry within chunk); one task = one 16-byte core row (8
    // entries of one kind) of one output column
    constexpr int kTasks = NY * 3 * E / 8;
    for (int task = ct; task < kTasks; task += 128) {
        const int n = task % NY, kc = task / NY;  // k-chunk: 6 per chunk
        const int c = kc / 6, kind = (kc % 6) / 2, half8 = kc % 2;
        const int t0 = c * CE + half8 * 8;
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float *gr = s_coef + (t0 + i) * 2 * KB;  // [g1 (KB) | g2 (KB)]
            float x = 0.f;
            if (n < KB) {  // acc1: g1 E_A + g2 E_C
                x = kind == 0 ? gr[n] : (kind == 2 ? gr[KB + n] : 0.f);
            } else if (n < 2 * KB) {  // acc2: g2 E_A + g1 E_B
                const int k = n - KB;
                x = kind == 0 ? gr[KB + k] : (kind == 1 ? gr[k] : 0.f);
            }
            v[i] = x;
        }
        uint4 hi, lo;
        uint32_t *hp = &hi.x, *lp = &lo.x;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
            const float2 hf = __bfloat1622float2(h2);
            const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
            hp[i] = *reinterpret_cast<const uint32_t *>(&h2);
            lp[i] = *reinterpret_cast<const uint32_t *>(&l2);
        }
        const int off = L::kOG + (kc * NY + n) * 16;
        *reinterpret_cast<uint4 *>(blk + off) = hi;
        *reinterpret_cast<uint4 *>(blk + L::kGBytes + off) = lo;
    }
}

template <int M, int KB>
__global__ void __launch_bounds__(kTccThreads, 1) detect_tcc_kernel(const TcArgs a, const unsigned char *packed) {
    using Sh = TcShape<M, kHalf>;
    using L = TccSmem<M, KB>;
    constexpr int E = kTcEntries, NB = 2 * kTcEntries, CE = kTccChunk, NY = L::NY;
    constexpr int kChunks = E / CE;
    static_assert(KB % 2 == 0 && 2 * KB <= NY, "users in pairs");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem + L::kA;
    unsigned char *sS = smem + L::kS;
    unsigned char *sX = smem + L::kX;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::kBar);
    uint64_t *s_full = bars, *mma_done = bars + 2, *epi_done = bars + 4, *g_free = bars + 6, *x_full = bars + 8,
             *x_free = bars + 8 + kTccXBuf;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + L::kTmem);
    constexpr uint32_t kCols = 512;  // Gram accumulators at [0, 2 NB), Y at [2 NB, 2 NB + NY)

    const int tid = threadIdx.x, warp = tid >> 5;
    const int q0 = blockIdx.x * kTcRows;
    int n_ent = a.n_entries;
    if (a.meta) n_ent = min(n_ent, max(__ldg(a.meta), 0));
    const int n_tiles = (n_ent + E - 1) / E;
    const int n_chunks = n_tiles * kChunks;
    const float g2 = 2.f * a.k2;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&s_full[i], 1);
            mbar_init(&mma_done[i], 1);
            mbar_init(&epi_done[i], kTcRows);
            mbar_init(&g_free[i], 1);
        }
        for (int i = 0; i < kTccXBuf; ++i) {
            mbar_init(&x_full[i], kTcRows);
            mbar_init(&x_free[i], 1);
        }
        fence_mbar_init();
    }
    // the first two tiles' copies go out before the query operand is built
    __syncthreads();
    if (tid == 128) {
        for (int t = 0; t < 2 && t < n_tiles; ++t) {
            mbar_arrive_expect_tx(&s_full[t], (uint32_t)L::kTile);
            bulk_g2s(sS + t * L::kTile, packed + (size_t)t * L::kTile, (uint32_t)L::kTile, &s_full[t]);
        }
    }
    // ---- the query operand (as detect_tc.cuh) -------------------------------------------------
    float nq = 0.f;
    if (warp < 4) {
        const int s = q0 + tid;
        const float2 *rq = a.rx + (size_t)s * M;
        if constexpr (tc_core_rows<M, kHalf>()) {
            constexpr int C = Sh::kCoreK;
#pragma unroll 2
            for (int p = 0; p < M / C; ++p) {
                float re[C], im[C];
                if (s < a.N) {
                    const float4 *src = reinterpret_cast<const float4 *>(rq + p * C);
#pragma unroll
                    for (int q = 0; q < C / 2; ++q) {
                        const float4 v = __ldg(src + q);
                        re[2 * q] = v.x; im[2 * q] = v.y; re[2 * q + 1] = v.z; im[2 * q + 1] = v.w;
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < C; ++c) re[c] = im[c] = 0.f;
                }
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    nq = fmaf(re[c], re[c], fmaf(im[c], im[c], nq));
                    re[c] *= g2;
                    im[c] *= g2;
                }
                put_core<kHalf, C>(sA, Sh::kBytesA, Sh::off(tid, p * C), re, a.half_fmt);
                put_core<kHalf, C>(sA, Sh::kBytesA, Sh::off(tid, M + p * C), im, a.half_fmt);
            }
        } else {
            for (int m = 0; m < M; ++m) {
                const float2 v = s < a.N ? __ldg(rq + m) : make_float2(0.f, 0.f);
                nq = fmaf(v.x, v.x, fmaf(v.y, v.y, nq));
                put_elem<kHalf>(sA, Sh::kBytesA, Sh::off(tid, m), g2 * v.x, a.half_fmt);
                put_elem<kHalf>(sA, Sh::kBytesA, Sh::off(tid, M + m), g2 * v.y, a.half_fmt);
            }
            for (int k = 2 * M; k < Sh::KD; ++k) put_elem<kHalf>(sA, Sh::kBytesA, Sh::off(tid, k), 0.f, a.half_fmt);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    const bool cta_in_range = __syncthreads_and(warp >= 4 || a.k2 * nq <= kFactorLimit);
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    bool ok = true;

    if (warp == 4) {
        // ================= tile copies and Gram MMAs (one thread) =================
        if (tid == 128) {
            const uint32_t idesc = (1u << 4) | ((a.half_fmt ? 1u : 0u) << 7) | ((a.half_fmt ? 1u : 0u) << 10) |
                                   ((uint32_t)(NB >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
            const uint32_t a0 = smem_u32(sA);
            int issued = min(2, n_tiles), committed = -1;
            for (int t = 0; t < n_tiles; ++t) {
                const int st = t & 1;
                // tile t has landed; the epilogue of tile t-2 freed TMEM stage st
                if (!mbar_wait_bounded(&s_full[st], (t >> 1) & 1) ||
                    (t >= 2 && !mbar_wait_sleepy(&epi_done[st], ((t - 2) >> 1) & 1))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(st * NB), b0 = smem_u32(sS + st * L::kTile);
#pragma unroll
                for (int s = 0; s < Sh::kSteps; ++s) {
                    const uint64_t ah = umma_sdesc(a0 + s * 256, Sh::SBO), bh = umma_sdesc(b0 + s * 256, Sh::SBO);
                    umma_f16(d, ah, bh, idesc, s > 0);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&mma_done[st]))
                             : "memory");
                committed = t;
                // the stage of tile t-1 is free once its epilogue and its coefficient GEMMs are done
                if (t >= 1 && t + 1 < n_tiles) {
                    const int so = (t - 1) & 1;
                    if (!mbar_wait_sleepy(&epi_done[so], ((t - 1) >> 1) & 1) ||
                        !mbar_wait_sleepy(&g_free[so], ((t - 1) >> 1) & 1)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&s_full[so], (uint32_t)L::kTile);
                    bulk_g2s(sS + so * L::kTile, packed + (size_t)(t + 1) * L::kTile, (uint32_t)L::kTile, &s_full[so]);
                    issued = t + 2;
                }
            }
            // every copy and MMA issued here has landed before the CTA may exit
            for (int t = max(0, issued - 2); t < issued; ++t) mbar_wait_sleepy(&s_full[t & 1], (t >> 1) & 1);
            if (committed >= 0) mbar_wait_sleepy(&mma_done[committed & 1], (committed >> 1) & 1);
        }
    } else if (warp == 5) {
        // ================= coefficient-GEMM issue (one thread) =================
        if (tid == 160) {
            const uint32_t coef_idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NY >> 3) << 17) |
                                        ((uint32_t)(kTcRows >> 4) << 24);
            const uint32_t y = tmem + 2 * NB;
            for (int g = 0; g < n_chunks; ++g) {
                const int xb = g % kTccXBuf, t = g / kChunks, c = g % kChunks, st = t & 1;
                if (!mbar_wait_bounded(&x_full[xb], (g / kTccXBuf) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // X chunk: [k-chunk of 8][128 rows][16 B]; G: [k-chunk of 8][NY rows][16 B], this
                // chunk's k-chunks are 6c .. 6c + 5
                const uint32_t x0 = smem_u32(sX + xb * L::kXBytes);
                const uint32_t gh = smem_u32(sS + st * L::kTile + L::kOG) + c * 6 * NY * 16;
                const uint32_t gl = gh + L::kGBytes;
#pragma unroll
                for (int ks = 0; ks < L::KX / 16; ++ks) {
                    const uint64_t xd = umma_sdesc_lbo(x0 + ks * 2 * kTcRows * 16, kTcRows * 16, 128);
                    const uint64_t hd = umma_sdesc_lbo(gh + ks * 2 * NY * 16, NY * 16, 128);
                    const uint64_t ld = umma_sdesc_lbo(gl + ks * 2 * NY * 16, NY * 16, 128);
                    umma_f16(y, xd, hd, coef_idesc, (g > 0 || ks > 0) ? 1u : 0u);
                    umma_f16(y, xd, ld, coef_idesc, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&x_free[xb]))
                             : "memory");
                if (c == kChunks - 1)  // the tile's last reader of its G
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&g_free[st]))
                                 : "memory");
            }
        }
    } else if (warp < 4) {
        // ================= epilogue: exponentials into X, exact pairs in FP32 =================
        const float hq = cta_in_range ? 0.f : -a.k2 * nq;
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        const int s_row = q0 + tid;
        const float one_m_theta = 1.f - kGuardHalf;
        const float thr_q = one_m_theta * a.k2 * nq;
        const float base_q = a.k2 * nq + hq;
        float acc1[KB], acc2[KB];  // direct-difference pairs only
#pragma unroll
        for (int k = 0; k < KB; ++k) acc1[k] = acc2[k] = 0.f;
        auto exact_pair = [&](int t) {
            if (t >= n_ent || s_row >= a.N) return;
            const float2 *rq = a.rx + (size_t)s_row * M;
            const float2 *rt = a.dict + (size_t)t * M;
            float dA = 0.f, dB = 0.f, dC = 0.f;
#pragma unroll 4
            for (int m = 0; m < M; ++m) {
                const float2 q = __ldg(rq + m), d = __ldg(rt + m);
                const float ax = d.x - q.x, ay = d.y - q.y;
                const float bx = d.x - q.y, by = d.y + q.x;
                const float cx = d.x + q.y, cy = d.y - q.x;
                dA = fmaf(ax, ax, fmaf(ay, ay, dA));
                dB = fmaf(bx, bx, fmaf(by, by, dB));
                dC = fmaf(cx, cx, fmaf(cy, cy, dC));
            }
            const float eA = ex2(base_q - a.k2 * dA), eB = ex2(base_q - a.k2 * dB), eC = ex2(base_q - a.k2 * dC);
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                const float g1 = k < a.K ? __ldg(a.gamma + ((size_t)t * 2) * a.K + k) : 0.f;
                const float gg = k < a.K ? __ldg(a.gamma + ((size_t)t * 2 + 1) * a.K + k) : 0.f;
                acc1[k] = fmaf(g1, eA, fmaf(gg, eC, acc1[k]));
                acc2[k] = fmaf(g1, eB, fmaf(gg, eA, acc2[k]));
            }
        };
        for (int tile = 0; tile < n_tiles && ok; ++tile) {
            const int st = tile & 1;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&s_full[st], (tile >> 1) & 1) &&
                                             mbar_wait_bounded(&mma_done[st], (tile >> 1) & 1))) {
                ok = false;
                break;
            }
            tc_fence_after();
            const float *hh = reinterpret_cast<const float *>(sS + st * L::kTile + L::kOH);
#pragma unroll 1
            for (int c = 0; c < kChunks; ++c) {
                const int g = tile * kChunks + c, xb = g % kTccXBuf;
                // the coefficient GEMM of chunk g - kTccXBuf has read buffer xb
                if (g >= kTccXBuf &&
                    !__all_sync(0xffffffffu, mbar_wait_bounded(&x_free[xb], ((g - kTccXBuf) / kTccXBuf) & 1))) {
                    ok = false;
                    break;
                }
                float vr[32];  // (Re z, Im z) of the chunk's 16 entries
                tmem_ld16(tmem + lane_base + (uint32_t)(st * NB + 32 * c), *reinterpret_cast<float(*)[16]>(vr));
                tmem_ld16(tmem + lane_base + (uint32_t)(st * NB + 32 * c + 16), *reinterpret_cast<float(*)[16]>(vr + 16));
                float hv[CE];
#pragma unroll
                for (int q = 0; q < CE / 4; ++q)
                    *reinterpret_cast<float4 *>(hv + 4 * q) = *reinterpret_cast<const float4 *>(hh + CE * c + 4 * q);
                float xA[CE], xB[CE], xC[CE];
                uint32_t fbits = 0;
#pragma unroll
                for (int j = 0; j < CE; ++j) {
                    const float re = vr[2 * j], im = vr[2 * j + 1];
                    float h = hv[j] + hq;
                    // flagged: max(v_re, |v_im|) > (1 - theta) k2 (n_s + n_t)
                    const bool f = fmaxf(re, fabsf(im)) > fmaf(-one_m_theta, hv[j], thr_q);
                    h = f ? -INFINITY : h;
                    fbits |= f ? (1u << j) : 0u;
                    float a2 = re, b2 = im;
                    add2_bcast(a2, b2, h);
                    xA[j] = ex2(a2);
                    xB[j] = ex2(b2);
                    xC[j] = ex2(h - im);
                }
                // X row: k-chunk 2 kind + (j / 8) holds entries 8 (j / 8) .. of one kind
                unsigned char *xrow = sX + xb * L::kXBytes + tid * 16;
                const float *src[3] = {xA, xB, xC};
#pragma unroll
                for (int kind = 0; kind < 3; ++kind) {
#pragma unroll
                    for (int h8 = 0; h8 < 2; ++h8) {
                        uint4 v;
                        uint32_t *vp = &v.x;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const __nv_bfloat162 b2 =
                                __floats2bfloat162_rn(src[kind][8 * h8 + 2 * i], src[kind][8 * h8 + 2 * i + 1]);
                            vp[i] = *reinterpret_cast<const uint32_t *>(&b2);
                        }
                        *reinterpret_cast<uint4 *>(xrow + (2 * kind + h8) * kTcRows * 16) = v;
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&x_full[xb]);
                if (__any_sync(0xffffffffu, fbits != 0)) {
#pragma unroll 1
                    while (fbits) {
                        const int j = __ffs(fbits) - 1;
                        fbits &= fbits - 1;
                        exact_pair(tile * E + CE * c + j);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&epi_done[st]);
        }
        // ---- Y (complete once the last chunk's GEMM has committed) plus the exact pairs -----------
        if (ok && n_chunks > 0) {
            const int gl = n_chunks - 1;
            ok = __all_sync(0xffffffffu, mbar_wait_bounded(&x_free[gl % kTccXBuf], (gl / kTccXBuf) & 1));
            tc_fence_after();
        }
        float y[NY];
#pragma unroll
        for (int n = 0; n < NY; ++n) y[n] = 0.f;
        if (ok && n_chunks > 0) {
#pragma unroll
            for (int n0 = 0; n0 < NY; n0 += 16)
                tmem_ld16(tmem + lane_base + (uint32_t)(2 * NB + n0), *reinterpret_cast<float(*)[16]>(y + n0));
        }
        const int s = s_row;
        if (ok && s < a.N) {
            const float fq = cta_in_range ? ex2(-a.k2 * nq) : 1.f;
            const float2 *rq = a.rx + (size_t)s * M;
            for (int k = 0; k < a.K && k < KB; ++k) {
                float l1 = 0.f, l2 = 0.f;
                for (int m = 0; m < M; ++m) {
                    const float2 cl = __ldg(a.clin + m * a.K + k), r = __ldg(rq + m);
                    l1 = fmaf(cl.x, r.x, fmaf(cl.y, r.y, l1));
                    l2 = fmaf(cl.x, r.y, fmaf(-cl.y, r.x, l2));
                }
                float y1 = 0.f, y2 = 0.f;
#pragma unroll
                for (int kk = 0; kk < KB; ++kk)
                    if (kk == k) {
                        y1 = y[kk] + acc1[kk];
                        y2 = y[KB + kk] + acc2[kk];
                    }
                y1 = fmaf(a.wL, l1, a.wG * fq * y1);
                y2 = fmaf(a.wL, l2, a.wG * fq * y2);
                a.soft[(size_t)s * a.K + k] = make_float2(y1, y2);
                if (a.hard) a.hard[(size_t)s * a.K + k] = (uint8_t)((y1 < 0.f ? 1 : 0) | (y2 < 0.f ? 2 : 0));
            }
        }
    }
    if (!ok && (tid == 0 || tid == 128 || tid == 160)) report(a.status, APSM_ERR_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

// Packs the dictionary's operands into `workspace` (tcc_workspace_bytes(D) bytes, 16-byte
// aligned) and runs the detection; with a smaller or missing workspace the form of
// detect_tc.cuh (coefficient sums on the FP32 pipe) runs instead.
template <int M, int KB>
cudaError_t launch_detect_tcc(const TcArgs &a, void *workspace, size_t ws_bytes, cudaStream_t stream) {
    using L = TccSmem<M, KB>;
    const int grid = (a.N + kTcRows - 1) / kTcRows;
    if (grid == 0) return cudaSuccess;
    const int n_tiles = (a.n_entries + kTcEntries - 1) / kTcEntries;
    if (!workspace || ws_bytes < tcc_workspace_bytes<M, KB>(a.n_entries) ||
        (reinterpret_cast<uintptr_t>(workspace) & 15))
        return launch_detect_tc<M, KB, kHalf>(a, stream);
    unsigned char *packed = static_cast<unsigned char *>(workspace);
    tcc_pack_kernel<M, KB><<<n_tiles, 128, 0, stream>>>(a, packed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto fn = detect_tcc_kernel<M, KB>;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes);
    if (e != cudaSuccess) return e;
    fn<<<grid, kTccThreads, L::kBytes, stream>>>(a, packed);  // ordinary launches (see launch_detect_tc)
    return cudaGetLastError();
}

using TccLauncher = cudaError_t (*)(const TcArgs &, void *, size_t, cudaStream_t);

}  // namespace apsm
