// detect_tc2.cuh -- FP32 detection with both contractions on the tensor cores (Sec. III-B).
//
// detect_tc.cuh forms the complex dist-Gram on the tensor cores and accumulates the coefficient
// sums y = sum_t (g1_t E_A + g2_t E_C) + i (g1_t E_B + g2_t E_A) with FP32 FMAs (4K per pair).
// Those sums are themselves a contraction over the entries: for a sub-chunk of 8 entries let
//   E[s][v*8 + e]  (v = 0: E_A, 1: E_B, 2: E_C of entry e and query s), 24 columns,
//   G[v*8 + e][k]      = g1_e^k (v = 0), g2_e^k (v = 2)          -> column k       = y1^k
//   G[v*8 + e][KB + k] = g1_e^k (v = 1), g2_e^k (v = 0)          -> column KB + k  = y2^k
// so y += E G, one MMA group per sub-chunk with the E operand read from tensor memory.  The
// epilogue threads only form the three exponentials per pair and store them (TF32 hi / lo
// split) to tensor memory; FP32 accuracy as in the Gram: y += E_lo G_hi + E_hi G_lo + E_hi G_hi.
//
// Tile = 32 entries (Gram N = 64), four coefficient sub-chunks of 8 entries per tile.  Tensor
// memory (256 columns): Gram accumulators 2 x 64, two E buffers of 24 (hi) + 24 (lo), y NY (16
// or 32).  Roles (288 threads): warps 0-3 epilogue (query row = thread), warps 4-7 converters
// (entry rows of the Gram operand, the tile's G operand), warp 8 issues every MMA (one thread),
// so the epilogue never waits on an MMA it could overlap.  Barriers:
//   conv_ready[st]  converters' stage written             mma_done[st]  Gram MMA of the tile done
//   gram_free[st]   epilogue read Gram buffer st          g_free[gs]    G stage gs (and its norms)
//   e_ready[b]      epilogue stored E buffer b            e_free[b]     its coefficient MMAs done
// The entry operand has two stages (reused once the Gram MMA two tiles back is done), the G
// operand and norms three (reused once the coefficient MMAs three tiles back are done), so the
// converters run well ahead of the epilogue.
// All waits are bounded.
#pragma once

#include "detect_tc.cuh"

namespace apsm {

constexpr int kTF32x3Coef = 2;  // precision id of this path (beside kTF32x3 and kHalf)
constexpr int kT2Entries = 32;  // entries per Gram tile (MMA N = 64)
constexpr int kT2Sub = 8;       // entries per coefficient sub-chunk
constexpr int kT2KG = 3 * kT2Sub;  // contraction length of a sub-chunk's coefficient MMAs (24)
constexpr int kT2Subs = kT2Entries / kT2Sub;  // sub-chunks per tile
constexpr int kT2Threads = 288;                // 4 epilogue + 4 converter warps + the MMA warp
constexpr int kT2GStages = 3;                  // stages of the G operand and the entry norms

template <int M, int KB>
struct Tc2Smem {
    using Sh = TcShape<M, kTF32x3>;                     // query operand layout (hi / lo copies)
    static constexpr int NB = 2 * kT2Entries;           // Gram columns per tile
    static constexpr int NY = round_up(2 * KB, 16);     // y columns (MMA N)
    static constexpr int kBytesB = NB / 8 * Sh::SBO;    // entry operand, one copy
    static constexpr int kSboG = (kT2KG / 4) * 128;
    static constexpr int kBytesG = NY / 8 * kSboG;      // G operand of one sub-chunk, one copy
    static constexpr int kA = 0;
    static constexpr int kB = kA + 2 * Sh::kBytesA;                 // 2 stages x 2 copies
    static constexpr int kG = kB + 2 * 2 * kBytesB;                 // G stages x sub-chunks x 2 copies
    static constexpr int kN = kG + kT2GStages * kT2Subs * 2 * kBytesG;  // G stages x [32] -k2 n_t
    static constexpr int kBar = round_up(kN + kT2GStages * kT2Entries * 4, 16);
    static constexpr int kTmem = kBar + 112;  // 13 mbarriers
    static constexpr int kBytes = kTmem + 16;
    __device__ static constexpr int offG(int r, int k) {
        return (r / 8) * kSboG + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4;
    }
};

// MMA with the A operand in tensor memory (kind::tf32)
__device__ __forceinline__ void umma_tf32_ta(uint32_t d, uint32_t a_tmem, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a_tmem), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

// two CTAs per SM where the shared memory allows it (registers are then capped accordingly)
template <int M, int KB>
constexpr int tc2_min_blocks() { return Tc2Smem<M, KB>::kBytes <= 113 * 1024 ? 2 : 1; }

template <int M, int KB>
__global__ void __launch_bounds__(kT2Threads, tc2_min_blocks<M, KB>()) detect_tc2_kernel(const TcArgs a) {
    using Sh = TcShape<M, kTF32x3>;
    using L = Tc2Smem<M, KB>;
    constexpr int NB = L::NB, NY = L::NY, E = kT2Entries;
    extern __shared__ __align__(1024) unsigned char smem[];
    pdl_enter();
    unsigned char *sA = smem + L::kA;
    unsigned char *sB = smem + L::kB;
    unsigned char *sG = smem + L::kG;
    float *sH = reinterpret_cast<float *>(smem + L::kN);
    uint64_t *mma_done = reinterpret_cast<uint64_t *>(smem + L::kBar);  // [2]: Gram commit
    uint64_t *gram_free = mma_done + 2;                                  // [2]: 128 epilogue threads
    uint64_t *e_free = mma_done + 4;                                     // [2]: coefficient commit
    uint64_t *conv_ready = mma_done + 6;                                 // [2]: 128 converters
    uint64_t *e_ready = mma_done + 8;                                    // [2]: 128 epilogue threads
    uint64_t *g_free = mma_done + 10;                                    // [3]: 128 epilogue threads
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + L::kTmem);
    // E buffer b: hi at kColE + 2 b kT2KG, lo kT2KG columns after it
    constexpr uint32_t kCols = 256, kColE = 2 * NB, kColY = kColE + 4 * kT2KG;
    static_assert(kColY + NY <= kCols, "tensor memory budget");

    const int tid = threadIdx.x, warp = tid >> 5;
    const int q0 = blockIdx.x * kTcRows;
    int n_ent = a.n_entries;
    if (a.meta) n_ent = min(n_ent, max(__ldg(a.meta), 0));
    const int n_tiles = (n_ent + E - 1) / E;
    const float g2 = 2.f * a.k2;

    // ---- set-up: TMEM, barriers, the query operand --------------------------------------------
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&mma_done[i], 1);
            mbar_init(&gram_free[i], kTcRows);
            mbar_init(&e_free[i], 1);
            mbar_init(&conv_ready[i], 128);
            mbar_init(&e_ready[i], kTcRows);
        }
        for (int i = 0; i < kT2GStages; ++i) mbar_init(&g_free[i], kTcRows);
        fence_mbar_init();
    }
    float nq = 0.f;  // squared norm of this epilogue thread's query
    if (warp < 4) {
        const int s = q0 + tid;
        const float2 *rq = a.rx + (size_t)s * M;
        for (int m = 0; m < M; ++m) {
            const float2 v = s < a.N ? __ldg(rq + m) : make_float2(0.f, 0.f);
            nq = fmaf(v.x, v.x, fmaf(v.y, v.y, nq));
            put_elem<kTF32x3>(sA, Sh::kBytesA, Sh::off(tid, m), g2 * v.x, 0);
            put_elem<kTF32x3>(sA, Sh::kBytesA, Sh::off(tid, M + m), g2 * v.y, 0);
        }
        for (int k = 2 * M; k < Sh::KD; ++k) put_elem<kTF32x3>(sA, Sh::kBytesA, Sh::off(tid, k), 0.f, 0);
    }
    // G operands start at zero: only the structural positions of the coefficients are ever written
    for (int i = tid; i < kT2GStages * kT2Subs * 2 * L::kBytesG / 4; i += kT2Threads)
        reinterpret_cast<uint32_t *>(sG)[i] = 0u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    const bool cta_in_range = __syncthreads_and(warp >= 4 || a.k2 * nq <= kFactorLimit);
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    const uint32_t ifmt = (1u << 4) | (2u << 7) | (2u << 10);  // F32 accumulate, TF32 A and B, K-major
    const uint32_t idesc_g = ifmt | ((uint32_t)(NB >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
    const uint32_t idesc_y = ifmt | ((uint32_t)(NY >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
    auto g_base = [&](int gs, int h) { return sG + ((gs * kT2Subs + h) * 2) * L::kBytesG; };  // hi; lo follows

    bool ok = true;
    if (warp == 8) {
        // ================= MMA issue (one thread) =================
        // Gram of tile t as soon as its operand is converted, then the coefficient MMAs of
        // tile t-1's sub-chunks as the epilogue stores their E.
        if ((tid & 31) == 0) {
            int ysub = 0;
            auto issue_y = [&](int tile) {
                const int gs = tile % kT2GStages;
                for (int h = 0; h < kT2Subs; ++h, ++ysub) {
                    const int b = ysub & 1;
                    if (!mbar_wait_bounded(&e_ready[b], (ysub >> 1) & 1)) return false;
                    tc_fence_after();
                    const uint32_t gb = smem_u32(g_base(gs, h));
                    const uint32_t ce = kColE + 2 * kT2KG * b;
#pragma unroll
                    for (int s = 0; s < kT2KG / 8; ++s) {
                        const uint64_t bh = umma_sdesc(gb + s * 256, L::kSboG);
                        const uint64_t bl = umma_sdesc(gb + L::kBytesG + s * 256, L::kSboG);
                        umma_tf32_ta(tmem + kColY, tmem + ce + kT2KG + 8 * s, bh, idesc_y, (ysub > 0 || s > 0) ? 1u : 0u);
                        umma_tf32_ta(tmem + kColY, tmem + ce + 8 * s, bl, idesc_y, 1);
                        umma_tf32_ta(tmem + kColY, tmem + ce + 8 * s, bh, idesc_y, 1);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&e_free[b]))
                                 : "memory");
                }
                return true;
            };
            for (int tile = 0; tile < n_tiles && ok; ++tile) {
                const int st = tile & 1;
                // the tile's operands are converted and the epilogue has read Gram buffer st (tile-2)
                if (!mbar_wait_bounded(&conv_ready[st], (tile >> 1) & 1) ||
                    (tile >= 2 && !mbar_wait_bounded(&gram_free[st], ((tile - 2) >> 1) & 1))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(st * NB);
                const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB + st * 2 * L::kBytesB);
#pragma unroll
                for (int s = 0; s < Sh::kSteps; ++s) {
                    const uint64_t ah = umma_sdesc(a0 + s * 256, Sh::SBO), bh = umma_sdesc(b0 + s * 256, Sh::SBO);
                    const uint64_t al = umma_sdesc(a0 + Sh::kBytesA + s * 256, Sh::SBO);
                    const uint64_t bl = umma_sdesc(b0 + L::kBytesB + s * 256, Sh::SBO);
                    umma_tf32(d, al, bh, idesc_g, s > 0);
                    umma_tf32(d, ah, bl, idesc_g, 1);
                    umma_tf32(d, ah, bh, idesc_g, 1);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&mma_done[st]))
                             : "memory");
                if (tile >= 1 && !issue_y(tile - 1)) ok = false;
            }
            if (ok && n_tiles > 0 && !issue_y(n_tiles - 1)) ok = false;
        }
    } else if (warp >= 4) {
        // ================= converters =================
        // Software-pipelined: the global loads of tile t+1 (entry vectors, coefficients, norms) go
        // into registers right after tile t is converted, so their latency overlaps the wait for
        // the stage.  Thread ct converts half (antennas [mh M/2, (mh+1) M/2)) of operand row ct/2.
        const int ct = tid - 128;
        const int row = ct >> 1, mh = ct & 1, hrow = row & 1;
        constexpr int MH = (M + 1) / 2;                         // antennas per half row
        constexpr int kGPer = (kT2Entries * 2 * KB + 127) / 128;  // coefficients per thread
        float2 rp[MH];
        float gp[kGPer], np = 0.f;
        auto prefetch = [&](int tile) {
            const int e0 = tile * E, te = e0 + (row >> 1);
            const float2 *rt = a.dict + (size_t)te * M + mh * MH;
#pragma unroll
            for (int m = 0; m < MH; ++m)
                rp[m] = (te < n_ent && mh * MH + m < M) ? __ldg(rt + m) : make_float2(0.f, 0.f);
            const int n_gam = min(E, max(n_ent - e0, 0)) * 2 * a.K;
#pragma unroll
            for (int j = 0; j < kGPer; ++j) {
                const int i = ct + 128 * j;
                gp[j] = i < n_gam ? __ldg(a.gamma + (size_t)e0 * 2 * a.K + i) : 0.f;
            }
            np = (ct < E && e0 + ct < n_ent) ? -a.k2 * __ldg(a.dict_norm + e0 + ct) : 0.f;
        };
        if (n_tiles > 0) prefetch(0);
        for (int tile = 0; tile < n_tiles; ++tile) {
            const int st = tile & 1;
            // entry stage st: the Gram MMA of tile-2 is done; G stage gs: the coefficient MMAs of
            // tile-3 are done (which the epilogue reports)
            const int gs = tile % kT2GStages;
            bool w = true;
            if (tile >= 2) w = mbar_wait_bounded(&mma_done[st], ((tile - 2) >> 1) & 1);
            if (tile >= kT2GStages) w = w && mbar_wait_bounded(&g_free[gs], ((tile - kT2GStages) / kT2GStages) & 1);
            if (!converters_and(w)) {
                ok = false;
                break;
            }
            unsigned char *bst = sB + st * 2 * L::kBytesB;
            // row 2e: [Re r_t; Im r_t] gives Re z;  row 2e+1: [-Im r_t; Re r_t] gives Im z
#pragma unroll
            for (int m0 = 0; m0 < MH; ++m0) {
                const int m = mh * MH + m0;
                if (m < M) {
                    put_elem<kTF32x3>(bst, L::kBytesB, Sh::off(row, m), hrow ? -rp[m0].y : rp[m0].x, 0);
                    put_elem<kTF32x3>(bst, L::kBytesB, Sh::off(row, M + m), hrow ? rp[m0].x : rp[m0].y, 0);
                }
            }
            if (mh == 0)
                for (int k = 2 * M; k < Sh::KD; ++k) put_elem<kTF32x3>(bst, L::kBytesB, Sh::off(row, k), 0.f, 0);
            // coefficient g_l^k of entry e (index (2e + l) K + k of the tile's block) goes to its two
            // positions of sub-chunk e / 8:  g1: (row k, E_A), (row KB + k, E_B);
            //                                g2: (row k, E_C), (row KB + k, E_A)
#pragma unroll
            for (int j = 0; j < kGPer; ++j) {
                const int i = ct + 128 * j;
                if (i < E * 2 * a.K) {
                    const int k = i % a.K, l = (i / a.K) & 1, e = i / (2 * a.K);
                    const int el = e % kT2Sub;
                    unsigned char *gb = g_base(gs, e / kT2Sub);
                    put_elem<kTF32x3>(gb, L::kBytesG, L::offG(k, (l ? 2 : 0) * kT2Sub + el), gp[j], 0);
                    put_elem<kTF32x3>(gb, L::kBytesG, L::offG(KB + k, (l ? 0 : 1) * kT2Sub + el), gp[j], 0);
                }
            }
            if (ct < E) sH[gs * E + ct] = np;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&conv_ready[st]);  // releases this thread's operand and sH writes
            if (tile + 1 < n_tiles) prefetch(tile + 1);
        }
    } else {
        // ================= epilogue: exponentials to tensor memory =================
        const float hq = cta_in_range ? 0.f : -a.k2 * nq;  // unfactored exponent when out of range
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        int sub = 0;
        for (int tile = 0; tile < n_tiles && ok; ++tile) {
            const int st = tile & 1;
            // warp-uniform decisions: tcgen05.ld / st below are executed by whole warps only
            // the Gram MMA of the tile, and the converters' sH writes (acquired from their barrier)
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&mma_done[st], (tile >> 1) & 1) &&
                                             mbar_wait_bounded(&conv_ready[st], (tile >> 1) & 1))) {
                ok = false;
                break;
            }
            tc_fence_after();
            const float *hh = sH + (tile % kT2GStages) * E;
            for (int h = 0; h < kT2Subs; ++h, ++sub) {
                const int b = sub & 1;
                float v[16], ex[kT2KG];
                tmem_ld16(tmem + lane_base + (uint32_t)(st * NB + 16 * h), v);
                if (h == kT2Subs - 1) {  // Gram buffer st read: the MMA warp may reuse it
                    tc_fence_before();
                    mbar_arrive(&gram_free[st]);
                }
#pragma unroll
                for (int e = 0; e < kT2Sub; ++e) {
                    const float hv = hh[h * kT2Sub + e] + hq;
                    ex[e] = ex2(v[2 * e] + hv);                    // E_A
                    ex[kT2Sub + e] = ex2(v[2 * e + 1] + hv);       // E_B
                    ex[2 * kT2Sub + e] = ex2(hv - v[2 * e + 1]);   // E_C
                }
                // the coefficient MMAs of sub-chunk sub-2 have read E buffer b
                if (sub >= 2 && !__all_sync(0xffffffffu, mbar_wait_bounded(&e_free[b], ((sub - 2) >> 1) & 1))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (h == 1 && tile >= 1)  // tile-1: its last sub-chunk's coefficient MMAs done -> G stage free
                    mbar_arrive(&g_free[(tile - 1) % kT2GStages]);
                const uint32_t ce = kColE + 2 * kT2KG * b;
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    uint32_t hi[8], lo[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float x = ex[p * 8 + j];
                        hi[j] = tf32_rna(x);
                        lo[j] = __float_as_uint(x - __uint_as_float(hi[j]));  // exact; read as TF32
                    }
                    tmem_st8(tmem + lane_base + ce + 8 * p, hi);
                    tmem_st8(tmem + lane_base + ce + kT2KG + 8 * p, lo);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                mbar_arrive(&e_ready[b]);  // the MMA warp issues this sub-chunk's coefficient MMAs
            }
        }
        // y: wait for the last sub-chunk's MMAs, read the accumulator row
        float y[NY];
#pragma unroll
        for (int c = 0; c < NY; ++c) y[c] = 0.f;
        if (ok && sub > 0) {
            // the last sub-chunk's MMAs (issued after every earlier one) complete last
            const int last = sub - 1;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&e_free[last & 1], (last >> 1) & 1))) {
                ok = false;
            } else {
                tc_fence_after();
#pragma unroll
                for (int c = 0; c < NY; c += 16) {
                    float t16[16];
                    tmem_ld16(tmem + lane_base + kColY + c, t16);
#pragma unroll
                    for (int j = 0; j < 16; ++j) y[c + j] = t16[j];
                }
            }
        }
        const int s = q0 + tid;
        if (ok && s < a.N) {
            const float fq = cta_in_range ? ex2(-a.k2 * nq) : 1.f;  // query factor
            const float2 *rq = a.rx + (size_t)s * M;
            for (int k = 0; k < a.K && k < KB; ++k) {
                float l1 = 0.f, l2 = 0.f;  // c_k^H r
                for (int m = 0; m < M; ++m) {
                    const float2 c = __ldg(a.clin + m * a.K + k), r = __ldg(rq + m);
                    l1 = fmaf(c.x, r.x, fmaf(c.y, r.y, l1));
                    l2 = fmaf(c.x, r.y, fmaf(-c.y, r.x, l2));
                }
                float y1 = 0.f, y2 = 0.f;
#pragma unroll
                for (int kk = 0; kk < KB; ++kk)
                    if (kk == k) { y1 = y[kk]; y2 = y[KB + kk]; }
                y1 = fmaf(a.wL, l1, a.wG * fq * y1);
                y2 = fmaf(a.wL, l2, a.wG * fq * y2);
                a.soft[(size_t)s * a.K + k] = make_float2(y1, y2);
                if (a.hard) a.hard[(size_t)s * a.K + k] = (uint8_t)((y1 < 0.f ? 1 : 0) | (y2 < 0.f ? 2 : 0));
            }
        }
    }
    if (!ok && (tid == 0 || tid == 128 || tid == 256)) report(a.status, APSM_ERR_TIMEOUT);

    // ---- teardown: every MMA has been waited for by the epilogue (or timed out) ----------------
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

template <int M, int KB>
cudaError_t launch_detect_tc2(const TcArgs &a, cudaStream_t stream) {
    using L = Tc2Smem<M, KB>;
    const int grid = (a.N + kTcRows - 1) / kTcRows;
    if (grid == 0) return cudaSuccess;
    auto fn = detect_tc2_kernel<M, KB>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes);
    if (e != cudaSuccess) return e;
    e = launch_pdl(fn, dim3(grid), dim3(kT2Threads), L::kBytes, stream, a);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace apsm
