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
// or 32).  Roles (256 threads): warps 0-3 epilogue (query row = thread; thread 0 issues the
// coefficient MMAs of each sub-chunk once the four warps have stored its E), warps 4-7
// converters (entry rows of the Gram operand, the tile's G operand; thread 128 issues the Gram
// MMAs).  Barriers:
//   mma_done[st]  converters' stage st written + Gram MMA of the tile committed
//   epi_done[st]  epilogue done with the Gram buffer and with the G operand of stage st
//   e_free[b]     the coefficient MMAs that read E buffer b have completed
// All waits are bounded.
#pragma once

#include "detect_tc.cuh"

namespace apsm {

constexpr int kTF32x3Coef = 2;  // precision id of this path (beside kTF32x3 and kHalf)
constexpr int kT2Entries = 32;  // entries per Gram tile (MMA N = 64)
constexpr int kT2Sub = 8;       // entries per coefficient sub-chunk
constexpr int kT2KG = 3 * kT2Sub;  // contraction length of a sub-chunk's coefficient MMAs (24)
constexpr int kT2Subs = kT2Entries / kT2Sub;  // sub-chunks per tile

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
    static constexpr int kG = kB + 2 * 2 * kBytesB;                 // 2 stages x sub-chunks x 2 copies
    static constexpr int kN = kG + 2 * kT2Subs * 2 * kBytesG;       // 2 stages x [32] -k2 n_t
    static constexpr int kGam = round_up(kN + 2 * kT2Entries * 4, 16);  // the tile's raw coefficients
    static constexpr int kBar = round_up(kGam + kT2Entries * 2 * KB * 4, 16);
    static constexpr int kTmem = kBar + 64;
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

template <int M, int KB>
__global__ void __launch_bounds__(kTcThreads, 2) detect_tc2_kernel(const TcArgs a) {
    using Sh = TcShape<M, kTF32x3>;
    using L = Tc2Smem<M, KB>;
    constexpr int NB = L::NB, NY = L::NY, E = kT2Entries;
    extern __shared__ __align__(1024) unsigned char smem[];
    pdl_enter();
    unsigned char *sA = smem + L::kA;
    unsigned char *sB = smem + L::kB;
    unsigned char *sG = smem + L::kG;
    float *sH = reinterpret_cast<float *>(smem + L::kN);
    float *sGam = reinterpret_cast<float *>(smem + L::kGam);  // [32][2][K] of the tile being converted
    uint64_t *mma_done = reinterpret_cast<uint64_t *>(smem + L::kBar);  // [2]: commit + 128 converters
    uint64_t *epi_done = mma_done + 2;                                   // [2]: 128 epilogue threads
    uint64_t *e_free = mma_done + 4;                                     // [2]: commit
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
        mbar_init(&mma_done[0], 1 + 128);
        mbar_init(&mma_done[1], 1 + 128);
        mbar_init(&epi_done[0], kTcRows);
        mbar_init(&epi_done[1], kTcRows);
        mbar_init(&e_free[0], 1);
        mbar_init(&e_free[1], 1);
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
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    const bool cta_in_range = __syncthreads_and(warp >= 4 || a.k2 * nq <= kFactorLimit);
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    const uint32_t ifmt = (1u << 4) | (2u << 7) | (2u << 10);  // F32 accumulate, TF32 A and B, K-major
    const uint32_t idesc_g = ifmt | ((uint32_t)(NB >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
    const uint32_t idesc_y = ifmt | ((uint32_t)(NY >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
    auto g_base = [&](int st, int h) { return sG + ((st * kT2Subs + h) * 2) * L::kBytesG; };  // hi; lo follows

    bool ok = true;
    if (warp >= 4) {
        // ================= converters + MMA issue =================
        const int ct = tid - 128;
        for (int tile = 0; tile < n_tiles; ++tile) {
            const int st = tile & 1;
            // the epilogue has released stage st (Gram buffer read, y MMAs of tile-2 done)
            bool w = true;
            if (tile >= 2) w = mbar_wait_bounded(&epi_done[st], ((tile - 2) >> 1) & 1);
            if (!converters_and(w)) {
                ok = false;
                break;
            }
            const int e0 = tile * E;
            unsigned char *bst = sB + st * 2 * L::kBytesB;
            // the tile's coefficients [32][2][K] are contiguous: coalesced loads, all in flight
            const int n_gam = min(E, max(n_ent - e0, 0)) * 2 * a.K;
            for (int i = ct; i < E * 2 * a.K; i += 128)
                sGam[i] = i < n_gam ? __ldg(a.gamma + (size_t)e0 * 2 * a.K + i) : 0.f;
            if (ct < NB) {
                const int t = e0 + (ct >> 1), h = ct & 1;
                // the entry's vector with 128-bit loads issued together, then converted
                float2 r[M];
                const float4 *rt = reinterpret_cast<const float4 *>(a.dict + (size_t)t * M);
#pragma unroll
                for (int m = 0; m < M / 2; ++m) {
                    const float4 v = t < n_ent ? __ldg(rt + m) : make_float4(0.f, 0.f, 0.f, 0.f);
                    r[2 * m] = make_float2(v.x, v.y);
                    r[2 * m + 1] = make_float2(v.z, v.w);
                }
                // row 2e: [Re r_t; Im r_t] gives Re z;  row 2e+1: [-Im r_t; Re r_t] gives Im z
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    put_elem<kTF32x3>(bst, L::kBytesB, Sh::off(ct, m), h ? -r[m].y : r[m].x, 0);
                    put_elem<kTF32x3>(bst, L::kBytesB, Sh::off(ct, M + m), h ? r[m].x : r[m].y, 0);
                }
                for (int k = 2 * M; k < Sh::KD; ++k) put_elem<kTF32x3>(bst, L::kBytesB, Sh::off(ct, k), 0.f, 0);
            }
            named_sync(1, 128);  // sGam complete
            // G operand of the tile's sub-chunks: rows = y columns, k = v * kT2Sub + e
            for (int idx = ct; idx < kT2Subs * NY * kT2KG; idx += 128) {
                const int h = idx / (NY * kT2KG), r = (idx / kT2KG) % NY, k = idx % kT2KG;
                const int v = k / kT2Sub, e = h * kT2Sub + k % kT2Sub;
                int l = -1, kk = r;  // coefficient g_l of user kk at this (row, k), or none
                if (r < KB) l = v == 0 ? 0 : (v == 2 ? 1 : -1);
                else if (r < 2 * KB) { kk = r - KB; l = v == 1 ? 0 : (v == 0 ? 1 : -1); }
                const float x = (l >= 0 && kk < a.K) ? sGam[(e * 2 + l) * a.K + kk] : 0.f;
                put_elem<kTF32x3>(g_base(st, h), L::kBytesG, L::offG(r, k), x, 0);
            }
            if (ct < E) {
                const int t = e0 + ct;
                sH[st * E + ct] = t < n_ent ? -a.k2 * __ldg(a.dict_norm + t) : 0.f;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            named_sync(1, 128);
            mbar_arrive(&mma_done[st]);  // releases this thread's sH writes
            if (ct == 0) {
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(st * NB);
                const uint32_t a0 = smem_u32(sA), b0 = smem_u32(bst);
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
            }
        }
    } else {
        // ================= epilogue: exponentials to tensor memory =================
        const float hq = cta_in_range ? 0.f : -a.k2 * nq;  // unfactored exponent when out of range
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        int sub = 0;
        for (int tile = 0; tile < n_tiles && ok; ++tile) {
            const int st = tile & 1;
            // warp-uniform decisions: tcgen05.ld / st below are executed by whole warps only
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&mma_done[st], (tile >> 1) & 1))) {
                ok = false;
                break;
            }
            tc_fence_after();
            const float *hh = sH + st * E;
            for (int h = 0; h < kT2Subs; ++h, ++sub) {
                const int b = sub & 1;
                float v[16], ex[kT2KG];
                tmem_ld16(tmem + lane_base + (uint32_t)(st * NB + 16 * h), v);
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
                if (h == 1 && tile >= 1) {  // tile-1: Gram read, its last sub-chunk's MMAs done -> stage free
                    tc_fence_before();
                    mbar_arrive(&epi_done[(tile - 1) & 1]);
                }
                const uint32_t ce = kColE + 2 * kT2KG * b;
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    uint32_t hi[8], lo[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float x = ex[p * 8 + j];
                        hi[j] = tf32_rna(x);
                        lo[j] = tf32_rna(x - __uint_as_float(hi[j]));
                    }
                    tmem_st8(tmem + lane_base + ce + 8 * p, hi);
                    tmem_st8(tmem + lane_base + ce + kT2KG + 8 * p, lo);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                named_sync(2, kTcRows);  // the four epilogue warps have stored this sub-chunk's E
                if (tid == 0) {
                    tc_fence_after();
                    const uint32_t gb = smem_u32(g_base(st, h));
#pragma unroll
                    for (int s = 0; s < kT2KG / 8; ++s) {
                        const uint64_t bh = umma_sdesc(gb + s * 256, L::kSboG);
                        const uint64_t bl = umma_sdesc(gb + L::kBytesG + s * 256, L::kSboG);
                        umma_tf32_ta(tmem + kColY, tmem + ce + kT2KG + 8 * s, bh, idesc_y, (sub > 0 || s > 0) ? 1u : 0u);
                        umma_tf32_ta(tmem + kColY, tmem + ce + 8 * s, bl, idesc_y, 1);
                        umma_tf32_ta(tmem + kColY, tmem + ce + 8 * s, bh, idesc_y, 1);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&e_free[b]))
                                 : "memory");
                }
                __syncwarp();
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
    if (!ok && (tid == 0 || tid == 128)) report(a.status, APSM_ERR_TIMEOUT);

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
    e = launch_pdl(fn, dim3(grid), dim3(kTcThreads), L::kBytes, stream, a);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace apsm
