// detect_tma.cuh -- FP32-accuracy detection on the tensor cores with every operand staged by
// the tensor memory accelerator (Sec. III-B detection; the same result as detect_tc.cuh).
//
// For a tile of 128 queries r_s and E = 64 dictionary entries r_t the complex Gram z = r_t^H r_s
// is two real GEMMs over the 2M interleaved components [Re r_1, Im r_1, Re r_2, ...]:
//   Re z = <[Re r_s, Im r_s]-pairs, raw entry row>      (A_re = the query row as stored)
//   Im z = <[Im r_s, -Re r_s]-pairs, raw entry row>     (A_im = each pair swapped, one negated)
// so the entry operand B is the dictionary row exactly as the state stores it, and the
// rotation of the real split (Sec. II-D) moves to the query operand.  Both products run in
// TF32 x3 (hi*hi + hi*lo + lo*hi, hi = tf32(x), lo = tf32(x - hi)) into two TMEM accumulators of
// 64 columns each.  The epilogue forms
//   E_A = 2^(2 k2 Re z - k2 n_t),  E_B = 2^(2 k2 Im z - k2 n_t),  E_C = 2^(-2 k2 Im z - k2 n_t)
// and the coefficient sums as detect_tc.cuh does (query factor 2^(-k2 n_s) applied at the end,
// the unfactored exponent and the direct-difference fallback for a query tile with a query
// outside the factor range).
//
// Work split: the units are (query tile of 128, entry tile of 64) pairs, query tile major.  A
// CTA takes a contiguous run of units, floor(c U / C) .. floor((c+1) U / C) for CTA c of C; it
// walks them as segments (the units of one query tile) through one continuous pipeline.  With
// C = the number of query tiles every segment is a whole tile (the plain form).  The balanced
// form launches C = (resident CTAs per SM) x SMs persistent CTAs, so every SM gets the same
// number of units whatever N is; a query tile split between CTAs leaves each part's sums in a
// workspace slot, and the CTA that completes the tile last (a per-tile arrival counter) adds
// the parts in CTA order, so the result does not depend on timing, and resets the counter.
//
// Staging: each query tile, each entry tile, its coefficients and its norms are tiled TMA loads
// of whole rows (one box each; rows past the tensor read as zero).  Query and entry rows land
// in the swizzled K-major operand layout whose swizzle width is the row (8M bytes: 128-, 64- or
// 32-byte swizzle for 16, 8 or 4 antennas), which the MMA reads directly.  Short shared-memory
// passes split each landed tile in place into its TF32 hi and lo copies (zeroing rows past the
// held entries), turn the entry norms into -k2 n_t and build the rotated query operand; every
// step is per element or per 16-byte chunk, so the swizzle (a permutation of a row's chunks)
// does not matter to them.
//
// Roles (288 threads): warps 0-7 = epilogue; warp w reads TMEM lanes 32 (w mod 4) .. and the
// entries 32 (w / 4) .. 32 (w / 4) + 31 of each tile, so two threads share every query row; at
// the end of a segment the second half passes its sums through TMEM to the first, which adds
// them in a fixed order.  The epilogue threads build a segment's query operand at its start
// (its rows were loaded as soon as the previous segment's MMAs were done) and convert entry
// tile j+1 at the start of tile j.  Warp 8, lane 0 = producer: issues the TMA loads and the
// MMAs.  Entry operand (hi, lo) two stages, coefficients and norms three, TMEM two accumulator
// pairs.  All waits are bounded.
//
// Used for FP32 detection with 4, 8 or 16 antennas and an even user count that is its own
// bucket (2, 4, 6, 8, 12, 16), where the state's arrays are 16-byte aligned.
#pragma once

#include <cuda.h>

#include <algorithm>

#include "detect_tc.cuh"

namespace apsm {

constexpr int kTmaRows = 128;        // queries per CTA (MMA M)
constexpr int kTmaEntries = 64;      // entries per tile (MMA N of each accumulator)
constexpr int kTmaEpi = 256;         // epilogue threads
constexpr int kTmaThreads = 288;     // + one producer warp
constexpr int kTmaChunk = 8;         // entries read from TMEM at a time (8 or 16)

struct TmaArgs {
    CUtensorMap tm_q;   // queries   [N][2M] float, box {2M, 128}, row swizzle
    CUtensorMap tm_d;   // entries   [D][2M] float, box {2M, 64}, row swizzle
    CUtensorMap tm_g;   // coefficients [D][2K] float, box {2K, 64}
    CUtensorMap tm_n;   // entry norms [D] float, box {64}
    const float2 *rx;   // [N][M] (exact fallback, linear part)
    int N;
    const float2 *dict;  // [D][M] (exact fallback)
    const float2 *clin;  // [M][K], K = KB
    const int *meta;
    int n_entries;       // host bound D
    float k2, wL, wG;
    float2 *soft;
    uint8_t *hard;
    int *status;
    int *counters;       // [query tiles] arrival counters (balanced form), else null
    float *parts;        // [2 C][128][2K] partial sums of split query tiles (balanced form)
};

template <int M, int KB>
struct TmaSmem {
    static constexpr int kRow = 8 * M;                    // bytes of one stored row (2M floats)
    static constexpr int kACopy = kTmaRows * kRow;        // one query operand copy
    static constexpr int kBCopy = kTmaEntries * kRow;     // one entry operand copy
    static constexpr int kCStage = kTmaEntries * 2 * KB * 4;
    static constexpr int kA = 0;                          // [re_hi, re_lo, im_hi, im_lo]
    static constexpr int kB = kA + 4 * kACopy;            // 2 stages x [hi, lo]
    static constexpr int kC = kB + 4 * kBCopy;            // 3 stages of coefficients [E][2K]
    static constexpr int kN = kC + 3 * kCStage;           // 3 stages of norms [E], then -k2 n_t
    static constexpr int kQ = kN + 3 * kTmaEntries * 4;   // query norms [128], a flag
    static constexpr int kBar = kQ + kTmaRows * 4 + 16;   // 13 mbarriers
    static constexpr int kTmem = kBar + 13 * 8;
    static constexpr int kBytes = kTmem + 16;
    static_assert(kRow % 16 == 0, "rows of whole 16-byte chunks");
    static_assert(kC % 1024 == 0 && kCStage % 128 == 0, "TMA destinations 128-byte aligned");
    static_assert(kBar % 8 == 0, "mbarrier alignment");
};

template <int M, int KB>
constexpr int tma_min_blocks() { return TmaSmem<M, KB>::kBytes <= 113 * 1024 ? 2 : 1; }

// Shared-memory matrix descriptor, K-major, rows of `row` bytes swizzled over the row (row =
// 128, 64 or 32 bytes: swizzle modes 2, 4, 6); sbo = bytes between 8-row groups.  A k-step
// inside the row advances the start address (the swizzle is applied to the full address).
template <int kRowBytes>
__device__ __forceinline__ uint64_t umma_desc_sw(uint32_t addr) {
    static_assert(kRowBytes == 128 || kRowBytes == 64 || kRowBytes == 32, "swizzle width = row");
    constexpr uint64_t mode = kRowBytes == 128 ? 2 : (kRowBytes == 64 ? 4 : 6);
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                                   // leading offset: unused here
    d |= (uint64_t)(((8 * kRowBytes) >> 4) & 0x3FFF) << 32;  // 8-row groups
    d |= (uint64_t)1 << 46;
    d |= mode << 61;
    return d;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_1d(void *dst, const CUtensorMap *tm, int x, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.1d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2}], [%3];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(smem_u32(bar))
        : "memory");
}

// 16 (8) columns of this warp's TMEM lanes, without waiting (tmem_wait_ld completes the loads).
__device__ __forceinline__ void tmem_ld_async(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_async(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Four 32-bit values into four consecutive columns of this warp's TMEM lanes.
__device__ __forceinline__ void tmem_st4(uint32_t taddr, float v0, float v1, float v2, float v3) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(__float_as_uint(v0)),
                 "r"(__float_as_uint(v1)), "r"(__float_as_uint(v2)), "r"(__float_as_uint(v3))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// (x0, x1) = (x0, x1) * a + (b, b), one packed FP32 FMA.
__device__ __forceinline__ void fma2_scale(float &x0, float &x1, float a, float b) {
    asm("{\n\t.reg .b64 x, a, b;\n\t"
        "mov.b64 x, {%0, %1};\n\tmov.b64 a, {%2, %2};\n\tmov.b64 b, {%3, %3};\n\t"
        "fma.rn.f32x2 x, x, a, b;\n\tmov.b64 {%0, %1}, x;\n\t}"
        : "+f"(x0), "+f"(x1)
        : "f"(a), "f"(b));
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(tf32_rna(x)); }

// AND over the 256 epilogue threads (named barrier 2); also orders their shared-memory writes.
__device__ __forceinline__ bool epi_and(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 2, 256, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

// The CTA that owns unit u when U units are split over C CTAs as floor(c U / C) ..
__device__ __forceinline__ int tma_unit_owner(long long u, long long U, long long C) {
    return (int)(((u + 1) * C - 1) / U);
}

template <int M, int KB>
__global__ void __launch_bounds__(kTmaThreads, (tma_min_blocks<M, KB>()))
    detect_tma_kernel(const __grid_constant__ TmaArgs a) {
    using L = TmaSmem<M, KB>;
    constexpr int E = kTmaEntries, CH = M / 2;  // 16-byte k-chunks per row
    constexpr int kSteps = M / 4;               // MMA k-steps of 8 TF32 elements
    constexpr int CE = kTmaChunk;               // entries per TMEM read
    static_assert(M % 4 == 0 && KB % 2 == 0, "whole k-steps, users in pairs");
    static_assert(2 * KB <= 32, "a half's sums fit its own TMEM columns");
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::kBar);
    uint64_t *a_full = bars, *full_b = bars + 1, *full_c = bars + 3, *conv = bars + 6, *a_ready = bars + 8,
             *mma_done = bars + 9, *epi_done = bars + 11;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + L::kTmem);
    float *sG = reinterpret_cast<float *>(smem + L::kC);
    float *sH = reinterpret_cast<float *>(smem + L::kN);  // norms as landed, then -k2 n_t
    float *s_nq = reinterpret_cast<float *>(smem + L::kQ);                 // [128]
    int *s_last = reinterpret_cast<int *>(smem + L::kQ + kTmaRows * 4);    // a split tile's last part

    const int tid = threadIdx.x, warp = tid >> 5;
    int n_ent = a.n_entries;
    if (a.meta) n_ent = min(n_ent, max(__ldg(a.meta), 0));
    // units: (query tile, entry tile); with no entry held, one empty entry tile per query tile
    const int NT = max(1, (n_ent + E - 1) / E), NQ = (a.N + kTmaRows - 1) / kTmaRows;
    const long long U = (long long)NQ * NT, C = gridDim.x;
    const int c = blockIdx.x;
    const int u_lo = (int)((long long)c * U / C), u_hi = (int)((long long)(c + 1) * U / C);
    const int J = u_hi - u_lo;  // tiles this CTA works through

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(a_full, 1);
        mbar_init(a_ready, kTmaEpi);
        for (int i = 0; i < 3; ++i) mbar_init(&full_c[i], 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&full_b[i], 1);
            mbar_init(&conv[i], kTmaEpi);
            mbar_init(&mma_done[i], 1);
            mbar_init(&epi_done[i], kTmaEpi);
        }
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    bool ok = true;

    if (warp == 8) {
        // ================= producer warp =================
        const int lane = tid & 31;
        auto issue_b = [&](int j) {  // entry tile of this CTA's tile j
            const int s = j & 1;
            mbar_arrive_expect_tx(&full_b[s], (uint32_t)L::kBCopy);
            tma_load_2d(smem + L::kB + s * 2 * L::kBCopy, &a.tm_d, 0, ((u_lo + j) % NT) * E, &full_b[s]);
        };
        auto issue_c = [&](int j) {
            const int s = j % 3, e0 = ((u_lo + j) % NT) * E;
            mbar_arrive_expect_tx(&full_c[s], (uint32_t)(L::kCStage + E * 4));
            tma_load_2d(smem + L::kC + s * L::kCStage, &a.tm_g, 0, e0, &full_c[s]);
            tma_load_1d(smem + L::kN + s * E * 4, &a.tm_n, e0, &full_c[s]);
        };
        int nb = 0, nc = 0, committed = -1, na = 0;  // (lane 0) loads issued, last MMA tile
        if (lane == 0) {
            for (; nb < 2 && nb < J; ++nb) issue_b(nb);
            for (; nc < 2 && nc < J; ++nc) issue_c(nc);
        }
        // F32 accumulate, TF32 A and B, both K-major, N = 64, M = 128
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(E >> 3) << 17) |
                               ((uint32_t)(kTmaRows >> 4) << 24);
        const uint32_t a0 = smem_u32(smem + L::kA);
        bool pok = true;
        int j = 0;
        for (int u = u_lo, k = 0; u < u_hi && pok; ++k) {
            const int q = u / NT, u_end = min(u_hi, (q + 1) * NT), j_end = j + (u_end - u);
            // ---- this segment's query rows: the previous segment's MMAs are done with A
            if (lane == 0) {
                if (k > 0) pok = mbar_wait_sleepy(&mma_done[(j - 1) & 1], ((j - 1) >> 1) & 1);
                if (pok) {
                    mbar_arrive_expect_tx(a_full, (uint32_t)L::kACopy);
                    tma_load_2d(smem + L::kA, &a.tm_q, 0, q * kTmaRows, a_full);
                    ++na;
                }
            }
            pok = __shfl_sync(0xffffffffu, pok, 0);
            if (!pok) break;
            // ---- the segment's tiles (lane 0)
            if (lane == 0) {
                const int j0 = j;
                for (; j < j_end && pok; ++j) {
                    const int s = j & 1;
                    // the epilogue converted tile j (and, before the segment's first tile, built
                    // the query operand); the epilogue of tile j-2 freed TMEM stage s
                    if ((j == j0 && !mbar_wait_sleepy(a_ready, k & 1)) || !mbar_wait_sleepy(&conv[s], (j >> 1) & 1) ||
                        (j >= 2 && !mbar_wait_sleepy(&epi_done[s], ((j - 2) >> 1) & 1))) {
                        pok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_re = tmem + (uint32_t)(s * 2 * E), d_im = d_re + E;
                    const uint32_t b0 = smem_u32(smem + L::kB + s * 2 * L::kBCopy);
#pragma unroll
                    for (int ks = 0; ks < kSteps; ++ks) {
                        const uint32_t ao = a0 + ks * 32, bo = b0 + ks * 32;  // 8 TF32 = 32 bytes per k-step
                        const uint64_t are_h = umma_desc_sw<L::kRow>(ao), are_l = umma_desc_sw<L::kRow>(ao + L::kACopy);
                        const uint64_t aim_h = umma_desc_sw<L::kRow>(ao + 2 * L::kACopy);
                        const uint64_t aim_l = umma_desc_sw<L::kRow>(ao + 3 * L::kACopy);
                        const uint64_t bh = umma_desc_sw<L::kRow>(bo), bl = umma_desc_sw<L::kRow>(bo + L::kBCopy);
                        umma_tf32(d_re, are_l, bh, idesc, ks > 0);
                        umma_tf32(d_re, are_h, bl, idesc, 1);
                        umma_tf32(d_re, are_h, bh, idesc, 1);
                        umma_tf32(d_im, aim_l, bh, idesc, ks > 0);
                        umma_tf32(d_im, aim_h, bl, idesc, 1);
                        umma_tf32(d_im, aim_h, bh, idesc, 1);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&mma_done[s]))
                                 : "memory");
                    committed = j;
                    if (j + 2 < J) {
                        // entry stage s is free once these MMAs are done; coefficient stage
                        // (j+2) mod 3 once the epilogue of tile j-1 is
                        if (!mbar_wait_sleepy(&mma_done[s], (j >> 1) & 1)) {
                            pok = false;
                            break;
                        }
                        issue_b(j + 2);
                        ++nb;
                        if (j >= 1 && !mbar_wait_sleepy(&epi_done[(j - 1) & 1], ((j - 1) >> 1) & 1)) {
                            pok = false;
                            break;
                        }
                        issue_c(j + 2);
                        ++nc;
                    }
                }
            }
            pok = __shfl_sync(0xffffffffu, pok, 0);
            j = __shfl_sync(0xffffffffu, j, 0);
            u = u_end;
        }
        ok = pok;
        if (lane == 0) {
            // every copy and MMA this warp issued has landed before the CTA may exit
            if (na > 0) mbar_wait_sleepy(a_full, (na - 1) & 1);
            for (int t = max(0, nb - 2); t < nb; ++t) mbar_wait_sleepy(&full_b[t & 1], (t >> 1) & 1);
            for (int t = max(0, nc - 3); t < nc; ++t) mbar_wait_sleepy(&full_c[t % 3], (t / 3) & 1);
            if (committed >= 0) mbar_wait_sleepy(&mma_done[committed & 1], (committed >> 1) & 1);
        }
    } else {
        // ================= epilogue =================
        const int row = tid & (kTmaRows - 1), hf = tid >> 7;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        const float g2 = 2.f * a.k2;
        // one tile's landed loads -> entry operand copies, -k2 n_t, zeros past the held entries
        auto convert = [&](int jj) -> bool {
            const int sb = jj & 1, sc = jj % 3;
            const bool w = mbar_wait_bounded(&full_b[sb], (jj >> 1) & 1) && mbar_wait_bounded(&full_c[sc], (jj / 3) & 1);
            if (!__all_sync(0xffffffffu, w)) return false;
            const int nvalid = n_ent - ((u_lo + jj) % NT) * E;  // rows at or past it are not held entries
            float4 *bh = reinterpret_cast<float4 *>(smem + L::kB + sb * 2 * L::kBCopy);
            float4 *bl = bh + L::kBCopy / 16;
            for (int f = tid; f < CH * E; f += kTmaEpi) {  // chunk f is one of the CH chunks of row f / CH
                const float4 x = bh[f];
                float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
                if (f / CH < nvalid) {
                    h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
                    l = make_float4(tf32_hi(x.x - h.x), tf32_hi(x.y - h.y), tf32_hi(x.z - h.z), tf32_hi(x.w - h.w));
                }
                bh[f] = h;
                bl[f] = l;
            }
            if (tid < E) sH[sc * E + tid] = tid < nvalid ? -a.k2 * sH[sc * E + tid] : -INFINITY;
            if (nvalid < E)
                for (int i = tid; i < E * 2 * KB; i += kTmaEpi)
                    if (i / (2 * KB) >= nvalid) sG[sc * E * 2 * KB + i] = 0.f;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&conv[sb]);
            return true;
        };
        if (J > 0) ok = convert(0);

        float acc1[KB], acc2[KB];
        int j = 0;
        for (int u = u_lo, k = 0; u < u_hi; ++k) {
            const int q = u / NT, u_end = min(u_hi, (q + 1) * NT), j_end = j + (u_end - u);
            const bool whole = u == q * NT && u_end == (q + 1) * NT;
            const int s_row = q * kTmaRows + row;
            // ---- the segment's query operand: raw rows -> [re_hi, re_lo, im_hi, im_lo] in place
            // per 16-byte chunk (chunk f is one of the CH chunks of row f / CH; CH consecutive
            // lanes hold one row), squared norms by row
            if (ok) ok = __all_sync(0xffffffffu, mbar_wait_bounded(a_full, k & 1));
            bool rows_in_range = true;
            {
                float4 *qv = reinterpret_cast<float4 *>(smem + L::kA);
                constexpr int QV = L::kACopy / 16;
#pragma unroll
                for (int i = 0; i < CH / 2; ++i) {
                    const int f = tid + kTmaEpi * i;
                    const float4 x = ok ? qv[f] : make_float4(0.f, 0.f, 0.f, 0.f);
                    float nqf = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, x.w * x.w)));
#pragma unroll
                    for (int o = 1; o < CH; o <<= 1) nqf += __shfl_xor_sync(0xffffffffu, nqf, o);
                    if ((f & (CH - 1)) == 0) s_nq[f / CH] = nqf;
                    rows_in_range = rows_in_range && a.k2 * nqf <= kFactorLimit;
                    const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
                    const float4 l = make_float4(tf32_hi(x.x - h.x), tf32_hi(x.y - h.y), tf32_hi(x.z - h.z),
                                                 tf32_hi(x.w - h.w));
                    qv[f] = h;
                    qv[QV + f] = l;
                    qv[2 * QV + f] = make_float4(h.y, -h.x, h.w, -h.z);  // (Im, -Re) pairs
                    qv[3 * QV + f] = make_float4(l.y, -l.x, l.w, -l.z);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(a_ready);
            const bool in_range = epi_and(rows_in_range);  // also: every query norm is written
            const float nq = s_nq[row];
#pragma unroll
            for (int kk = 0; kk < KB; ++kk) acc1[kk] = acc2[kk] = 0.f;
            const float hq = in_range ? 0.f : -a.k2 * nq;  // unfactored exponent when out of range
            // direct-difference fallback (as in detect_tc.cuh), for query tiles outside the factor
            // range only: inside it the TF32 x3 Gram error is below 2^-21 S in the exponent
            const float one_m_theta = 1.f - kGuardF32;
            const float thr_q = one_m_theta * a.k2 * nq;
            const float base_q = a.k2 * nq + hq;
            auto exact_pair = [&](const float *g_tile, int e, int e0) {
                const int t = e0 + e;
                if (t >= n_ent || s_row >= a.N) return;
                const float2 *rq = a.rx + (size_t)s_row * M;
                const float2 *rt = a.dict + (size_t)t * M;
                float dA = 0.f, dB = 0.f, dC = 0.f;
#pragma unroll 4
                for (int m = 0; m < M; ++m) {
                    const float2 qq = __ldg(rq + m), d = __ldg(rt + m);
                    const float ax = d.x - qq.x, ay = d.y - qq.y;
                    const float bx = d.x - qq.y, by = d.y + qq.x;
                    const float cx = d.x + qq.y, cy = d.y - qq.x;
                    dA = fmaf(ax, ax, fmaf(ay, ay, dA));
                    dB = fmaf(bx, bx, fmaf(by, by, dB));
                    dC = fmaf(cx, cx, fmaf(cy, cy, dC));
                }
                const float eA = ex2(base_q - a.k2 * dA), eB = ex2(base_q - a.k2 * dB),
                            eC = ex2(base_q - a.k2 * dC);
                float g1[KB], gg[KB];
                load_coef<KB>(g_tile + e * 2 * KB, g1, gg);
#pragma unroll
                for (int kk = 0; kk < KB; ++kk) {
                    acc1[kk] = fmaf(g1[kk], eA, fmaf(gg[kk], eC, acc1[kk]));
                    acc2[kk] = fmaf(g1[kk], eB, fmaf(gg[kk], eA, acc2[kk]));
                }
            };
            auto run_tiles = [&](auto guard_c) {
                constexpr bool kGuard = decltype(guard_c)::value;
                for (; j < j_end; ++j) {
                    const int s = j & 1, sc = j % 3;
                    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&mma_done[s], (j >> 1) & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    if (j + 1 < J && !convert(j + 1)) {  // the MMAs of tile j+1 run beside this epilogue
                        ok = false;
                        break;
                    }
                    const float *g_tile = sG + sc * E * 2 * KB;
                    const float *g = g_tile + hf * 32 * 2 * KB;
                    const float *hh = sH + sc * E + hf * 32;
#pragma unroll 1
                    for (int cc = 0; cc < 32 / CE; ++cc) {
                        uint32_t vr[CE], vi[CE];
                        const uint32_t col = tmem + lane_base + (uint32_t)(s * 2 * E + hf * 32 + CE * cc);
                        tmem_ld_async(col, vr);
                        tmem_ld_async(col + E, vi);
                        float hv[CE];
#pragma unroll
                        for (int v4 = 0; v4 < CE / 4; ++v4)
                            *reinterpret_cast<float4 *>(hv + 4 * v4) =
                                *reinterpret_cast<const float4 *>(hh + CE * cc + 4 * v4);
                        tmem_wait_ld();
                        uint32_t fbits = 0;
#pragma unroll
                        for (int jj = 0; jj < CE; ++jj) {
                            const float re = __uint_as_float(vr[jj]), im = __uint_as_float(vi[jj]);
                            float h = hv[jj];
                            if constexpr (kGuard) {
                                h += hq;
                                // flagged: 2 k2 max(Re z, |Im z|) > (1 - theta) k2 (n_s + n_t)
                                const bool f = g2 * fmaxf(re, fabsf(im)) > fmaf(-one_m_theta, hv[jj], thr_q);
                                h = f ? -INFINITY : h;
                                fbits |= f ? (1u << jj) : 0u;
                            }
                            float xA = re, xB = im;
                            fma2_scale(xA, xB, g2, h);  // (2 k2 Re z + h, 2 k2 Im z + h)
                            const float eA = ex2(xA), eB = ex2(xB), eC = ex2(fmaf(-g2, im, h));
                            float g1[KB], gg[KB];
                            load_coef<KB>(g + (CE * cc + jj) * 2 * KB, g1, gg);
#pragma unroll
                            for (int kk = 0; kk < KB; kk += 2) {
                                fma2_pair(acc1[kk], acc1[kk + 1], gg[kk], gg[kk + 1], eC);
                                fma2_pair(acc1[kk], acc1[kk + 1], g1[kk], g1[kk + 1], eA);
                                fma2_pair(acc2[kk], acc2[kk + 1], gg[kk], gg[kk + 1], eA);
                                fma2_pair(acc2[kk], acc2[kk + 1], g1[kk], g1[kk + 1], eB);
                            }
                        }
                        if constexpr (kGuard) {
                            if (__any_sync(0xffffffffu, fbits != 0)) {
#pragma unroll 1
                                while (fbits) {
                                    const int jj = __ffs(fbits) - 1;
                                    fbits &= fbits - 1;
                                    exact_pair(g_tile, hf * 32 + CE * cc + jj, ((u_lo + j) % NT) * E);
                                }
                            }
                        }
                    }
                    if (j + 1 < j_end) {  // (the last tile's stage is released after the merge)
                        tc_fence_before();
                        mbar_arrive(&epi_done[s]);
                    }
                }
            };
            if (ok) {
                if (in_range) run_tiles(std::false_type{});
                else run_tiles(std::true_type{});
            }
            ok = epi_and(ok);  // every epilogue thread goes on to the merge's barriers, or none
            if (!ok) break;
            // ---- merge the two halves through the last tile's TMEM stage: the second half's
            // sums and its half of the linear part go into its own columns of that stage, which
            // nothing reads any more until its epilogue-done arrival below
            float l1[KB], l2[KB];  // c_k^H r over this half's antennas [hf M/2, (hf+1) M/2)
#pragma unroll
            for (int kk = 0; kk < KB; ++kk) l1[kk] = l2[kk] = 0.f;
            if (s_row < a.N) {
                const float2 *rq = a.rx + (size_t)s_row * M;
#pragma unroll 2
                for (int m = hf * (M / 2); m < (hf + 1) * (M / 2); ++m) {
                    const float2 r = __ldg(rq + m);
#pragma unroll
                    for (int kk = 0; kk < KB; ++kk) {
                        const float2 cl = __ldg(a.clin + m * KB + kk);
                        l1[kk] = fmaf(cl.x, r.x, fmaf(cl.y, r.y, l1[kk]));
                        l2[kk] = fmaf(cl.x, r.y, fmaf(-cl.y, r.x, l2[kk]));
                    }
                }
            }
            const int sl = (j_end - 1) & 1;
            const uint32_t mcol = tmem + lane_base + (uint32_t)(sl * 2 * E + 32);        // acc1, acc2
            const uint32_t lcol = tmem + lane_base + (uint32_t)(sl * 2 * E + E + 32);    // l1, l2
            if (hf == 1) {
#pragma unroll
                for (int kk = 0; kk < KB; kk += 2) {
                    tmem_st4(mcol + 2 * kk, acc1[kk], acc1[kk + 1], acc2[kk], acc2[kk + 1]);
                    tmem_st4(lcol + 2 * kk, l1[kk], l1[kk + 1], l2[kk], l2[kk + 1]);
                }
                tmem_wait_st();
            }
            tc_fence_before();
            asm volatile("bar.sync 1, 256;" ::: "memory");
            tc_fence_after();
            if (hf == 0) {
#pragma unroll
                for (int kk = 0; kk < KB; kk += 2) {
                    float v[4], w[4];
                    tmem_ld4(mcol + 2 * kk, v);
                    tmem_ld4(lcol + 2 * kk, w);
                    acc1[kk] += v[0];
                    acc1[kk + 1] += v[1];
                    acc2[kk] += v[2];
                    acc2[kk + 1] += v[3];
                    l1[kk] += w[0];
                    l1[kk + 1] += w[1];
                    l2[kk] += w[2];
                    l2[kk + 1] += w[3];
                }
            }
            tc_fence_before();
            mbar_arrive(&epi_done[sl]);
            if (hf == 0) {
                bool fin = whole;
                if (!whole) {
                    // a part of a split query tile: leave the sums in this CTA's slot; the CTA that
                    // brings the tile's last part adds all parts in CTA order
                    const int slot = 2 * c + (q == u_lo / NT ? 0 : 1);
                    float *dst = a.parts + ((size_t)slot * kTmaRows + row) * 2 * KB;
#pragma unroll
                    for (int kk = 0; kk < KB; ++kk) {
                        dst[kk] = acc1[kk];
                        dst[KB + kk] = acc2[kk];
                    }
                    __threadfence();
                    asm volatile("bar.sync 3, 128;" ::: "memory");
                    // the tile's parts: the distinct owners of its units, in unit order (CTAs
                    // that own no unit at all own none of them)
                    int n_parts = 0;
                    for (int uu = q * NT, prev = -1; uu < (q + 1) * NT; ++uu) {
                        const int o = tma_unit_owner(uu, U, C);
                        n_parts += o != prev;
                        prev = o;
                    }
                    if (row == 0) *s_last = atomicAdd(a.counters + q, 1) == n_parts - 1;
                    asm volatile("bar.sync 3, 128;" ::: "memory");
                    fin = *s_last != 0;
                    if (fin) {
                        __threadfence();
#pragma unroll
                        for (int kk = 0; kk < KB; ++kk) acc1[kk] = acc2[kk] = 0.f;
                        for (int uu = q * NT, prev = -1; uu < (q + 1) * NT; ++uu) {
                            const int cp = tma_unit_owner(uu, U, C);
                            if (cp == prev) continue;
                            prev = cp;
                            const int ulo_p = (int)((long long)cp * U / C);
                            const int slot_p = 2 * cp + (q == ulo_p / NT ? 0 : 1);
                            const float *src = a.parts + ((size_t)slot_p * kTmaRows + row) * 2 * KB;
#pragma unroll
                            for (int kk = 0; kk < KB; ++kk) {
                                acc1[kk] += __ldcg(src + kk);
                                acc2[kk] += __ldcg(src + KB + kk);
                            }
                        }
                        if (row == 0) a.counters[q] = 0;  // the workspace is left as it was found
                    }
                    asm volatile("bar.sync 3, 128;" ::: "memory");  // (*s_last is reused)
                }
                if (fin && s_row < a.N) {
                    const float fq = in_range ? ex2(-a.k2 * nq) : 1.f;  // query factor
#pragma unroll
                    for (int kk = 0; kk < KB; ++kk) {
                        const float y1 = fmaf(a.wL, l1[kk], a.wG * fq * acc1[kk]);
                        const float y2 = fmaf(a.wL, l2[kk], a.wG * fq * acc2[kk]);
                        a.soft[(size_t)s_row * KB + kk] = make_float2(y1, y2);
                        if (a.hard)
                            a.hard[(size_t)s_row * KB + kk] = (uint8_t)((y1 < 0.f ? 1 : 0) | (y2 < 0.f ? 2 : 0));
                    }
                }
            }
            j = j_end;
            u = u_end;
        }
    }
    if (!ok && (tid == 0 || tid == 256)) report(a.status, APSM_ERR_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
}

// ---- host side: tensor maps and launch ------------------------------------------------------

using TmaEncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
TmaEncodeFn tma_encode_fn();  // the driver's tiled tensor-map encoder (detect_dispatch.cu); null if absent

// FP32 tensor map over `rows` rows of `inner` floats (row pitch row_bytes), box box_inner x
// box_rows (rank 1 when rows == 0: `inner` floats, box box_inner).  Out-of-range boxes read zero.
inline bool tma_map_f32(CUtensorMap *m, const void *base, uint64_t inner, uint64_t rows, uint64_t row_bytes,
                        uint32_t box_inner, uint32_t box_rows,
                        CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_NONE) {
    const TmaEncodeFn enc = tma_encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[2] = {inner, rows};
    const cuuint64_t strides[1] = {row_bytes};
    const cuuint32_t box[2] = {box_inner, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rows ? 2 : 1, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Layout of the balanced form's workspace for N queries and up to `ctas` CTAs:
// counters [ceil(N / 128)] int (256-byte aligned), then parts [2 ctas][128][2 KB] float.
struct TmaWorkspace {
    size_t counters, parts, total;
    int ctas;
};
inline TmaWorkspace tma_workspace(int N, int KB, int ctas) {
    TmaWorkspace w{};
    const size_t nq = (size_t)(N + kTmaRows - 1) / kTmaRows;
    w.ctas = ctas;
    w.counters = 0;
    w.parts = (nq * 4 + 255) / 256 * 256;
    w.total = w.parts + (size_t)2 * ctas * kTmaRows * 2 * KB * 4;
    return w;
}

// Launches the kernel for (M, KB): the balanced form (resident CTAs per SM x `sms` CTAs) when
// `workspace` (tma_workspace(N, KB, 2 sms) bytes, zeroed before its first use) is given, else
// one CTA per query tile.  Returns 0 when launched, 1 when this form does not apply (user count
// not its own bucket, unaligned arrays, no tensor-map encoder, workspace too small: use
// detect_tc.cuh), -1 on a CUDA error.
template <int M, int KB>
int launch_detect_tma(const TcArgs &in, void *workspace, size_t ws_bytes, int sms, cudaStream_t stream) {
    using L = TmaSmem<M, KB>;
    if (in.K != KB || in.N <= 0 || in.n_entries <= 0) return 1;
    auto al16 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    if (!al16(in.rx) || !al16(in.dict) || !al16(in.gamma) || !al16(in.dict_norm)) return 1;
    TmaArgs a{};
    const uint64_t D = (uint64_t)in.n_entries;
    constexpr CUtensorMapSwizzle swz = M == 16 ? CU_TENSOR_MAP_SWIZZLE_128B
                                       : (M == 8 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
    if (!tma_map_f32(&a.tm_q, in.rx, 2 * M, (uint64_t)in.N, 8 * M, 2 * M, kTmaRows, swz) ||
        !tma_map_f32(&a.tm_d, in.dict, 2 * M, D, 8 * M, 2 * M, kTmaEntries, swz) ||
        !tma_map_f32(&a.tm_g, in.gamma, 2 * KB, D, 8 * KB, 2 * KB, kTmaEntries) ||
        !tma_map_f32(&a.tm_n, in.dict_norm, D, 0, 0, kTmaEntries, 1))
        return 1;
    a.rx = in.rx;
    a.N = in.N;
    a.dict = in.dict;
    a.clin = in.clin;
    a.meta = in.meta;
    a.n_entries = in.n_entries;
    a.k2 = in.k2;
    a.wL = in.wL;
    a.wG = in.wG;
    a.soft = in.soft;
    a.hard = in.hard;
    a.status = in.status;
    const int nq = (in.N + kTmaRows - 1) / kTmaRows;
    int grid = nq;
    if (workspace) {
        const int ctas = tma_min_blocks<M, KB>() * sms;
        const TmaWorkspace w = tma_workspace(in.N, KB, 2 * sms);
        if (sms < 1 || ws_bytes < w.total || (reinterpret_cast<uintptr_t>(workspace) & 255)) return 1;
        a.counters = reinterpret_cast<int *>(static_cast<char *>(workspace) + w.counters);
        a.parts = reinterpret_cast<float *>(static_cast<char *>(workspace) + w.parts);
        const long long units = (long long)nq * ((in.n_entries + kTmaEntries - 1) / kTmaEntries);
        grid = (int)std::min<long long>(ctas, units);
    }
    auto fn = detect_tma_kernel<M, KB>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes) != cudaSuccess) return -1;
    // an ordinary launch: every read may take the L1 path (see launch_detect_tc)
    fn<<<grid, kTmaThreads, L::kBytes, stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

using TmaLauncher = int (*)(const TcArgs &, void *, size_t, int, cudaStream_t);

}  // namespace apsm
