// detect_tc_batch.cuh -- the batched form of the tensor-core detection (many detector instances
// of one antenna count and user bucket in one persistent launch).
//
// The same per-tile arithmetic as detect_tc_kernel (Sec. III-B detection; the dist-Gram on
// tcgen05, exponentials and coefficient sums in the epilogue), but each CTA stays resident and
// takes work items -- (instance, first query of a 128-query tile) -- from a device counter until
// the list is exhausted.  Items are listed longest instance first, so the last items to start are
// the short ones and the CTAs finish together.  The pipeline's stage and phase bookkeeping runs
// over all tiles a CTA processes (gt0 + tile), so items follow one another without resetting
// barriers or TMEM; one CTA barrier between items guarantees that the next item's query operand
// is written only after every MMA of the previous item has been waited for.  Each item's
// instance descriptor is staged in shared memory.  Per item the results are those of
// detect_tc_kernel for that instance bit for bit (the same tiles in the same order).
#pragma once

#include "detect_tc.cuh"

namespace apsm {

struct TcBatchArgs {
    const TcArgs *jobs;   // [n_jobs] one descriptor per instance of this class
    const int2 *items;    // [n_items] (job, first query), longest instance first
    int n_items;
    int *counter;         // work counter, zero when the launch starts
    int half_fmt;         // kHalf only: 1 = BF16, 0 = FP16
};

template <int M, int KB, int kPrec>
__global__ void __launch_bounds__(kTcThreads, (tc_min_blocks<M, KB, kPrec>())) detect_tc_batch_kernel(const TcBatchArgs ba) {
    using Sh = TcShape<M, kPrec>;
    using L = TcSmem<M, KB, kPrec>;
    static_assert(KB % 2 == 0, "the coefficient sums run over user pairs");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem + L::kA;
    unsigned char *sB = smem + L::kB;
    float *sG = reinterpret_cast<float *>(smem + L::kG);
    float *sH = reinterpret_cast<float *>(smem + L::kN);
    uint64_t *mma_done = reinterpret_cast<uint64_t *>(smem + L::kBar);  // [2]: commit + 128 converters
    uint64_t *epi_done = mma_done + 2;                                   // [2]: 128 epilogue threads
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + L::kTmem);
    __shared__ TcArgs s_job;   // the current item's instance
    __shared__ int s_item;
    constexpr int E = kTcEntries, NB = 2 * kTcEntries;
    constexpr uint32_t kCols = 2 * NB;  // two accumulators of NB fp32 columns

    const int tid = threadIdx.x, warp = tid >> 5;

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
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();  // TMEM address and barrier initialisation visible to every thread
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    const int half_fmt = ba.half_fmt;
    int gt0 = 0;      // tiles this CTA has run so far: stage = gt & 1, phase parity = (gt >> 1) & 1
    bool ok = true;
    for (;;) {
    // ---- next item: (instance, first query) from the work counter -------------------------------
    if (tid == 0) {
        s_item = atomicAdd(ba.counter, 1);
        if (s_item < ba.n_items) s_job = ba.jobs[ba.items[s_item].x];
    }
    __syncthreads();
    if (s_item >= ba.n_items) break;
    const TcArgs &a = s_job;
    const int q0 = ba.items[s_item].y;
    int n_ent = a.n_entries;
    if (a.meta) n_ent = min(n_ent, max(__ldg(a.meta), 0));
    const int n_tiles = (n_ent + E - 1) / E;
    const float g2 = 2.f * a.k2;
    float nq = 0.f;  // squared norm of this epilogue thread's query
    if (warp < 4) {
        const int s = q0 + tid;
        const float2 *rq = a.rx + (size_t)s * M;
        if constexpr (tc_core_rows<M, kPrec>()) {
            // this thread's query row by whole core rows: [Re | Im] x 2 k2 (a quarter-warp writes
            // eight consecutive rows of one core column: conflict-free 16-byte stores)
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
                put_core<kPrec, C>(sA, Sh::kBytesA, Sh::off(tid, p * C), re, half_fmt);
                put_core<kPrec, C>(sA, Sh::kBytesA, Sh::off(tid, M + p * C), im, half_fmt);
            }
        } else {
            for (int m = 0; m < M; ++m) {
                const float2 v = s < a.N ? __ldg(rq + m) : make_float2(0.f, 0.f);
                nq = fmaf(v.x, v.x, fmaf(v.y, v.y, nq));
                put_elem<kPrec>(sA, Sh::kBytesA, Sh::off(tid, m), g2 * v.x, half_fmt);
                put_elem<kPrec>(sA, Sh::kBytesA, Sh::off(tid, M + m), g2 * v.y, half_fmt);
            }
            for (int k = 2 * M; k < Sh::KD; ++k) put_elem<kPrec>(sA, Sh::kBytesA, Sh::off(tid, k), 0.f, half_fmt);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    const bool cta_in_range = __syncthreads_and(warp >= 4 || a.k2 * nq <= kFactorLimit);
    tc_fence_after();


    uint32_t idesc;
    if constexpr (kPrec == kTF32x3) {
        idesc = (1u << 4) | (2u << 7) | (2u << 10);  // F32 accumulate, TF32 A and B, K-major
    } else {
        const uint32_t f = half_fmt ? 1u : 0u;    // BF16 (1) or FP16 (0)
        idesc = (1u << 4) | (f << 7) | (f << 10);
    }
    idesc |= ((uint32_t)(NB >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);

    float acc1[KB], acc2[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) acc1[k] = acc2[k] = 0.f;

    if (warp >= 4) {
        // ================= converters + MMA issue =================
        const int ct = tid - 128;  // converter index (element-wise form: B row ct = entry ct/2, half ct%2)
        // global loads of a tile issued ahead of the wait for its stage (whole-core-row form)
        constexpr bool kVecG = (2 * KB) % 4 == 0;
        constexpr int kQ = 2 * KB / 4, kGQ = (E * kQ + 127) / 128;
        const bool vec_g = kVecG && a.K == KB;
        EntryRows<M, kPrec> rows;
        float4 gpf[kGQ];
        float hpf = 0.f;
        auto prefetch = [&](int tile) {
            const int e0 = tile * E;
            if constexpr (tc_core_rows<M, kPrec>()) rows.prefetch(a.dict, e0, n_ent, ct);
            if (vec_g) {
#pragma unroll
                for (int j = 0; j < kGQ; ++j) {
                    const int idx = ct + 128 * j, e = idx / kQ, q = idx % kQ, t = e0 + e;
                    gpf[j] = (idx < E * kQ && t < n_ent)
                                 ? __ldg(reinterpret_cast<const float4 *>(a.gamma + (size_t)t * 2 * KB) + q)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            hpf = (ct < E && e0 + ct < n_ent) ? -a.k2 * __ldg(a.dict_norm + e0 + ct) : 0.f;
        };
        if (n_tiles > 0) prefetch(0);
        for (int tile = 0; tile < n_tiles; ++tile) {
            const int gt = gt0 + tile, st = gt & 1;
            // the epilogue of tile gt-2 (this item's or an earlier one's) has released stage st,
            // and it waited for the MMAs of gt-2, the last readers of B stage st
            bool w = true;
            if (gt >= 2) w = mbar_wait_bounded(&epi_done[st], ((gt - 2) >> 1) & 1);
            if (!converters_and(w)) {
                ok = false;
                break;
            }
            const int e0 = tile * E;
            unsigned char *bst = sB + st * Sh::kCopies * Sh::kBytesB;
            if constexpr (tc_core_rows<M, kPrec>()) {
                rows.write(bst, a.dict, e0, n_ent, ct, half_fmt);
            } else {
                const int t = e0 + (ct >> 1), h = ct & 1;
                const float2 *rt = a.dict + (size_t)t * M;
                // row 2e: [Re r_t; Im r_t] gives Re z;  row 2e+1: [-Im r_t; Re r_t] gives Im z
                for (int m = 0; m < M; ++m) {
                    const float2 v = t < n_ent ? __ldg(rt + m) : make_float2(0.f, 0.f);
                    put_elem<kPrec>(bst, Sh::kBytesB, Sh::off(ct, m), h ? -v.y : v.x, half_fmt);
                    put_elem<kPrec>(bst, Sh::kBytesB, Sh::off(ct, M + m), h ? v.x : v.y, half_fmt);
                }
                for (int k = 2 * M; k < Sh::KD; ++k) put_elem<kPrec>(bst, Sh::kBytesB, Sh::off(ct, k), 0.f, half_fmt);
            }
            if (vec_g) {
                // the tile's coefficients row by row as float4 (global [2][K] = shared [2 KB])
#pragma unroll
                for (int j = 0; j < kGQ; ++j) {
                    const int idx = ct + 128 * j, e = idx / kQ, q = idx % kQ;
                    if (idx < E * kQ) *reinterpret_cast<float4 *>(sG + (st * E + e) * 2 * KB + 4 * q) = gpf[j];
                }
            } else if (ct < E) {  // the tile's coefficients (zero past the last entry and user)
                const int t = e0 + ct;
                float *g = sG + (st * E + ct) * 2 * KB;
#pragma unroll
                for (int j = 0; j < 2 * KB; ++j) {
                    const int l = j / KB, k = j % KB;
                    g[j] = (t < n_ent && k < a.K) ? __ldg(a.gamma + ((size_t)t * 2 + l) * a.K + k) : 0.f;
                }
            }
            if (ct < E) sH[st * E + ct] = hpf;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            named_sync(1, 128);
            mbar_arrive(&mma_done[st]);  // releases this thread's coefficient and norm writes
            if (ct == 0) {
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(st * NB);
                const uint32_t a0 = smem_u32(sA), b0 = smem_u32(bst);
#pragma unroll
                for (int s = 0; s < Sh::kSteps; ++s) {
                    const uint64_t ah = umma_sdesc(a0 + s * 256, Sh::SBO), bh = umma_sdesc(b0 + s * 256, Sh::SBO);
                    if constexpr (kPrec == kTF32x3) {
                        const uint64_t al = umma_sdesc(a0 + Sh::kBytesA + s * 256, Sh::SBO);
                        const uint64_t bl = umma_sdesc(b0 + Sh::kBytesB + s * 256, Sh::SBO);
                        umma_tf32(d, al, bh, idesc, s > 0);
                        umma_tf32(d, ah, bl, idesc, 1);
                        umma_tf32(d, ah, bh, idesc, 1);
                    } else {
                        umma_f16(d, ah, bh, idesc, s > 0);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&mma_done[st]))
                             : "memory");
            }
            if (tile + 1 < n_tiles) prefetch(tile + 1);
        }
    } else {
        // ================= epilogue: exponentials and coefficient sums =================
        const float hq = cta_in_range ? 0.f : -a.k2 * nq;  // unfactored exponent when out of range
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        const int s_row = q0 + tid;
        // Cancellation guard (direct-difference fallback).  With S = k2 (n_s + n_t) and v the
        // Gram's exponent columns (2 k2 Re z, 2 k2 Im z), the three scaled squared distances are
        // S - v_re, S - v_im and S + v_im; their minimum is S - max(v_re, |v_im|).  A pair whose
        // minimum falls below theta S (theta = kGuardHalf for BF16/FP16, kGuardF32 for TF32 x3)
        // is one where the norm expansion cancels while its exponential still matters: its
        // terms are dropped from the fast loop (exponent -inf) and recomputed from the FP32 query
        // and entry by direct differences.  TF32 x3 needs it only for queries outside the factor
        // range (inside it the Gram error is below 2^-21 S <= 6e-5 in the exponent).
        const bool guard = kPrec == kHalf || !cta_in_range;
        const float one_m_theta = 1.f - (kPrec == kHalf ? kGuardHalf : kGuardF32);
        const float thr_q = one_m_theta * a.k2 * nq;  // (1 - theta) k2 n_s
        const float base_q = a.k2 * nq + hq;           // exponent offset of the exact terms
        const float *g_all = sG;
        // exact terms of entry e of the current tile (stage st): three squared distances by direct
        // differences of the FP32 query and entry (no norm expansion)
        auto exact_pair = [&](int st, int e, int e0) {
            const int t = e0 + e;
            if (t >= n_ent || s_row >= a.N) return;
            const float2 *rq = a.rx + (size_t)s_row * M;
            const float2 *rt = a.dict + (size_t)t * M;
            float dA = 0.f, dB = 0.f, dC = 0.f;
#pragma unroll 4
            for (int m = 0; m < M; ++m) {
                const float2 q = __ldg(rq + m), d = __ldg(rt + m);
                const float ax = d.x - q.x, ay = d.y - q.y;  // r_t - r_s
                const float bx = d.x - q.y, by = d.y + q.x;  // r_t + i r_s  (r1(t) vs r2(s))
                const float cx = d.x + q.y, cy = d.y - q.x;  // r_t - i r_s  (r2(t) vs r1(s))
                dA = fmaf(ax, ax, fmaf(ay, ay, dA));
                dB = fmaf(bx, bx, fmaf(by, by, dB));
                dC = fmaf(cx, cx, fmaf(cy, cy, dC));
            }
            const float eA = ex2(base_q - a.k2 * dA), eB = ex2(base_q - a.k2 * dB), eC = ex2(base_q - a.k2 * dC);
            float g1[KB], gg[KB];
            load_coef<KB>(g_all + (st * E + e) * 2 * KB, g1, gg);
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                acc1[k] = fmaf(g1[k], eA, fmaf(gg[k], eC, acc1[k]));
                acc2[k] = fmaf(g1[k], eB, fmaf(gg[k], eA, acc2[k]));
            }
        };
        auto run_tiles = [&](auto guard_c) {
            constexpr bool kGuard = decltype(guard_c)::value;
            for (int tile = 0; tile < n_tiles; ++tile) {
                const int gt = gt0 + tile, st = gt & 1;
                // warp-uniform decision: tcgen05.ld below is executed by whole warps only
                if (!__all_sync(0xffffffffu, mbar_wait_bounded(&mma_done[st], (gt >> 1) & 1))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const float *g = sG + st * E * 2 * KB;
                const float *hh = sH + st * E;
#pragma unroll 1
                for (int c = 0; c < NB / 16; ++c) {
                    float v[16], hv[8];
                    tmem_ld16(tmem + lane_base + (uint32_t)(st * NB + 16 * c), v);
                    *reinterpret_cast<float4 *>(hv) = *reinterpret_cast<const float4 *>(hh + 8 * c);
                    *reinterpret_cast<float4 *>(hv + 4) = *reinterpret_cast<const float4 *>(hh + 8 * c + 4);
                    bool flagged = false;
                    uint32_t fbits = 0;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int e = 8 * c + j;
                        float h = hv[j] + hq;
                        if constexpr (kGuard) {
                            // flagged: max(v_re, |v_im|) > (1 - theta) k2 (n_s + n_t)
                            const bool f = fmaxf(v[2 * j], fabsf(v[2 * j + 1])) > fmaf(-one_m_theta, hv[j], thr_q);
                            h = f ? -INFINITY : h;
                            fbits |= f ? (1u << j) : 0u;
                            flagged |= f;
                        }
                        float xA = v[2 * j], xB = v[2 * j + 1];
                        add2_bcast(xA, xB, h);  // (Re z + h, Im z + h)
                        const float eA = ex2(xA), eB = ex2(xB), eC = ex2(h - v[2 * j + 1]);
                        float g1[KB], gg[KB];
                        load_coef<KB>(g + e * 2 * KB, g1, gg);
                        // acc1 = g1 E_A + g2 E_C + acc1,  acc2 = g1 E_B + g2 E_A + acc2, users in pairs
#pragma unroll
                        for (int k = 0; k < KB; k += 2) {
                            fma2_pair(acc1[k], acc1[k + 1], gg[k], gg[k + 1], eC);
                            fma2_pair(acc1[k], acc1[k + 1], g1[k], g1[k + 1], eA);
                            fma2_pair(acc2[k], acc2[k + 1], gg[k], gg[k + 1], eA);
                            fma2_pair(acc2[k], acc2[k + 1], g1[k], g1[k + 1], eB);
                        }
                    }
                    if constexpr (kGuard) {
                        if (__any_sync(0xffffffffu, flagged)) {
#pragma unroll 1
                            while (fbits) {
                                const int j = __ffs(fbits) - 1;
                                fbits &= fbits - 1;
                                exact_pair(st, 8 * c + j, tile * E);
                            }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(&epi_done[st]);
            }
        };
        if constexpr (kPrec == kHalf) {
            run_tiles(std::true_type{});
        } else {
            if (guard) run_tiles(std::true_type{});
            else run_tiles(std::false_type{});
        }
        const int s = s_row;
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
                    if (kk == k) { y1 = acc1[kk]; y2 = acc2[kk]; }
                y1 = fmaf(a.wL, l1, a.wG * fq * y1);
                y2 = fmaf(a.wL, l2, a.wG * fq * y2);
                a.soft[(size_t)s * a.K + k] = make_float2(y1, y2);
                if (a.hard) a.hard[(size_t)s * a.K + k] = (uint8_t)((y1 < 0.f ? 1 : 0) | (y2 < 0.f ? 2 : 0));
            }
        }
    }
    if (!ok && (tid == 0 || tid == 128)) report(a.status, APSM_ERR_TIMEOUT);
    gt0 += n_tiles;
    // every thread is done with this item (its MMAs were all waited for by the epilogue) before
    // the next item's query operand is written; a CTA whose wait ran out stops taking items
    if (__syncthreads_or(!ok)) break;
    }

    // ---- teardown: every MMA has been waited for by the epilogue (or timed out) ----------------
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}


template <int M, int KB, int kPrec>
cudaError_t launch_detect_tc_batch(const TcBatchArgs &ba, int grid, cudaStream_t stream) {
    using L = TcSmem<M, KB, kPrec>;
    if (grid <= 0 || ba.n_items <= 0) return cudaSuccess;
    auto fn = detect_tc_batch_kernel<M, KB, kPrec>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes);
    if (e != cudaSuccess) return e;
    fn<<<grid, kTcThreads, L::kBytes, stream>>>(ba);  // ordinary launch, as detect_tc_kernel
    return cudaGetLastError();
}

// resident CTAs per SM of one instantiation (its shared-memory footprint decides)
template <int M, int KB, int kPrec>
int tc_batch_ctas_per_sm() { return tc_min_blocks<M, KB, kPrec>(); }

using TcBatchLauncher = cudaError_t (*)(const TcBatchArgs &, int, cudaStream_t);

}  // namespace apsm
