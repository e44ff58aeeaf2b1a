// detect_tc.cuh -- detection with the complex dist-Gram on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in TMEM).  Same result as detect_f32.cuh (Sec. III-B detection).
//
// For a tile of 128 queries and E dictionary entries the Gram is one GEMM
//   C[s][2e]   = <q_s, [Re r_t; Im r_t]>  = Re z,   C[s][2e+1] = <q_s, [-Im r_t; Re r_t]> = Im z,
// with q_s = 2 k2 [Re r_s; Im r_s] (the factor of the exponent pre-applied), z = r_t^H r_s.
// The epilogue (one thread per query row, reading its row of C from TMEM with tcgen05.ld) forms
//   E_A = 2^(C[s][2e] - k2 n_t),  E_B = 2^(C[s][2e+1] - k2 n_t),  E_C = 2^(-C[s][2e+1] - k2 n_t)
// and multiplies the sums by the query factor 2^(-k2 n_s) at the end (see detect_f32.cuh for the
// factorisation).  Every such term is at most 2^(k2 n_s), so while k2 n_s <= kFactorLimit for
// all queries of the CTA nothing leaves the FP32 range; a CTA holding a query outside that
// range adds -k2 n_s inside the exponent instead (the unfactored exponent).
//
// Precision (template kPrec):
//   kTF32x3  FP32 accuracy from three TF32 products per k-step: hi*hi + hi*lo + lo*hi, with
//            hi = tf32(x), lo = tf32(x - hi) (relative error of the Gram ~2^-21);
//   kHalf    one BF16 or FP16 product per k-step (runtime choice), FP32 accumulation.
//
// Hard decisions here are QPSK (sign test); square-QAM labels are formed from the soft outputs by
// a separate pass (apsm_api.cu), so that this loop compiles the same for every modulation.
//
// Roles (256 threads): warps 0-3 = epilogue (query row = thread; coefficient sums over user
// pairs with packed f32x2 FMAs), warps 4-7 = converters (entry rows of B by whole 16-byte core
// rows where M allows, the tile's coefficients and norms; thread 128 issues the MMAs; the next
// tile's global loads are issued before the wait for its stage).  Two smem stages of
// B / coefficients and two TMEM accumulators: the converters and the tensor core work on
// tile i+1 while the epilogue reads tile i.  All waits are bounded.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "apsm_common.cuh"
#include "detect_f32.cuh"

namespace apsm {

enum TcPrec { kTF32x3 = 0, kHalf = 1 };

constexpr int kTcRows = 128;     // queries per CTA (MMA M)
constexpr int kTcEntries = 64;   // entries per tile (MMA N = 2 * kTcEntries)
constexpr int kTcThreads = 256;

// Cancellation-guard thresholds theta of the per-pair direct-difference fallback (relative to
// k2 (n_s + n_t)): 2^-4 for a BF16/FP16 Gram, 2^-12 for the TF32 x3 Gram.
constexpr float kGuardHalf = 0.0625f;
constexpr float kGuardF32 = 1.f / 4096.f;

struct TcArgs {
    const float2 *rx;         // [N][M]
    int N;
    const float2 *dict;       // [A][M]
    const float *dict_norm;   // [A]
    const float *gamma;       // [A][2][K]
    const float2 *clin;       // [M][K]
    const int *meta;          // meta[0] = entries held
    int n_entries;            // host bound
    int K;                    // users (<= KB)
    int half_fmt;             // kHalf only: 1 = BF16, 0 = FP16
    float k2, wL, wG;
    float2 *soft;             // [N][K]
    uint8_t *hard;            // [N][K] nullable
    int *status;
};

// Operand layout: K-major, no swizzle; core matrix = 8 rows x 16 bytes.  KD = contraction
// length padded to the MMA k-step; SBO = bytes per 8-row group; LBO = 128 (adjacent k cores).
template <int M, int kPrec>
struct TcShape {
    static constexpr int kEl = kPrec == kTF32x3 ? 4 : 2;           // bytes per element
    static constexpr int kStep = kPrec == kTF32x3 ? 8 : 16;        // MMA K per instruction
    static constexpr int KD = round_up(2 * M, kStep);
    static constexpr int kCoreK = 16 / kEl;                        // elements per core row
    static constexpr int SBO = (KD / kCoreK) * 128;
    static constexpr int kRowsB = 2 * kTcEntries;
    static constexpr int kBytesA = kTcRows / 8 * SBO;              // one operand copy
    static constexpr int kBytesB = kRowsB / 8 * SBO;
    static constexpr int kCopies = kPrec == kTF32x3 ? 2 : 1;       // hi (+ lo)
    static constexpr int kSteps = KD / kStep;
    __device__ static constexpr int off(int r, int k) {
        return (r / 8) * SBO + (k / kCoreK) * 128 + (r % 8) * 16 + (k % kCoreK) * kEl;
    }
};

template <int M, int KB, int kPrec>
struct TcSmem {
    using Sh = TcShape<M, kPrec>;
    static constexpr int kA = 0;                                       // A copies
    static constexpr int kB = kA + Sh::kCopies * Sh::kBytesA;          // 2 stages x B copies
    static constexpr int kG = kB + 2 * Sh::kCopies * Sh::kBytesB;      // 2 stages x [E][2KB] coefficients
    static constexpr int kN = kG + 2 * kTcEntries * 2 * KB * 4;        // 2 stages x [E] -k2 n_t
    static constexpr int kBar = round_up(kN + 2 * kTcEntries * 4, 16); // 4 mbarriers
    static constexpr int kTmem = kBar + 32;
    static constexpr int kBytes = kTmem + 16;
};

__device__ __forceinline__ uint64_t umma_sdesc(uint32_t addr, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;  // leading byte offset (adjacent k cores)
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;   // stride byte offset (8-row groups)
    d |= (uint64_t)1 << 46;                       // descriptor version; no swizzle
    return d;
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t y;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void umma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_f16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Packed FP32 pair add: (x0, x1) += b, each lane one IEEE add.
__device__ __forceinline__ void add2_bcast(float &x0, float &x1, float b) {
    asm("{\n\t.reg .b64 x, b;\n\t"
        "mov.b64 x, {%0, %1};\n\tmov.b64 b, {%2, %2};\n\t"
        "add.rn.f32x2 x, x, b;\n\tmov.b64 {%0, %1}, x;\n\t}"
        : "+f"(x0), "+f"(x1)
        : "f"(b));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Writes one operand element (value x) at byte offset `off` of every operand copy.
template <int kPrec>
__device__ __forceinline__ void put_elem(unsigned char *base, int copy_bytes, int off, float x, int half_fmt) {
    if constexpr (kPrec == kTF32x3) {
        const uint32_t hi = tf32_rna(x);
        const uint32_t lo = tf32_rna(x - __uint_as_float(hi));
        *reinterpret_cast<uint32_t *>(base + off) = hi;
        *reinterpret_cast<uint32_t *>(base + copy_bytes + off) = lo;
    } else {
        uint16_t h;
        if (half_fmt) {
            const __nv_bfloat16 b = __float2bfloat16_rn(x);
            h = *reinterpret_cast<const uint16_t *>(&b);
        } else {
            const __half b = __float2half_rn(x);
            h = *reinterpret_cast<const uint16_t *>(&b);
        }
        *reinterpret_cast<uint16_t *>(base + off) = h;
    }
}

// Writes one 16-byte core row (TcShape::kCoreK consecutive elements x[]) at byte offset `off` of
// every operand copy: packed BF16/FP16 pairs, or TF32 hi and lo words.
template <int kPrec, int C>
__device__ __forceinline__ void put_core(unsigned char *base, int copy_bytes, int off, const float (&x)[C],
                                         int half_fmt) {
    if constexpr (kPrec == kTF32x3) {
        static_assert(C == 4, "a TF32 core row holds four elements");
        uint4 hi, lo;
        uint32_t *h = &hi.x, *l = &lo.x;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            h[c] = tf32_rna(x[c]);
            l[c] = tf32_rna(x[c] - __uint_as_float(h[c]));
        }
        *reinterpret_cast<uint4 *>(base + off) = hi;
        *reinterpret_cast<uint4 *>(base + copy_bytes + off) = lo;
    } else {
        static_assert(C == 8, "a 16-bit core row holds eight elements");
        uint4 v;
        uint32_t *p = &v.x;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (half_fmt) {
                const __nv_bfloat162 b = __floats2bfloat162_rn(x[2 * c], x[2 * c + 1]);
                p[c] = *reinterpret_cast<const uint32_t *>(&b);
            } else {
                const __half2 b = __floats2half2_rn(x[2 * c], x[2 * c + 1]);
                p[c] = *reinterpret_cast<const uint32_t *>(&b);
            }
        }
        *reinterpret_cast<uint4 *>(base + off) = v;
    }
}

// Whole core rows can be written when a core row never straddles the real and imaginary halves
// and the contraction needs no padding (M a multiple of the elements per core row).
template <int M, int kPrec>
constexpr bool tc_core_rows() {
    using Sh = TcShape<M, kPrec>;
    return M % Sh::kCoreK == 0 && Sh::KD == 2 * M;
}

// The entry operand of one tile by whole core rows.  Task = (entry e, half h, piece p): B row
// 2e+h at k = p C.. and k = M + p C.. from the C complex values r_t[p C .. p C + C), i.e.
//   row 2e: [Re | Im],  row 2e+1: [-Im | Re].
// The eight lanes of a quarter-warp take the same piece of four consecutive entries (both
// halves), i.e. eight consecutive B rows, so their 16-byte stores hit all 32 banks once.
// The first PF tasks' global loads can be issued ahead (prefetch), before the converters wait
// for the stage they will write, so that their L2 latency overlaps the wait.
template <int M, int kPrec, int kMaxPf = 8>
struct EntryRows {
    using Sh = TcShape<M, kPrec>;
    // (instantiated for every M; used only where tc_core_rows<M, kPrec>() holds, so that P >= 1)
    static constexpr int C = Sh::kCoreK, P = M / C > 0 ? M / C : 1, V = C / 2;  // float4 loads per task
    static constexpr int PF = P * V <= kMaxPf ? P : kMaxPf / V;                // prefetched tasks (<= kMaxPf float4)
    float4 pf[PF][V];

    // task i of thread ct: 64 entries x 2 halves x P pieces over 128 threads
    __device__ __forceinline__ static void task(int ct, int i, int &e, int &h, int &p) {
        const int lane = ct & 31, w = ct >> 5;
        const int R = (lane >> 3) + 4 * (w + 4 * i);  // [0, 16 P): (entry group of 4, piece)
        h = lane & 1;
        p = R % P;
        e = 4 * (R / P) + ((lane >> 1) & 3);
    }
    __device__ __forceinline__ static void load(const float2 *__restrict__ dict, int t, int n_ent, int p,
                                                float4 (&v)[V]) {
        if (t < n_ent) {
            const float4 *src = reinterpret_cast<const float4 *>(dict + (size_t)t * M + p * C);
#pragma unroll
            for (int q = 0; q < V; ++q) v[q] = __ldg(src + q);
        } else {
#pragma unroll
            for (int q = 0; q < V; ++q) v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __device__ __forceinline__ void prefetch(const float2 *__restrict__ dict, int e0, int n_ent, int ct) {
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            int e, h, p;
            task(ct, i, e, h, p);
            load(dict, e0 + e, n_ent, p, pf[i]);
        }
    }
    __device__ __forceinline__ static void put(unsigned char *bst, int e, int h, int p, const float4 (&v)[V],
                                               int half_fmt) {
        float x0[C], x1[C];
#pragma unroll
        for (int q = 0; q < V; ++q) {
            // v[q] = (Re, Im) of two consecutive antennas
            x0[2 * q] = h ? -v[q].y : v[q].x;
            x0[2 * q + 1] = h ? -v[q].w : v[q].z;
            x1[2 * q] = h ? v[q].x : v[q].y;
            x1[2 * q + 1] = h ? v[q].z : v[q].w;
        }
        const int r = 2 * e + h;
        put_core<kPrec, C>(bst, Sh::kBytesB, Sh::off(r, p * C), x0, half_fmt);
        put_core<kPrec, C>(bst, Sh::kBytesB, Sh::off(r, M + p * C), x1, half_fmt);
    }
    __device__ __forceinline__ void write(unsigned char *bst, const float2 *__restrict__ dict, int e0, int n_ent,
                                          int ct, int half_fmt) const {
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            int e, h, p;
            task(ct, i, e, h, p);
            put(bst, e, h, p, pf[i], half_fmt);
        }
#pragma unroll 1
        for (int i = PF; i < P; ++i) {
            int e, h, p;
            task(ct, i, e, h, p);
            float4 v[V];
            load(dict, e0 + e, n_ent, p, v);
            put(bst, e, h, p, v, half_fmt);
        }
    }
};

__device__ __forceinline__ bool converters_and(bool v) {
    // AND over the 128 converter threads (named barrier 1)
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

// two CTAs per SM where the shared memory allows it (registers are then capped accordingly)
template <int M, int KB, int kPrec>
constexpr int tc_min_blocks() { return TcSmem<M, KB, kPrec>::kBytes <= 113 * 1024 ? 2 : 1; }

template <int M, int KB, int kPrec>
__global__ void __launch_bounds__(kTcThreads, (tc_min_blocks<M, KB, kPrec>())) detect_tc_kernel(const TcArgs a) {
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
    constexpr int E = kTcEntries, NB = 2 * kTcEntries;
    constexpr uint32_t kCols = 2 * NB;  // two accumulators of NB fp32 columns

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
        fence_mbar_init();
    }
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
                put_core<kPrec, C>(sA, Sh::kBytesA, Sh::off(tid, p * C), re, a.half_fmt);
                put_core<kPrec, C>(sA, Sh::kBytesA, Sh::off(tid, M + p * C), im, a.half_fmt);
            }
        } else {
            for (int m = 0; m < M; ++m) {
                const float2 v = s < a.N ? __ldg(rq + m) : make_float2(0.f, 0.f);
                nq = fmaf(v.x, v.x, fmaf(v.y, v.y, nq));
                put_elem<kPrec>(sA, Sh::kBytesA, Sh::off(tid, m), g2 * v.x, a.half_fmt);
                put_elem<kPrec>(sA, Sh::kBytesA, Sh::off(tid, M + m), g2 * v.y, a.half_fmt);
            }
            for (int k = 2 * M; k < Sh::KD; ++k) put_elem<kPrec>(sA, Sh::kBytesA, Sh::off(tid, k), 0.f, a.half_fmt);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    const bool cta_in_range = __syncthreads_and(warp >= 4 || a.k2 * nq <= kFactorLimit);
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    uint32_t idesc;
    if constexpr (kPrec == kTF32x3) {
        idesc = (1u << 4) | (2u << 7) | (2u << 10);  // F32 accumulate, TF32 A and B, K-major
    } else {
        const uint32_t f = a.half_fmt ? 1u : 0u;    // BF16 (1) or FP16 (0)
        idesc = (1u << 4) | (f << 7) | (f << 10);
    }
    idesc |= ((uint32_t)(NB >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);

    bool ok = true;
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
            const int st = tile & 1;
            // the epilogue of tile-2 has released stage st (TMEM accumulator, coefficients), and
            // it waited for the MMAs of tile-2, the last readers of B stage st
            bool w = true;
            if (tile >= 2) w = mbar_wait_bounded(&epi_done[st], ((tile - 2) >> 1) & 1);
            if (!converters_and(w)) {
                ok = false;
                break;
            }
            const int e0 = tile * E;
            unsigned char *bst = sB + st * Sh::kCopies * Sh::kBytesB;
            if constexpr (tc_core_rows<M, kPrec>()) {
                rows.write(bst, a.dict, e0, n_ent, ct, a.half_fmt);
            } else {
                const int t = e0 + (ct >> 1), h = ct & 1;
                const float2 *rt = a.dict + (size_t)t * M;
                // row 2e: [Re r_t; Im r_t] gives Re z;  row 2e+1: [-Im r_t; Re r_t] gives Im z
                for (int m = 0; m < M; ++m) {
                    const float2 v = t < n_ent ? __ldg(rt + m) : make_float2(0.f, 0.f);
                    put_elem<kPrec>(bst, Sh::kBytesB, Sh::off(ct, m), h ? -v.y : v.x, a.half_fmt);
                    put_elem<kPrec>(bst, Sh::kBytesB, Sh::off(ct, M + m), h ? v.x : v.y, a.half_fmt);
                }
                for (int k = 2 * M; k < Sh::KD; ++k) put_elem<kPrec>(bst, Sh::kBytesB, Sh::off(ct, k), 0.f, a.half_fmt);
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
                const int st = tile & 1;
                // warp-uniform decision: tcgen05.ld below is executed by whole warps only
                if (!__all_sync(0xffffffffu, mbar_wait_bounded(&mma_done[st], (tile >> 1) & 1))) {
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

    // ---- teardown: every MMA has been waited for by the epilogue (or timed out) ----------------
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

template <int M, int KB, int kPrec>
cudaError_t launch_detect_tc(const TcArgs &a, cudaStream_t stream) {
    using L = TcSmem<M, KB, kPrec>;
    const int grid = (a.N + kTcRows - 1) / kTcRows;
    if (grid == 0) return cudaSuccess;
    auto fn = detect_tc_kernel<M, KB, kPrec>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes);
    if (e != cudaSuccess) return e;
    // An ordinary launch (not a programmatic dependent one): the kernel starts only after the
    // previous work of the stream has finished, so every read (dictionary tiles, which both CTAs
    // of an SM share, and the linear filter, read per query row) may take the L1 path; an early
    // launch would have to take them through L2 (see launch_pdl).
    fn<<<grid, kTcThreads, L::kBytes, stream>>>(a);
    return cudaGetLastError();
}

using TcLauncher = cudaError_t (*)(const TcArgs &, cudaStream_t);

}  // namespace apsm
