// train_f32.cuh -- FP32 APSM training kernels (Eq. apsm, Eq. beta, window J_n of Sec. II-D;
// Sec. III-B training).
//
// The recurrence runs over the 2P real-split samples n = 2t + l, in chunks of T pilots.
// For chunk c (pilots [t0, t0+Tc), samples [s0, s1)) every sample that can be touched in the
// chunk lies in the live range L = [l0, s1), l0 = max(0, s0 - W + 1) rounded down to a pilot
// boundary: the window samples carried from the previous chunk plus the chunk's own.  Each
// sample m in L keeps a running prediction p_m = f_n(x_m) of the current filter.  Because f is
// linear in its coefficients,
//   f_{n+1}(x_m) = f_n(x_m) + mu q sum_{i in J_n} beta_i kappa(x_i, x_m)          (Eq. apsm)
// exactly, so one step needs only the window's residuals, its betas (Eq. beta) and the
// kernel values kappa(x_i, x_m) between samples of L; dropping a dictionary entry subtracts its
// Gaussian terms.
//
// The chunk's new samples enter with f at the chunk start.  Split the dictionary at the start of
// chunk c+1 into the entries of chunk c's live range and the older ("frozen") ones, whose
// coefficients no longer change after chunk c-1.  Phase B of chunk c tracks the first part for
// the next chunk's samples as it goes (the same incremental identity, applied once per step
// block from the block's summed coefficient changes); the frozen part is the detection kernel
// in partial mode over those entries only (phase A), launched before chunk c's phase B and run
// on other SMs at the same time.  When tracking is not available (single-warp live range, or
// windows above 24) phase A covers the whole dictionary and runs between the chunks.
//
// Kernels:
//   train_gram_kernel   kappa(x_u, x_v) for all u, v in L of every chunk (sum kernel, Fact 1),
//                       kappa_G between each entry dropped during a chunk and L, and kappa
//                       between L and the next chunk's samples.
//   train_chunk_kernel  phase B of one chunk.
#pragma once

#include <type_traits>

#include "apsm_common.cuh"

namespace apsm {

struct TrainGeom {
    int M, K, W, D;
    int P;         // pilots of the extended sequence: nc0 carried + the call's new vectors
    int nc0;       // pilots carried over from the previous call (the window reaches into them)
    int t_base;    // running index of extended pilot 0 (vectors trained on before it)
    int evict;     // FIFO eviction can occur in this call (t_base + P > D, or unknown)
    int T;         // pilots per chunk
    int n_chunks;
    int RMAX;      // 2T + W: live-range capacity
    int RS;        // row stride of the per-chunk kernel tables: RMAX rounded up to 32
    int WP;        // window W rounded up to a supported multiple of 4
    int slice;     // entries per phase-A slice
    int KXS;       // row stride of the next-chunk table: 2T rounded up to 32
    int track;     // phase B tracks the next chunk's samples (phase A then covers frozen entries)
};

// first sample of the live range of a chunk starting at sample s0 (a pilot boundary)
__host__ __device__ inline int live_start(int s0, int W) { return max(0, s0 - W + 1) & ~1; }

// Chunk c covers extended pilots [t0, t0 + Tc), after the nc0 carried ones.
__host__ __device__ inline void chunk_range(const TrainGeom &g, int c, int &t0, int &Tc, int &s0, int &s1,
                                            int &l0) {
    t0 = g.nc0 + c * g.T;
    Tc = min(g.T, g.P - t0);
    s0 = 2 * t0;
    s1 = 2 * (t0 + Tc);
    l0 = live_start(s0, g.W);
}

// Real-split inner product and squared distance between sample (a, la) and sample (b, lb),
// a, b pilot indices, la, lb in {0: r1, 1: r2}, from one complex inner product z = r_a^H r_b:
//   r1(a).r1(b) = r2(a).r2(b) = Re z,  r1(a).r2(b) = Im z,  r2(a).r1(b) = -Im z,
//   ||x_a - x_b||^2 = ||r_a||^2 + ||r_b||^2 - 2 x_a.x_b.
__device__ inline void sample_pair(const float2 *ra, const float2 *rb, int M, int la, int lb, float &dot,
                                   float &dist2) {
    float zr = 0.f, zi = 0.f, na = 0.f, nb = 0.f;
    for (int m = 0; m < M; ++m) {
        const float2 x = __ldg(ra + m), y = __ldg(rb + m);
        zr = fmaf(x.x, y.x, fmaf(x.y, y.y, zr));
        zi = fmaf(x.x, y.y, fmaf(-x.y, y.x, zi));
        na = fmaf(x.x, x.x, fmaf(x.y, x.y, na));
        nb = fmaf(y.x, y.x, fmaf(y.y, y.y, nb));
    }
    dot = (la == lb) ? zr : (la == 0 ? zi : -zi);
    dist2 = fmaxf(na + nb - 2.f * dot, 0.f);
}

// Tables per chunk c (zero outside the live range):
//   kmat[c][u][v] = kappa(x_{l0+u}, x_{l0+v})                       u, v < R        (stride RS)
//   gev[c][e][l][v] = kappa_G(x_{2(t0+e-D)+l}, x_{l0+v})            entry t0+e-D dropped at n = 2(t0+e)
//   kx[c][u][v] = kappa(x_{l0+u}, x_{s1+v})                         v < next chunk's 2Tc (stride KXS)
// (train_gram_kernel, defined in train_chunk.cu; kx only when g.track).
// Pilot vectors come from the extended sequence rx; an entry dropped during the call that was
// trained on before it (running index < t_base) is read from its dictionary slot.
cudaError_t launch_train_gram(const float2 *rx, const float2 *dict, const TrainGeom &g, float k2, float wL, float wG,
                              float *kmat, float *gev, float *kx, cudaStream_t stream);

struct ChunkArgs {
    TrainGeom g;
    int chunk;
    float mu, eps, wL, wG;
    const float2 *rx;       // [P][M] extended sequence (carried pilots, then the new ones)
    float2 *sym;            // [P][K] its targets (decision-directed: decided ones written back)
    float2 *dict;           // [A][M]
    float *dict_norm;       // [A]
    float *gamma;           // [A][2][K]
    float2 *clin;           // [M][K]
    int *meta;              // [4]
    const float *kmat;      // [n_chunks][RS][RS]
    const float *gev;       // [n_chunks][T][2][RS]
    const float *partial;   // [n_slices][part_rows][2K]: rows = pilots part_p0, part_p0 + 1, ..
    int n_slices;
    int part_p0, part_rows;
    int fresh_carry;        // carried samples start from phase A (first chunk of a continuation)
    float *carry;           // [W][K]
    int8_t *case_log;       // [2 (P - nc0)][W][K] nullable
    float *target;          // state: [A][K] complex targets of the held entries
    float *soft_out;        // [P - nc0][K] complex output at arrival, nullable
    uint8_t *hard_out;      // [P - nc0][K] labels of the targets, nullable
    int decide;             // targets of the new samples are decided at arrival
    int qviol;              // weights q_j = 1/|V_n| on the violated slabs
    int qam_half;           // slicer: bits per axis and amplitude unit
    float qam_a;
    const float *kx;        // [RS][KXS] of this chunk (tracking)
    const float *track_in;  // [2T][K]: tracked part of f at this chunk's start, at its samples
    float *track_out;       // [2T][K]: the same for the next chunk (null: no tracking)
    // When this launch waits for the previous one (programmatic dependent launch):
    // 0: first thing; 1: after staging the kernel tables and pilots (tracked form: the previous
    // launch is the frozen-entry phase A of this chunk, which completes after the previous chunk's
    // phase B); 2: after staging everything but the phase-A sums (the previous launch is this
    // chunk's whole-dictionary phase A, launched after the previous phase B had completed)
    int pdl_mode;
};

// Shared-memory layout of phase B (bytes; every region 16-byte aligned).
struct ChunkSmem {
    int bar, kmat, gev, egam, beta, dg, tgt, clin, pil, trk, bytes;
    __host__ __device__ ChunkSmem(const TrainGeom &g) {
        const int RS = g.RS;
        const int npil = g.T + (g.W + 1) / 2 + 1;
        bar = 0;
        kmat = 16;                                   // WP zero rows, then RS rows of RS
        gev = kmat + (g.WP + RS) * RS * 4;
        egam = gev + (g.evict ? g.T * 2 * RS * 4 : 0);     // dropped-entry table only with eviction
        beta = egam + round_up(g.T * 2 * 4, 16);
        dg = beta + (4 * RS + 2 * g.WP + 224) * 4;  // beta ring, or p / gamma / b / 1/kappa + rings + mu q tables
        tgt = dg + RS * 4;                          // final targets of the live range
        clin = tgt + RS * 4;
        pil = clin + round_up(g.M * 8, 16);
        trk = pil + npil * g.M * 8;                   // carried coefficients [32], reduced filter [M]
        bytes = trk + (g.track ? 32 * 4 + g.M * 8 : 0);
    }
};

constexpr int kRingMax = 32;  // windows up to this padded size keep their kernel column in registers
constexpr int kBlockMin = 8;  // shortest step block of the blocked form (padded windows up to 24)

// Phase B of one chunk for one user (blockIdx.x = k).  Thread u owns live-range sample u
// (RS = 32 S threads); a step is one CTA barrier: window threads publish their beta, then every
// thread adds the window's contribution to its own prediction.  WP is the window rounded up to a
// multiple of 4; the WP slots below the window hold zero so the sum has a fixed length.
// kExt: the instantiation that also serves violated-slab weights, outputs at arrival and
// decision-directed targets; the plain one (kExt = false) compiles none of that into its step
// loops, which keeps the recurrence's code as small as the method itself needs.
template <int S, int WP, bool kExt>
__global__ void __launch_bounds__(32 * S, 1) train_chunk_kernel(const ChunkArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int RS = 32 * S;
    if (a.pdl_mode == 0) {
        pdl_wait();
        pdl_trigger();
    }
    const TrainGeom &g = a.g;
    const ChunkSmem L(g);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar);
    float *s_kmat = reinterpret_cast<float *>(smem + L.kmat) + WP * RS;  // row 0 after WP zero rows
    float *s_gev = reinterpret_cast<float *>(smem + L.gev);
    float *s_egam = reinterpret_cast<float *>(smem + L.egam);
    float *s_beta = reinterpret_cast<float *>(smem + L.beta);
    float *s_dg = reinterpret_cast<float *>(smem + L.dg);
    float *s_tgt = reinterpret_cast<float *>(smem + L.tgt);
    float2 *s_clin = reinterpret_cast<float2 *>(smem + L.clin);
    float2 *s_pil = reinterpret_cast<float2 *>(smem + L.pil);
    float *s_gcar = reinterpret_cast<float *>(smem + L.trk);             // carried gamma at chunk start
    float2 *s_clinw = reinterpret_cast<float2 *>(smem + L.trk + 32 * 4);  // filter minus carried terms

    const int M = g.M, K = g.K, W = g.W, D = g.D;
    int t0, Tc, s0, s1, l0;
    chunk_range(g, a.chunk, t0, Tc, s0, s1, l0);
    const int R = s1 - l0;
    const int pa0 = l0 >> 1;  // first pilot touching L
    const int npil = t0 + Tc - pa0;
    const int k = blockIdx.x;  // user
    const int u = threadIdx.x;  // live-range sample of this thread
    const int tb = g.t_base;    // running index = tb + extended pilot index; its slot is that mod D
    const int sb = 2 * tb;      // running index of extended sample 0
    const int n_first = 2 * g.nc0;  // first sample this call trains on (case log / outputs index from it)
    const bool evict = (tb + t0 + Tc - 1) >= D;

    // ---- stage the chunk's kernel tables and pilots with the bulk-copy engine ---------------
    if (u == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        const uint32_t kb = (uint32_t)R * RS * 4, gb = evict ? (uint32_t)Tc * 2 * RS * 4 : 0u,
                       pb = (uint32_t)npil * M * 8;
        mbar_arrive_expect_tx(bar, kb + gb + pb);
        bulk_g2s(s_kmat, a.kmat + (size_t)a.chunk * RS * RS, kb, bar);
        if (evict) bulk_g2s(s_gev, a.gev + (size_t)a.chunk * g.T * 2 * RS, gb, bar);
        bulk_g2s(s_pil, a.rx + (size_t)pa0 * M, pb, bar);
    }
    __syncthreads();  // the barrier's initialisation is visible before any thread waits on it
    const bool valid = u < R;
    const int m = l0 + u, pa = m >> 1, l = m & 1;
    // targets: given ones are read at once; decided ones only after the wait below (the previous
    // chunk decides the carried samples' targets)
    float b = 0.f;
    auto read_target = [&]() {
        if (valid) {
            const float2 sy = __ldcg(a.sym + (size_t)pa * K + k);
            b = l ? sy.y : sy.x;  // b_{2t} = Re b(t), b_{2t+1} = Im b(t)
        }
    };
    if (!a.decide) read_target();
    for (int i = u; i < 2 * (WP + RS); i += RS) s_beta[i] = 0.f;
    for (int i = u; i < WP * RS; i += RS) s_kmat[i - WP * RS] = 0.f;
    float rk = 0.f;  // 1 / kappa(x_j, x_j)
    // Every thread reaches this wait; the CTA votes on its outcome so that either all threads
    // go on or all leave together (no thread may skip a later barrier the others wait at).
    auto tables_ready = [&]() {
        if (!__syncthreads_and(mbar_wait_bounded(bar, 0))) {
            if (u == 0) report(a.meta + 3, APSM_ERR_TIMEOUT);
            return false;
        }
        if (valid) {
            const float kjj = s_kmat[u * RS + u];
            rk = kjj != 0.f ? 1.f / kjj : 0.f;
        }
        return true;
    };
    if (a.pdl_mode == 1) {  // the staged tables do not depend on the previous chunk
        if (!tables_ready()) return;
        pdl_wait();
        pdl_trigger();
    }
    // every global load of the prologue is issued before the first use (one round trip)
    if (a.decide) read_target();
    float2 clin_r[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};  // M <= 64 <= 2 RS
#pragma unroll
    for (int i = 0; i < 2; ++i)
        if (u + i * RS < M) clin_r[i] = __ldcg(a.clin + (u + i * RS) * K + k);
    // coefficients of the entries dropped in this chunk (entry t0+e-D at step 2(t0+e))
    // (the dropped entry and the arriving one share the slot (tb + t0 + e) mod D)
    float egam_r = 0.f;
    if (evict && u < 2 * Tc && tb + t0 + (u >> 1) >= D)
        egam_r = __ldcg(a.gamma + ((size_t)((tb + t0 + (u >> 1)) % D) * 2 + (u & 1)) * K + k);

    // ---- this thread's sample: target, coefficient, prediction at chunk start ---------------
    float p = 0.f, gam = 0.f;
    if (valid) {
        if (m < s0) {
            if (!a.fresh_carry) p = __ldcg(a.carry + u * K + k);
            gam = __ldcg(a.gamma + ((size_t)((tb + pa) % D) * 2 + l) * K + k);
        } else if (a.track_in) {
            p = __ldcg(a.track_in + (m - s0) * K + k);
        }
    }
    const float gam0 = gam;
#pragma unroll
    for (int i = 0; i < 2; ++i)
        if (u + i * RS < M) s_clin[u + i * RS] = clin_r[i];
    if (evict && u < 2 * Tc) s_egam[u] = egam_r;
    // carried gamma at the chunk start (zero past the carried samples), for the tracking threads
    const bool track = a.track_out != nullptr;  // (the region exists only in the tracked form)
    if (track && u < 32) s_gcar[u] = (valid && m < s0) ? gam : 0.f;
    __syncthreads();
    if (a.pdl_mode != 1 && !tables_ready()) return;
    // samples whose prediction starts from phase A: the chunk's new ones (untracked form), and
    // in the first chunk of a continuation also the carried ones
    const bool from_a = valid && ((m >= s0 && !a.track_in) || (m < s0 && a.fresh_carry));
    if (from_a) {  // linear part w_L <w, x_m> = w_L Re / Im (c^H r) at chunk start
        // each pilot starts at its own antenna so the lanes of a warp hit distinct banks
        const float2 *rv = s_pil + (pa - pa0) * M;
        float lin0 = 0.f, lin1 = 0.f;
        int mm = pa % M;
        for (int i = 0; i < M; i += 2) {
            const int mb = mm + 1 == M ? 0 : mm + 1;
            const float2 c = s_clin[mm], x = rv[mm], cb = s_clin[mb], xb = rv[mb];
            lin0 = l ? fmaf(c.x, x.y, fmaf(-c.y, x.x, lin0)) : fmaf(c.x, x.x, fmaf(c.y, x.y, lin0));
            lin1 = l ? fmaf(cb.x, xb.y, fmaf(-cb.y, xb.x, lin1)) : fmaf(cb.x, xb.x, fmaf(cb.y, xb.y, lin1));
            mm = mb + 1 == M ? 0 : mb + 1;
        }
        p = a.wL * (lin0 + lin1);
    }
    // In mode 2 everything above reads only what the previous chunk's phase B (complete before
    // this kernel could launch) and the kernel tables wrote; the phase-A sums need phase A itself.
    if (a.pdl_mode == 2) {
        pdl_wait();
        pdl_trigger();
    }
    if (valid && (m >= s0 || a.fresh_carry)) {
        // Gaussian part of f_{s0}(x_m) from the phase-A slices: 32 loads in flight at a time,
        // summed into eight partial sums (slice i into sum i mod 8) combined in a fixed order
        const float *src = a.partial + (size_t)(pa - a.part_p0) * 2 * K + l * K + k;
        const size_t stride = (size_t)a.part_rows * 2 * K;
        float gs[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int sl = 0; sl < a.n_slices; sl += 32) {
            float v[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = sl + j < a.n_slices ? __ldcg(src + (sl + j) * stride) : 0.f;
#pragma unroll
            for (int j = 0; j < 32; ++j) gs[j & 7] += v[j];
        }
        p = fmaf(a.wG, ((gs[0] + gs[1]) + (gs[2] + gs[3])) + ((gs[4] + gs[5]) + (gs[6] + gs[7])), p);
    }
    const int nc = s0 - l0;  // carried samples (rows 0 .. nc-1 of the tables)

    // ---- the recurrence over the chunk's samples -----------------------------------------------
    // Blocked form with more than one warp: the idle warps also accumulate the filter change
    // c_k += sum_j dgamma_j x~_j block by block (thread = antenna x part of the block's lanes).
    constexpr bool kBlocked = WP + kBlockMin - 1 <= 32;
    constexpr bool kDcInRegs = kBlocked && S > 1;
    const int ntr = RS - 32, tu = u - 32;
    const int dc_parts = max(1, ntr / M);
    float dcx[2] = {0.f, 0.f}, dcy[2] = {0.f, 0.f};
    const bool log_cases = a.case_log != nullptr;
    const float muq_full = a.mu / (float)W;  // mu q with q = 1/W once the window is full
    const float *kcol = s_kmat + u;          // column u of the kernel table
    if constexpr (kBlocked) {
        // Blocked form.  Over a block of B = 32 - WP steps from n0, every sample that is in a
        // window of the block lies in [n0 - WP + 1, n0 + B - 1]: 31 samples, one per lane of warp 0.
        // That warp runs the B steps alone: the window lanes compute mu q beta (Eq. beta, written
        // as beta = clamp(p, b - eps, b + eps) - p over kappa_jj), publish it in a 32-float ring and
        // every lane adds the window sum to its own prediction with the kernel values held in
        // registers; one warp barrier per step.  Since kappa(x_j, x_m) does not depend on the step,
        // the block then moves every later sample m >= n0 + B by
        //   sum_j kappa(x_j, x_m) sum_{n in block} mu q_n beta_j(n)
        // at once: the lanes publish their summed updates and all threads apply them.
        constexpr int B = 32 - WP;
        constexpr int NL = WP + B - 1;
        float *s_p = s_beta, *s_g = s_p + RS, *s_b = s_g + RS, *s_rk = s_b + RS, *s_agg = s_rk + RS;  // [2][32]
        float *s_w = s_agg + 64, *s_muq = s_w + 64;
        if (valid) {
            s_p[u] = p;
            s_g[u] = gam;
            s_b[u] = b;
            s_rk[u] = rk;
        }
        float *s_muqv = s_muq + 32;
        if (u < 32) {
            s_muq[u] = a.mu / (float)(u + 1);                 // mu q while the window is filling (n < W - 1)
            s_muqv[u] = u == 0 ? 0.f : a.mu / (float)u;       // mu q with q = 1/|V_n|, |V_n| = u
        }
        for (int i = u; i < 64; i += RS) s_w[i] = 0.f;
        __syncthreads();
        const int lane = u & 31;
        // Tracking threads (warps 1..S-1, idle while warp 0 runs a block) keep the next chunk's
        // samples: starting value during the first block, then each block's summed coefficient
        // changes (published by warp 0) applied during the following block, kernel values from
        // the next-chunk table in global memory (off the recurrence's critical path).
        const int n_next = track ? 2 * min(g.T, g.P - (t0 + Tc)) : 0;
        float tp[2] = {0.f, 0.f};
        // x~ = r(t) for r1(t) and -i r(t) for r2(t); lanes outside L carry a zero change
        auto dc_apply = [&](const float *agg, int wl0b) {
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const int idx = tu + it * ntr;
                if (idx >= dc_parts * M) continue;
                const int mm = idx % M, part = idx / M;
                const int j0 = part * NL / dc_parts, j1 = (part + 1) * NL / dc_parts;
                for (int j = j0; j < j1; ++j) {
                    const float d = agg[j];
                    const int ms = wl0b + j;
                    const int pi = min(max((ms >> 1) - pa0, 0), npil - 1);
                    const float2 x = s_pil[pi * M + mm];
                    if (ms & 1) { dcx[it] = fmaf(d, x.y, dcx[it]); dcy[it] = fmaf(-d, x.x, dcy[it]); }
                    else        { dcx[it] = fmaf(d, x.x, dcx[it]); dcy[it] = fmaf(d, x.y, dcy[it]); }
                }
            }
        };
        // At this chunk's start the entries of L hold gamma only at the carried samples (the new
        // ones start at 0), so the tracked part of f_{s0} at a next-chunk sample x is
        //   w_L <w, x> + w_G sum_{carried j} gamma_j kappa_G(x_j, x)
        //     = w_L <w - sum_{carried j} gamma_j x_j, x> + sum_{carried j} gamma_j kappa(x_j, x),
        // the second form using the tabulated sum kernel; the tracking threads form the reduced
        // filter, meet at a named barrier of their own, then evaluate their samples.
        auto track_init = [&]() {
            for (int mm = tu; mm < M; mm += ntr) {
                float2 c = s_clin[mm];
                for (int j = 0; j < nc; ++j) {
                    const float d = -s_gcar[j];
                    const float2 x = s_pil[(((l0 + j) >> 1) - pa0) * M + mm];
                    if ((l0 + j) & 1) { c.x = fmaf(d, x.y, c.x); c.y = fmaf(-d, x.x, c.y); }
                    else              { c.x = fmaf(d, x.x, c.x); c.y = fmaf(d, x.y, c.y); }
                }
                s_clinw[mm] = c;
            }
            asm volatile("bar.sync 1, %0;" ::"r"(ntr) : "memory");
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int v = tu + i * ntr;
                if (v >= n_next) continue;
                const int tv = t0 + Tc + (v >> 1), lvv = v & 1;
                const float2 *rv = a.rx + (size_t)tv * M;
                float l0s = 0.f, l1s = 0.f;
                for (int mm = 0; mm < M; mm += 2) {
                    const float4 x = __ldcg(reinterpret_cast<const float4 *>(rv + mm));
                    const float2 c = s_clinw[mm], cb = s_clinw[mm + 1];
                    l0s = lvv ? fmaf(c.x, x.y, fmaf(-c.y, x.x, l0s)) : fmaf(c.x, x.x, fmaf(c.y, x.y, l0s));
                    l1s = lvv ? fmaf(cb.x, x.w, fmaf(-cb.y, x.z, l1s)) : fmaf(cb.x, x.z, fmaf(cb.y, x.w, l1s));
                }
                // s_gcar is zero past the carried samples; rows clamped into the table
                float acc4[4] = {a.wL * (l0s + l1s), 0.f, 0.f, 0.f};
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    acc4[j & 3] = fmaf(s_gcar[j], __ldcg(a.kx + (size_t)min(j, R - 1) * g.KXS + v), acc4[j & 3]);
                tp[i] = (acc4[0] + acc4[1]) + (acc4[2] + acc4[3]);
            }
        };
        auto track_apply = [&](const float *agg, int r0) {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int v = tu + i * ntr;
                if (v >= n_next) continue;
                // rows outside [0, R) belong to lanes whose summed change is zero: clamp, no branch,
                // so that all NL loads are in flight together
                float kv[NL];
#pragma unroll
                for (int j = 0; j < NL; ++j) kv[j] = __ldcg(a.kx + (size_t)min(max(r0 + j, 0), R - 1) * g.KXS + v);
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int j = 0; j < NL; ++j) acc[j & 3] = fmaf(agg[j], kv[j], acc[j & 3]);
                tp[i] += (acc[0] + acc[1]) + (acc[2] + acc[3]);
            }
        };
        int blk = 0;
        for (int n0 = s0; n0 < s1; n0 += B, ++blk) {
            const int wl0 = n0 - WP + 1;  // sample of lane 0
            float *agg_cur = s_agg + (blk & 1) * 32;
            if (S > 1 && u >= 32 && blk > 0) dc_apply(s_agg + ((blk - 1) & 1) * 32, wl0 - B);
            if (S > 1 && track && u >= 32) {
                if (blk == 0) track_init();
                else track_apply(s_agg + ((blk - 1) & 1) * 32, wl0 - B - l0);
            }
            if (u < 32) {
                const int ms = wl0 + lane, lu = ms - l0;
                const bool lv = lane < NL && ms >= l0 && ms < s1;
                const int col = lv ? lu : 0;
                float pl = 0.f, c1 = 0.f, c2 = 0.f, rkl = 0.f, agg = 0.f, bl = 0.f;
                if (lv) {
                    pl = s_p[lu];
                    bl = s_b[lu];
                    c1 = bl - a.eps;  // the hyperslab [b - eps, b + eps]
                    c2 = bl + a.eps;
                    rkl = s_rk[lu];
                }
                float kc[NL];  // kappa(x_{wl0+j}, x of this lane)
#pragma unroll
                for (int j = 0; j < NL; ++j) {
                    // rows >= -WP + 1 (the zero rows); rows past R belong to invalid lanes, whose
                    // beta is 0: clamp instead of branching so that the loads issue together
                    kc[j] = s_kmat[min(wl0 + j - l0, R - 1) * RS + col];
                }
                // kChecked: a partial last block, the filling window (n < W - 1), case logging,
                // outputs at arrival or decided targets; kViol: weights on the violated slabs
                auto steps = [&](auto checked_c, auto evict_c, auto viol_c) {
                    constexpr bool kChecked = decltype(checked_c)::value, kEvict = decltype(evict_c)::value;
                    constexpr bool kViol = decltype(viol_c)::value;
#pragma unroll
                    for (int s = 0; s < B; ++s) {
                        const int n = n0 + s;
                        if (kChecked && n >= s1) break;
                        if (kEvict && !(n & 1) && (n >> 1) + tb >= D) {
                            const int e = (n >> 1) - t0;
                            pl -= a.wG * fmaf(s_egam[2 * e], s_gev[e * 2 * RS + col],
                                              s_egam[2 * e + 1] * s_gev[(e * 2 + 1) * RS + col]);
                        }
                        if (kExt && kChecked && lane == s + WP - 1) {  // sample n arrives: pl = f_n(x_n)
                            if (a.soft_out) a.soft_out[((size_t)((n - n_first) >> 1) * K + k) * 2 + (n & 1)] = pl;
                            if (a.decide) {  // its target: the decision on the filter's own output
                                bl = pam_value(pam_level(pl, a.qam_half, a.qam_a), a.qam_half, a.qam_a);
                                c1 = bl - a.eps;
                                c2 = bl + a.eps;
                            }
                        }
                        // window J_n = samples [n - W + 1, n] = lanes [s + WP - W, s + WP - 1]
                        const bool inw = lv && lane >= s + WP - W && lane <= s + WP - 1;
                        float muq;
                        if constexpr (kViol) {  // mu q with q = 1/|V_n| on the violated slabs
                            const bool viol = inw && (pl < c1 || pl > c2);
                            muq = s_muqv[__popc(__ballot_sync(0xffffffffu, viol))];
                        } else {                // mu q with q = 1/|J_n|
                            muq = kChecked && n + sb < W - 1 ? s_muq[n + sb] : muq_full;
                        }
                        const float sc = inw ? muq * rkl : 0.f;
                        const float mb = (fminf(fmaxf(pl, c1), c2) - pl) * sc;  // mu q beta_j
                        agg += mb;
                        if (kChecked && log_cases && inw)
                            a.case_log[((size_t)(n - n_first) * W + (ms - n + W - 1)) * K + k] =
                                (int8_t)(pl < c1 ? -1 : (pl > c2 ? 1 : 0));
                        float *ring = s_w + (s & 1) * 32;
                        ring[lane] = mb;
                        __syncwarp();
                        float acc[4] = {pl, 0.f, 0.f, 0.f};
                        const int b4 = s & ~3;
#pragma unroll
                        for (int q4 = 0; q4 < WP + 4; q4 += 4) {
                            const float4 v = *reinterpret_cast<const float4 *>(ring + b4 + q4);
                            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                            for (int r = 0; r < 4; ++r) {
                                const int j = b4 + q4 + r;
                                if (j >= s && j < s + WP) acc[(j - s) & 3] = fmaf(vv[r], kc[j], acc[(j - s) & 3]);
                            }
                        }
                        pl = (acc[0] + acc[1]) + (acc[2] + acc[3]);
                    }
                };
                using T_ = std::true_type;
                using F_ = std::false_type;
                const bool checked = n0 + B > s1 || n0 + sb < W - 1 || log_cases || (kExt && (a.decide || a.soft_out));
                if (kExt && a.qviol) {
                    if constexpr (kExt) {
                        if (evict) steps(T_{}, T_{}, T_{});
                        else steps(T_{}, F_{}, T_{});
                    }
                } else if (evict) {
                    if (checked) steps(T_{}, T_{}, F_{});
                    else steps(F_{}, T_{}, F_{});
                } else {
                    if (checked) steps(T_{}, F_{}, F_{});
                    else steps(F_{}, F_{}, F_{});
                }
                if (lv) {
                    s_p[lu] = pl;
                    s_g[lu] += agg;
                    s_b[lu] = bl;
                }
                agg_cur[lane] = lv ? agg : 0.f;
            }
            __syncthreads();
            // the block's moves of every later sample, and its dropped entries
            if (valid && m >= n0 + B) {
                const int r0 = wl0 - l0;
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int j = 0; j < NL; ++j)  // rows past R: lanes with zero change (rows < 0: zero rows)
                    acc[j & 3] = fmaf(agg_cur[j], kcol[min(r0 + j, R - 1) * RS], acc[j & 3]);
                float pv = s_p[u] + ((acc[0] + acc[1]) + (acc[2] + acc[3]));
                if (evict) {
                    for (int n = n0 + (n0 & 1); n < min(n0 + B, s1); n += 2) {
                        if ((n >> 1) + tb < D) continue;
                        const int e = (n >> 1) - t0;
                        pv -= a.wG * fmaf(s_egam[2 * e], s_gev[e * 2 * RS + u],
                                          s_egam[2 * e + 1] * s_gev[(e * 2 + 1) * RS + u]);
                    }
                }
                s_p[u] = pv;
            }
            __syncthreads();
        }
        if (S > 1 && u >= 32 && blk > 0) dc_apply(s_agg + ((blk - 1) & 1) * 32, s0 + (blk - 1) * B - WP + 1);
        if (S > 1 && track && u >= 32) {  // the last block's changes, then hand over
            if (blk == 0) track_init();
            else track_apply(s_agg + ((blk - 1) & 1) * 32, s0 + (blk - 1) * B - WP + 1 - l0);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int v = tu + i * ntr;
                if (v < n_next) a.track_out[v * K + k] = tp[i];
            }
        }
        if (valid) {
            p = s_p[u];
            gam = s_g[u];
            b = s_b[u];
        }
    } else if constexpr (WP <= kRingMax) {
        // Window ring: sample j sits in slot (j - s0) mod WP.  kc[r] holds kappa(x_j, x_u) of the
        // sample j currently in slot r, the betas of the step sit in a ring of WP floats (two,
        // alternating by step parity), so the window sum is WP register FMAs over broadcast
        // vector loads.  Slots of samples that left the window (WP > W) hold beta = 0.
        float kc[WP];
#pragma unroll
        for (int r = 0; r < WP; ++r) kc[r] = kcol[(s0 - WP + r - l0) * RS];  // rows >= -WP: zero rows
        const int slot = valid ? (m - s0 + WP) % WP : 0;
        for (int nb = s0; nb < s1; nb += WP) {
#pragma unroll
            for (int r = 0; r < WP; ++r) {
                const int n = nb + r;
                if (n >= s1) break;
                const int un = n - l0;
                kc[r] = kcol[un * RS];  // sample n enters slot r
                if (evict && !(n & 1) && (n >> 1) + tb >= D) {
                    const int e = (n >> 1) - t0;
                    p -= a.wG * fmaf(s_egam[2 * e], s_gev[e * 2 * RS + u],
                                     s_egam[2 * e + 1] * s_gev[(e * 2 + 1) * RS + u]);
                }
                if (kExt && valid && m == n) {  // sample n arrives: p = f_n(x_n)
                    if (a.soft_out) a.soft_out[((size_t)((n - n_first) >> 1) * K + k) * 2 + (n & 1)] = p;
                    if (a.decide) b = pam_value(pam_level(p, a.qam_half, a.qam_a), a.qam_half, a.qam_a);
                }
                float muq = muq_full;
                if (n + sb < W - 1) muq = a.mu / (float)(n + sb + 1);  // mu q, q = 1/|J_n|
                float *ring = s_beta + (r & 1) * WP;          // nb - s0 is a multiple of WP (even)
                float beta = 0.f;
                bool viol = false;
                if (valid && m <= n && m > n - WP) {
                    if (m > n - W) {
                        const float e = p - b;  // <f_n, kappa(x_j,.)> - b_j
                        // Eq. beta without branches: (-e - eps) below the slab, (eps - e) above, 0 inside
                        beta = (fmaxf(-e - a.eps, 0.f) - fmaxf(e - a.eps, 0.f)) * rk;
                        viol = e < -a.eps || e > a.eps;
                        if (log_cases)
                            a.case_log[((size_t)(n - n_first) * W + (m - n + W - 1)) * K + k] =
                                (int8_t)(e < -a.eps ? -1 : (e > a.eps ? 1 : 0));
                    }
                    ring[slot] = beta;
                }
                if (kExt && a.qviol) {  // q = 1/|V_n| on the violated slabs
                    const int nv = __syncthreads_count(viol);
                    muq = nv > 0 ? a.mu / (float)nv : 0.f;
                } else {
                    __syncthreads();
                }
                gam = fmaf(muq, beta, gam);  // (beta = 0 outside the window)
                // p_u += mu q sum_{i in J_n} beta_i kappa(x_i, x_u)
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int q4 = 0; q4 < WP; q4 += 4) {
                    const float4 bv = *reinterpret_cast<const float4 *>(ring + q4);
                    acc[0] = fmaf(bv.x, kc[q4], acc[0]);
                    acc[1] = fmaf(bv.y, kc[q4 + 1], acc[1]);
                    acc[2] = fmaf(bv.z, kc[q4 + 2], acc[2]);
                    acc[3] = fmaf(bv.w, kc[q4 + 3], acc[3]);
                }
                p = fmaf(muq, (acc[0] + acc[1]) + (acc[2] + acc[3]), p);
            }
        }
    } else {
        for (int n = s0; n < s1; ++n) {
            const int un = n - l0;
            // a new pilot arrives at n = 2t: the oldest entry is dropped once D are held
            if (evict && !(n & 1) && (n >> 1) + tb >= D) {
                const int e = (n >> 1) - t0;
                p -= a.wG * fmaf(s_egam[2 * e], s_gev[e * 2 * RS + u], s_egam[2 * e + 1] * s_gev[(e * 2 + 1) * RS + u]);
            }
            if (kExt && valid && m == n) {  // sample n arrives: p = f_n(x_n)
                if (a.soft_out) a.soft_out[((size_t)((n - n_first) >> 1) * K + k) * 2 + (n & 1)] = p;
                if (a.decide) b = pam_value(pam_level(p, a.qam_half, a.qam_a), a.qam_half, a.qam_a);
            }
            const int ujlo = max(0, n - W + 1) - l0;
            float muq = (n + sb >= W - 1) ? muq_full : a.mu / (float)(n + sb + 1);  // mu q, q = 1/|J_n|
            float *bb = s_beta + (n & 1) * (WP + RS) + WP;
            float beta = 0.f;
            bool viol = false;
            if (u >= ujlo && u <= un) {
                const float e = p - b;  // <f_n, kappa(x_j,.)> - b_j
                // Eq. beta without branches: (-e - eps) below the slab, (eps - e) above it, 0 inside
                beta = (fmaxf(-e - a.eps, 0.f) - fmaxf(e - a.eps, 0.f)) * rk;
                viol = e < -a.eps || e > a.eps;
                bb[u] = beta;
                if (log_cases)
                    a.case_log[((size_t)(n - n_first) * W + (m - n + W - 1)) * K + k] =
                        (int8_t)(e < -a.eps ? -1 : (e > a.eps ? 1 : 0));
            } else if (u < ujlo && u > un - WP) {
                bb[u] = 0.f;
            }
            if (kExt && a.qviol) {  // q = 1/|V_n| on the violated slabs
                const int nv = __syncthreads_count(viol);
                muq = nv > 0 ? a.mu / (float)nv : 0.f;
            } else {
                __syncthreads();
            }
            gam = fmaf(muq, beta, gam);  // (beta = 0 outside the window)
            // p_u += mu q sum_{i in J_n} beta_i kappa(x_i, x_u)
            const float *kp = kcol + (un - WP + 1) * RS;
            const float *bp = bb + (un - WP + 1);
            float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
            for (int d = 0; d < WP; d += 2) {
                acc0 = fmaf(bp[d], kp[d * RS], acc0);
                acc1 = fmaf(bp[d + 1], kp[(d + 1) * RS], acc1);
            }
            p = fmaf(muq, acc0 + acc1, p);
        }
    }

    // ---- write back: coefficients, carried predictions, linear filter ---------------------------
    if (valid) {
        const size_t slot = (size_t)((tb + pa) % D);
        a.gamma[(slot * 2 + l) * K + k] = gam;
        s_dg[u] = gam - gam0;
        s_tgt[u] = b;
        const int l0n = live_start(s1, W);
        if (m >= l0n) a.carry[(m - l0n) * K + k] = p;
        if (m >= s0) {  // the chunk's new samples: their targets (decided or given) join the state
            a.target[(slot * K + k) * 2 + l] = b;
            if (a.decide) reinterpret_cast<float *>(a.sym)[((size_t)pa * K + k) * 2 + l] = b;
        }
    }
    __syncthreads();
    if (a.hard_out && valid && l == 0 && m >= s0)  // Gray-QAM label of the vector's two targets
        a.hard_out[(size_t)(pa - g.nc0) * K + k] = qam_label(s_tgt[u], s_tgt[u + 1], a.qam_half, a.qam_a);
    // c_k += sum_u dgamma_u x~_u, with x~ = r(t) for r1(t) and -i r(t) for r2(t): the live range
    // is split into np parts per antenna, partial sums combined in a fixed order
    {
        const int np = kDcInRegs ? dc_parts : max(1, min(RS / M, 16));
        float2 *s_part = reinterpret_cast<float2 *>(s_beta);  // free after the recurrence
        if (kDcInRegs && u >= 32) {
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const int idx = tu + it * ntr;
                if (idx < dc_parts * M) s_part[(idx / M) * M + idx % M] = make_float2(dcx[it], dcy[it]);
            }
        }
        for (int tid = u; !kDcInRegs && tid < np * M; tid += RS) {
            const int mm = tid % M, part = tid / M;
            const int v0 = R * part / np, v1 = R * (part + 1) / np;
            float2 c0 = make_float2(0.f, 0.f), c1 = make_float2(0.f, 0.f);
            int v = v0;
            for (; v + 1 < v1; v += 2) {
                const int ma = l0 + v, mb = ma + 1;
                const float da = s_dg[v], db = s_dg[v + 1];
                const float2 xa = s_pil[((ma >> 1) - pa0) * M + mm], xb = s_pil[((mb >> 1) - pa0) * M + mm];
                if (ma & 1) { c0.x = fmaf(da, xa.y, c0.x); c0.y = fmaf(-da, xa.x, c0.y); }
                else        { c0.x = fmaf(da, xa.x, c0.x); c0.y = fmaf(da, xa.y, c0.y); }
                if (mb & 1) { c1.x = fmaf(db, xb.y, c1.x); c1.y = fmaf(-db, xb.x, c1.y); }
                else        { c1.x = fmaf(db, xb.x, c1.x); c1.y = fmaf(db, xb.y, c1.y); }
            }
            if (v < v1) {
                const int ma = l0 + v;
                const float da = s_dg[v];
                const float2 xa = s_pil[((ma >> 1) - pa0) * M + mm];
                if (ma & 1) { c0.x = fmaf(da, xa.y, c0.x); c0.y = fmaf(-da, xa.x, c0.y); }
                else        { c0.x = fmaf(da, xa.x, c0.x); c0.y = fmaf(da, xa.y, c0.y); }
            }
            s_part[part * M + mm] = make_float2(c0.x + c1.x, c0.y + c1.y);
        }
        __syncthreads();
        for (int mm = u; mm < M; mm += RS) {
            float2 c = s_clin[mm];
            for (int part = 0; part < np; ++part) {
                const float2 d = s_part[part * M + mm];
                c.x += d.x;
                c.y += d.y;
            }
            a.clin[mm * K + k] = c;
        }
    }

    // ---- new dictionary entries of this chunk (slot (tb + t) % D), their norms, bookkeeping --
    // (spread over the K user CTAs, which all hold the chunk's pilots)
    for (int i = k * RS + u; i < Tc * M; i += K * RS) {
        const int t = t0 + i / M, mm = i % M;
        a.dict[(size_t)((tb + t) % D) * M + mm] = s_pil[(t - pa0) * M + mm];
    }
    for (int i = k * RS + u; i < Tc; i += K * RS) {
        const float2 *rv = s_pil + (t0 + i - pa0) * M;
        float nrm = 0.f;
        for (int mm = 0; mm < M; ++mm) nrm = fmaf(rv[mm].x, rv[mm].x, fmaf(rv[mm].y, rv[mm].y, nrm));
        a.dict_norm[(tb + t0 + i) % D] = nrm;
    }
    if (k == 0) {
        if (a.chunk == g.n_chunks - 1 && u == 0) {
            const int total = tb + g.P;  // vectors trained on since the state was emptied
            a.meta[0] = min(total, D);
            a.meta[1] = total >= D ? total % D : 0;
            a.meta[2] = total;
        }
    }
}

}  // namespace apsm
