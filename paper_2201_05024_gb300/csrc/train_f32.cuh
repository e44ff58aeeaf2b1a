// train_f32.cuh -- FP32 APSM training kernels (Eq. apsm, Eq. beta, window J_n of Sec. II-D;
// Sec. III-B training).
//
// The recurrence runs over the 2P real-split samples n = 2t + l, in chunks of T pilots.
// For chunk c (pilots [t0, t0+Tc), samples [s0, s1)) every sample that can be touched in the
// chunk lies in the live range L = [l0, s1), l0 = max(0, s0 - W + 1): the W-1 window samples
// carried from the previous chunk plus the chunk's own.  Each sample m in L keeps a running
// prediction p_m = f_n(x_m) of the current filter.  Because f is linear in its coefficients,
//   f_{n+1}(x_m) = f_n(x_m) + mu q sum_{i in J_n} beta_i kappa(x_i, x_m)          (Eq. apsm)
// exactly, so one step needs only the window's residuals, its betas (Eq. beta) and the
// kernel values kappa(x_i, x_m) between samples of L; dropping a dictionary entry subtracts its
// Gaussian terms.  The expensive part -- f at the start of the chunk evaluated at the chunk's
// new samples against the whole dictionary -- is the detection kernel in partial mode, run on
// all SMs between chunks (phase A).  The serial part (phase B) is one CTA with one warp per
// user: users are independent, so a step needs only warp-level synchronisation.
//
// Kernels:
//   train_gram_kernel   kappa(x_u, x_v) for all u, v in L of every chunk (sum kernel, Fact 1)
//                       and kappa_G between each entry dropped during a chunk and L.
//   train_chunk_kernel  phase B of one chunk.
#pragma once

#include "apsm_common.cuh"

namespace apsm {

struct TrainGeom {
    int M, K, W, D, P;
    int T;         // pilots per chunk
    int n_chunks;
    int RMAX;      // 2T + W - 1: live-range capacity
    int slice;     // entries per phase-A slice
};

__host__ __device__ inline void chunk_range(const TrainGeom &g, int c, int &t0, int &Tc, int &s0, int &s1,
                                            int &l0) {
    t0 = c * g.T;
    Tc = min(g.T, g.P - t0);
    s0 = 2 * t0;
    s1 = 2 * (t0 + Tc);
    l0 = max(0, s0 - g.W + 1);
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

__global__ void train_gram_kernel(const float2 *__restrict__ rx, TrainGeom g, float k2, float wL, float wG,
                                  float *__restrict__ kmat, float *__restrict__ gev) {
    const int c = blockIdx.y;
    int t0, Tc, s0, s1, l0;
    chunk_range(g, c, t0, Tc, s0, s1, l0);
    const int R = s1 - l0;
    const int RM = g.RMAX;
    const int n_k = RM * RM, n_e = g.T * 2 * RM;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n_k + n_e; idx += gridDim.x * blockDim.x) {
        if (idx < n_k) {
            const int u = idx / RM, v = idx % RM;
            float val = 0.f;
            if (u < R && v < R) {
                const int mu_ = l0 + u, mv = l0 + v;
                float dot, d2;
                sample_pair(rx + (size_t)(mu_ >> 1) * g.M, rx + (size_t)(mv >> 1) * g.M, g.M, mu_ & 1, mv & 1, dot,
                            d2);
                val = fmaf(wL, dot, wG * ex2(-k2 * d2));  // kappa = w_L kappa_L + w_G kappa_G (Fact 1)
            }
            kmat[(size_t)c * n_k + idx] = val;
        } else {
            const int j = idx - n_k;
            const int e = j / (2 * RM), l = (j / RM) & 1, v = j % RM;
            const int t = t0 + e;
            float val = 0.f;
            if (e < Tc && t >= g.D && v < R) {
                const int mv = l0 + v;
                float dot, d2;
                sample_pair(rx + (size_t)(t - g.D) * g.M, rx + (size_t)(mv >> 1) * g.M, g.M, l, mv & 1, dot, d2);
                val = ex2(-k2 * d2);
            }
            gev[(size_t)c * n_e + j] = val;
        }
    }
}

struct ChunkArgs {
    TrainGeom g;
    int chunk;
    float mu, eps, wL, wG;
    const float2 *rx;       // [P][M]
    const float2 *sym;      // [P][K]
    float2 *dict;           // [A][M]
    float *dict_norm;       // [A]
    float *gamma;           // [A][2][K]
    float2 *clin;           // [M][K]
    int *meta;              // [4]
    const float *kmat;      // [n_chunks][RMAX][RMAX]
    const float *gev;       // [n_chunks][T][2][RMAX]
    const float *partial;   // [n_slices][Tc][2K]
    int n_slices;
    float *carry;           // [W][K]
    int8_t *case_log;       // [2P][W][K] nullable
};

struct ChunkSmem {
    int kmat, gev, egam, beta, dg, pil, bytes;
    __host__ __device__ ChunkSmem(const TrainGeom &g) {
        const int RM = g.RMAX;
        const int npil = g.T + (g.W + 1) / 2 + 1;
        kmat = 0;
        gev = kmat + RM * RM * 4;
        egam = gev + g.T * 2 * RM * 4;
        beta = egam + g.T * 2 * g.K * 4;
        dg = beta + g.K * 2 * RM * 4;
        pil = round_up(dg + g.K * RM * 4, 16);
        bytes = pil + npil * g.M * 8;
    }
};

template <int S>
__global__ void __launch_bounds__(512) train_chunk_kernel(const ChunkArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const TrainGeom &g = a.g;
    const ChunkSmem L(g);
    float *s_kmat = reinterpret_cast<float *>(smem + L.kmat);
    float *s_gev = reinterpret_cast<float *>(smem + L.gev);
    float *s_egam = reinterpret_cast<float *>(smem + L.egam);
    float *s_beta = reinterpret_cast<float *>(smem + L.beta);
    float *s_dg = reinterpret_cast<float *>(smem + L.dg);
    float2 *s_pil = reinterpret_cast<float2 *>(smem + L.pil);

    const int M = g.M, K = g.K, W = g.W, D = g.D, RM = g.RMAX;
    int t0, Tc, s0, s1, l0;
    chunk_range(g, a.chunk, t0, Tc, s0, s1, l0);
    const int R = s1 - l0;
    const int pa0 = l0 >> 1;            // first pilot touching L
    const int npil = t0 + Tc - pa0;
    const int tid = threadIdx.x, nthr = blockDim.x;

    // ---- stage the chunk's kernel values, dropped-entry data and pilots -------------------
    {
        const float *src = a.kmat + (size_t)a.chunk * RM * RM;
        for (int i = tid; i < RM * RM; i += nthr) s_kmat[i] = src[i];
        const bool evict = (t0 + Tc - 1) >= D;
        if (evict) {
            const float *gs = a.gev + (size_t)a.chunk * g.T * 2 * RM;
            for (int i = tid; i < g.T * 2 * RM; i += nthr) s_gev[i] = gs[i];
            for (int i = tid; i < Tc * 2 * K; i += nthr) {
                const int e = i / (2 * K), r = i % (2 * K);
                const int t = t0 + e;
                s_egam[i] = (t >= D) ? a.gamma[(size_t)((t - D) % D) * 2 * K + r] : 0.f;
            }
        }
        for (int i = tid; i < npil * M; i += nthr) s_pil[i] = a.rx[(size_t)pa0 * M + i];
    }
    __syncthreads();

    const int k = tid >> 5, lane = tid & 31;
    if (k < K) {
        float p[S], gam[S], gam0[S], b[S];
        // ---- initial predictions p_m = f_{s0}(x_m) and coefficients ------------------------
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int u = lane + 32 * s;
            p[s] = gam[s] = gam0[s] = b[s] = 0.f;
            if (u < R) {
                const int m = l0 + u, pa = m >> 1, l = m & 1;
                const float2 sy = a.sym[(size_t)pa * K + k];
                b[s] = l ? sy.y : sy.x;  // b_{2t} = Re b(t), b_{2t+1} = Im b(t)
                if (m < s0) {
                    p[s] = a.carry[u * K + k];
                    gam[s] = a.gamma[((size_t)(pa % D) * 2 + l) * K + k];
                } else {
                    float lin = 0.f;  // Re / Im of c_k^H r
                    const float2 *rv = s_pil + (pa - pa0) * M;
                    for (int mm = 0; mm < M; ++mm) {
                        const float2 c = a.clin[mm * K + k], x = rv[mm];
                        lin = l ? fmaf(c.x, x.y, fmaf(-c.y, x.x, lin)) : fmaf(c.x, x.x, fmaf(c.y, x.y, lin));
                    }
                    float gs = 0.f;
                    for (int sl = 0; sl < a.n_slices; ++sl)
                        gs += a.partial[((size_t)sl * Tc + (pa - t0)) * 2 * K + l * K + k];
                    p[s] = fmaf(a.wL, lin, a.wG * gs);
                }
                gam0[s] = gam[s];
            }
        }

        // ---- the recurrence over the chunk's samples -----------------------------------------
        float *beta_buf = s_beta + k * 2 * RM;
        for (int n = s0; n < s1; ++n) {
            const int un = n - l0;
            // a new pilot arrives at n = 2t: the oldest entry is dropped once D are held
            if (!(n & 1) && (n >> 1) >= D) {
                const int e = (n >> 1) - t0;
                const float ge1 = s_egam[(e * 2 + 0) * K + k], ge2 = s_egam[(e * 2 + 1) * K + k];
                const float *gv = s_gev + e * 2 * RM;
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const int u = lane + 32 * s;
                    if (u < R && u >= un - W + 1) p[s] -= a.wG * fmaf(ge1, gv[u], ge2 * gv[RM + u]);
                }
            }
            const int jlo = max(0, n - W + 1);
            const int ujlo = jlo - l0;
            const float muq = a.mu / (float)(n - jlo + 1);  // mu q, q = 1/|J_n|
            float *bb = beta_buf + (n & 1) * RM;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const int u = lane + 32 * s;
                if (u >= ujlo && u <= un) {
                    const float e = p[s] - b[s];                 // <f_n, kappa(x_j,.)> - b_j
                    const float kjj = s_kmat[u * RM + u];         // kappa(x_j, x_j)
                    int cs = 0;
                    float beta = 0.f;                              // Eq. beta
                    if (e < -a.eps) { cs = -1; beta = (-e - a.eps) / kjj; }
                    else if (e > a.eps) { cs = 1; beta = (-e + a.eps) / kjj; }
                    if (kjj == 0.f) beta = 0.f;
                    gam[s] = fmaf(muq, beta, gam[s]);
                    bb[u] = beta;
                    if (a.case_log) a.case_log[((size_t)n * W + (l0 + u - n + W - 1)) * K + k] = (int8_t)cs;
                }
            }
            __syncwarp();
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const int u = lane + 32 * s;
                if (u < R && u >= un - W + 2) {
                    float acc = 0.f;
                    for (int i = ujlo; i <= un; ++i) acc = fmaf(bb[i], s_kmat[i * RM + u], acc);
                    p[s] = fmaf(muq, acc, p[s]);
                }
            }
        }

        // ---- write back: coefficients, linear filter, carried predictions -------------------
        float *dg = s_dg + k * RM;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int u = lane + 32 * s;
            if (u < R) {
                const int m = l0 + u, pa = m >> 1, l = m & 1;
                a.gamma[((size_t)(pa % D) * 2 + l) * K + k] = gam[s];
                dg[u] = gam[s] - gam0[s];
            }
        }
        const int l0n = max(0, s1 - W + 1);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int u = lane + 32 * s;
            if (u < R && l0 + u >= l0n) a.carry[(l0 + u - l0n) * K + k] = p[s];
        }
        __syncwarp();
        // c_k += sum_u dgamma_u x~_u, with x~ = r(t) for r1(t) and -i r(t) for r2(t)
        for (int mm = lane; mm < M; mm += 32) {
            float2 c = a.clin[mm * K + k];
            for (int u = 0; u < R; ++u) {
                const int m = l0 + u, pa = m >> 1;
                const float d = dg[u];
                const float2 x = s_pil[(pa - pa0) * M + mm];
                if (m & 1) { c.x = fmaf(d, x.y, c.x); c.y = fmaf(-d, x.x, c.y); }
                else       { c.x = fmaf(d, x.x, c.x); c.y = fmaf(d, x.y, c.y); }
            }
            a.clin[mm * K + k] = c;
        }
    }

    // ---- new dictionary entries of this chunk (slot t % D), their norms, bookkeeping -------
    for (int i = tid; i < Tc * M; i += nthr) {
        const int t = t0 + i / M, mm = i % M;
        a.dict[(size_t)(t % D) * M + mm] = s_pil[(t - pa0) * M + mm];
    }
    for (int i = tid; i < Tc; i += nthr) {
        const float2 *rv = s_pil + (t0 + i - pa0) * M;
        float nrm = 0.f;
        for (int mm = 0; mm < M; ++mm) nrm = fmaf(rv[mm].x, rv[mm].x, fmaf(rv[mm].y, rv[mm].y, nrm));
        a.dict_norm[(t0 + i) % D] = nrm;
    }
    if (a.chunk == g.n_chunks - 1 && tid == 0) {
        a.meta[0] = min(g.P, D);
        a.meta[1] = g.P >= D ? g.P % D : 0;
        a.meta[2] = g.P;
    }
}

}  // namespace apsm
