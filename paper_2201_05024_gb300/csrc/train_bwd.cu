// train_bwd.cu -- adjoint of the APSM training recurrence (apsm_train_backward).
//
// Forward (Eq. apsm with Eq. beta over the window J_n, Sec. II-D), per user, state
// S_n = (w, gamma_i for every centre):
//   y_j = w_L <w, x_j> + w_G sum_{i alive at n} gamma_i kappa_G(x_i, x_j),  e_j = y_j - b_j,
//   kappa_jj = w_L ||x_j||^2 + w_G,  beta_j = (-e_j - s_j eps) / kappa_jj for s_j = +1 (e < -eps)
//   or -1 (e > eps), beta_j = 0 inside the slab;
//   S_{n+1} = S_n + sum_{j in J_n} a_j (unit vector of centre j, x_j),  a_j = mu q beta_j.
// Reverse mode, with (gbar, wbar) the adjoint of S_{n+1}:
//   abar_j = gbar_j + <wbar, x_j>;  mubar += q beta_j abar_j;  betabar_j = mu q abar_j;
//   outside the slab: ybar_j = -betabar_j / kappa_jj, epsbar += -s_j betabar_j / kappa_jj,
//   w_Lbar += (-betabar_j beta_j / kappa_jj) (||x_j||^2 - 1);
//   then wbar += ybar_j w_L x_j, w_Lbar += ybar_j (<w, x_j> - gauss_j),
//   sigmabar += ybar_j w_G sum_i gamma_i kappa_G(x_i, x_j) d_ij^2 / sigma^3,
//   gbar_i += ybar_j w_G kappa_G(x_i, x_j) for every alive centre i.
// Inside the slab the derivative is taken as 0 (also at |e| = eps exactly).
//
// Cost per step O(W^2 + S) instead of O(W S):
//  * forward: the predictions of the window samples are carried from step to step (the W
//    projections of a step change them by sum_o a_o kappa(x_{j_o}, x_j); an evicted centre's
//    contribution is subtracted), and a sample's prediction is formed once, on arrival, from the
//    live centres; every step's tape (beta, branch, kappa, <w, x_j>, gauss_j, its sigma weight)
//    goes to the workspace, so nothing is re-run;
//  * reverse: gbar_i is read only while centre i is in the window.  R_j, the sum of the cg terms
//    of sample j over the steps swept so far, gives centre i's adjoint when it enters the window
//    from below: gbar_i = final_i + sum_j R_j kappa_G(x_i, x_j) over the steps in which i is
//    alive (for a centre evicted during the call, R at the eviction step is kept and subtracted);
//    from then on it is pushed the W terms of each step like the forward predictions.
// Kernel values between samples come from tables built once per call.  One CTA of 4 warps per
// user: the threads split the O(S) sums of an arrival, a thread per window slot for the scalar
// terms (summed in slot order at the end), a thread per component or window sample for the
// O(W) updates.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "apsm_common.cuh"
#include "train_f32.cuh"

namespace apsm {

extern std::atomic<long long> g_launches;  // apsm_api.cu

struct Tape {  // one window slot of one step
    float beta, s, kappa, dotw, gauss, gd2;
};

struct TrainBwdArgs {
    int M, K, W, D, P;
    int Sp;                 // row stride of the tables: 2P rounded up to a multiple of 4
    float sigma, mu, eps, wL, wG, k2;
    const float2 *rx;       // [P][M]
    const float2 *sym;      // [P][K]
    const float2 *clin0;    // [M][K] or null
    const float *dgamma;    // [A][2][K] adjoint of the final coefficients (ring layout)
    const float2 *dclin;    // [M][K] adjoint of the final linear filter
    float *ltab;            // [2P][Sp] x_i . x_j
    float *gtab;            // [2P][Sp] kappa_G(x_i, x_j)
    float *gdtab;           // [2P][Sp] kappa_G(x_i, x_j) ||x_i - x_j||^2
    Tape *tape;             // [K][2P][W]
    float *snap;            // [K][P - D][W] R at the eviction steps (P > D only)
    float *scal;            // [K][4] per-user sigma, mu, eps, w_L adjoints
    float2 *dclin0;         // [M][K] out
    float *dscalars;        // [4] out
    // instance i of a batch: the pointers above advanced by i times these (elements; ws_stride in
    // bytes for the workspace regions ltab, gtab, gdtab, tape, snap, scal)
    size_t st_rx, st_sym, st_clin0, st_dgamma, st_mk, ws_stride;
    int mode;  // 1: tables' forward pass (tape), 2: reverse sweep, 3: both
};

// The arguments of instance i (blockIdx.y of every launch below).
__device__ __forceinline__ TrainBwdArgs for_instance(const TrainBwdArgs &a0, int i) {
    TrainBwdArgs a = a0;
    auto adv = [&](auto *ptr) {
        return reinterpret_cast<decltype(ptr)>(reinterpret_cast<unsigned char *>(ptr) + i * a0.ws_stride);
    };
    a.rx += i * a.st_rx;
    a.sym += i * a.st_sym;
    if (a.clin0) a.clin0 += i * a.st_clin0;
    a.dgamma += i * a.st_dgamma;
    a.dclin += i * a.st_mk;
    a.dclin0 += i * a.st_mk;
    a.dscalars += 4 * (size_t)i;
    a.ltab = adv(a.ltab);
    a.gtab = adv(a.gtab);
    a.gdtab = adv(a.gdtab);
    a.tape = adv(a.tape);
    a.snap = adv(a.snap);
    a.scal = adv(a.scal);
    return a;
}

__global__ void train_bwd_tables_kernel(const TrainBwdArgs a0) {
    const TrainBwdArgs a = for_instance(a0, blockIdx.y);
    const int S = 2 * a.P, Sp = a.Sp;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)S * Sp;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i0 = (int)(idx / Sp), j0 = (int)(idx % Sp);
        if (j0 >= S) {  // row padding
            a.ltab[idx] = 0.f;
            a.gtab[idx] = 0.f;
            a.gdtab[idx] = 0.f;
            continue;
        }
        const int i = min(i0, j0), j = max(i0, j0);  // both halves from one ordering: exactly symmetric
        float dot, d2;
        sample_pair(a.rx + (size_t)(i >> 1) * a.M, a.rx + (size_t)(j >> 1) * a.M, a.M, i & 1, j & 1, dot, d2);
        const float g = ex2(-a.k2 * d2);
        a.ltab[idx] = dot;
        a.gtab[idx] = g;
        a.gdtab[idx] = g * d2;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// component m of the real-split sample j (Sec. II-D): x_{2t} = [Re r; Im r], x_{2t+1} = [Im r; -Re r]
__device__ __forceinline__ float xcomp(const float2 *rx, int M, int j, int m) {
    const float2 *r = rx + (size_t)(j >> 1) * M;
    if (m < M) {
        const float2 v = __ldg(r + m);
        return (j & 1) ? v.y : v.x;
    }
    const float2 v = __ldg(r + (m - M));
    return (j & 1) ? -v.x : v.y;
}

// Slot of a sample in a ring of R slots from the slot b of a reference sample below it and the
// offset off in [0, 3R] between the two (no integer division on the per-step path).
__device__ __forceinline__ int ring_slot(int b, int off, int R) {
    int x = b + off;
    x -= x >= R ? R : 0;
    x -= x >= R ? R : 0;
    x -= x >= R ? R : 0;
    return x;
}

// Loads issued a step ahead of their use: predicated rather than followed by a select, so that no
// instruction waits on the data before it is used; volatile, so that they stay ahead of the barriers.
// (the predicate is set inside the asm, so no branch surrounds the load)
__device__ __forceinline__ float ldg_if(bool c, const float *p) {  // read-only data of earlier kernels
    float v = 0.f;
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q ld.global.nc.f32 %0, [%1];\n\t}"
                 : "+f"(v)
                 : "l"(p), "r"((int)c));
    return v;
}
__device__ __forceinline__ float2 ld2_if(bool c, const float *p) {  // data this kernel wrote; 8-byte aligned
    float2 v = make_float2(0.f, 0.f);
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t@q ld.global.v2.f32 {%0, %1}, [%2];\n\t}"
                 : "+f"(v.x), "+f"(v.y)
                 : "l"(p), "r"((int)c)
                 : "memory");
    return v;
}

constexpr int kBwdThreads = 128;  // 4 warps per user
constexpr int kWarpUsersMax = 16;  // users (warps) per CTA of train_bwd_warp_kernel
constexpr int kPf = 4;            // entries of the next O(S) row a thread fetches a step ahead, per table

// Entries lo + tid + q * kBwdThreads (q < kPf, below hi) of one or two table rows, a step early.
struct RowPf {
    float g[kPf], d[kPf];
};

__device__ __forceinline__ void row_fetch(RowPf &f, const float *grow, const float *drow, int lo, int hi) {
#pragma unroll
    for (int q = 0; q < kPf; ++q) {
        const int i = lo + (int)threadIdx.x + q * kBwdThreads;
        f.g[q] = ldg_if(i < hi, grow + i);
        f.d[q] = ldg_if(drow != nullptr && i < hi, drow + i);
    }
}

// The band of row r that the window needs: entries s0 + t, t = 0..W (thread t holds one, thread 0
// also t = W when W = kBwdThreads), inside [0, S).  Stored into the window rings kg, kd, kl
// [(W+1)^2] (sample j in slot j mod (W+1)) at both (r, j) and (j, r): the tables are exactly
// symmetric.
struct BandPf {
    float g[2], d[2], l[2];
};

__device__ __forceinline__ void band_fetch(BandPf &b, const TrainBwdArgs &a, int S, int W, int r, int s0) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int t = (int)threadIdx.x + q * kBwdThreads, j = s0 + t;
        const bool ok = r >= 0 && r < S && t <= W && j >= 0 && j < S;
        const size_t x = ok ? (size_t)r * a.Sp + j : 0;
        b.g[q] = ldg_if(ok, a.gtab + x);
        b.d[q] = ldg_if(ok, a.gdtab + x);
        b.l[q] = ldg_if(ok, a.ltab + x);
    }
}

// (sr, s0r: the ring slots of r and s0)
__device__ __forceinline__ void band_store(const BandPf &b, float *kg, float *kd, float *kl, int S, int W, int r,
                                           int s0, int sr, int s0r) {
    const int WR = W + 1;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int t = (int)threadIdx.x + q * kBwdThreads, j = s0 + t;
        if (r >= 0 && r < S && t <= W && j >= 0 && j < S) {
            const int sj = ring_slot(s0r, t, WR);
            const int u = sr * WR + sj, v = sj * WR + sr;
            kg[u] = b.g[q];
            kg[v] = b.g[q];
            kd[u] = b.d[q];
            kd[v] = b.d[q];
            kl[u] = b.l[q];
            kl[v] = b.l[q];
        }
    }
}

// smem (floats): gamma (forward) / R (reverse) [2P], norms [2P], w / wbar [2M], window rings
// py, pd, pw [W] (forward: gauss_j, its sigma weight, <w, x_j>; reverse: py = abar_j), ca, cb [W],
// targets pb [W], warp partials [3 * 4], kg, kd, kl [(W+1)^2] (kappa_G, kappa_G d^2 and x_i . x_j
// among the samples of the window and the one entering or leaving it), xw [(W+1)][2M] (their
// components)
__global__ void __launch_bounds__(kBwdThreads, 6) train_bwd_kernel(const TrainBwdArgs a0) {
    extern __shared__ __align__(16) float sm[];
    const TrainBwdArgs a = for_instance(a0, blockIdx.y);
    constexpr int T = kBwdThreads, NW = T / 32;
    const int k = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int M = a.M, K = a.K, W = a.W, D = a.D, P = a.P, S = 2 * P, L2 = 2 * M, WR = W + 1;
    float *gam = sm, *nrm = gam + S, *w = nrm + S, *py = w + L2, *pd = py + W, *pw = pd + W;
    float *ca = pw + W, *cb = ca + W, *pb = cb + W, *part = pb + W, *kg = part + 3 * NW, *kd = kg + WR * WR;
    float *kl = kd + WR * WR, *xw = kl + WR * WR;
    Tape *tape = a.tape + (size_t)k * S * W;
    float *snap = a.snap + (size_t)k * (P > D ? P - D : 0) * W;
    const float inv_s3 = 1.f / (a.sigma * a.sigma * a.sigma);
    const float mqW = a.mu / (float)W, qW = 1.f / (float)W;  // mu q and q of a full window
    // ring slots relative to the reference sample n - W - 1 of the current step: sW, sR are its
    // slots (mod W, mod W + 1), kept up to date as n moves (the samples used lie in [n - W - 1, n + 1])
    auto pmod = [](int x, int R) { return ((x % R) + R) % R; };
    int sW = 0, sR = 0;
    auto slotW = [&](int n, int j) { return ring_slot(sW, j - (n - W - 1), W); };
    auto slotR = [&](int n, int j) { return ring_slot(sR, j - (n - W - 1), WR); };

    auto first_centre = [&](int n) { return 2 * max(0, (n >> 1) - D + 1); };
    // centre i takes part in the steps n < evict_step(i) (its entry leaves at that step)
    auto evict_step = [&](int i) { return 2 * ((i >> 1) + D); };
    auto reduce3 = [&](float x, float y, float z) {  // per-warp partials, combined in warp order
        x = warp_sum(x);
        y = warp_sum(y);
        z = warp_sum(z);
        if (lane == 0) {
            part[3 * warp] = x;
            part[3 * warp + 1] = y;
            part[3 * warp + 2] = z;
        }
    };
    auto total = [&](int c) {
        float s = 0.f;
        for (int v = 0; v < NW; ++v) s += part[3 * v + c];
        return s;
    };
    // component tid of sample j as stored (x_{2t+1}'s upper half is the negated real part: xsign)
    auto xc = [&](int j) {
        const bool ok = tid < L2 && j >= 0 && j < S;
        const bool up = tid >= M, odd = j & 1;
        const int mm = up ? tid - M : tid, comp = up ? (odd ? 0 : 1) : (odd ? 1 : 0);
        return ldg_if(ok, reinterpret_cast<const float *>(a.rx + (ok ? (size_t)(j >> 1) * M + mm : 0)) + comp);
    };
    auto xsign = [&](int j, float v) { return (tid >= M && (j & 1)) ? -v : v; };
    // target b_j of user k (real part for even j, imaginary for odd)
    auto target_at = [&](bool ok, int j) {
        return ldg_if(ok, reinterpret_cast<const float *>(a.sym + (ok ? (size_t)(j >> 1) * K + k : 0)) + (j & 1));
    };

    for (int i = tid; i < S; i += T) {
        gam[i] = 0.f;
        nrm[i] = a.ltab[(size_t)i * a.Sp + i];  // ||x_i||^2
    }
    for (int m = tid; m < M; m += T) {
        const float2 c = a.clin0 ? a.clin0[m * K + k] : make_float2(0.f, 0.f);
        w[m] = c.x;  // w = [Re c; Im c]
        w[M + m] = c.y;
    }
    RowPf pf;
    BandPf bp;
    float xn = 0.f;
    if (a.mode & 1) {
        sW = pmod(-W - 1, W);
        sR = pmod(-W - 1, WR);
        band_fetch(bp, a, S, W, 0, -W);
        band_store(bp, kg, kd, kl, S, W, 0, -W, slotR(0, 0), slotR(0, -W));
        band_fetch(bp, a, S, W, 1, 1 - W);
        if (S > 1) row_fetch(pf, a.gtab + a.Sp, a.gdtab + a.Sp, first_centre(1), 1);
        if (tid < L2) xw[slotR(0, 0) * L2 + tid] = xcomp(a.rx, M, 0, tid);
        xn = xc(1);
        float bn = target_at(tid == T - 1 && S > 1, 1);  // the target of the next arrival, a step early
        if (tid == 0) pb[0] = target_at(true, 0);
        __syncthreads();

        // ---- forward: sample 0 arrives with no live centre --------------------------------------------
        reduce3(0.f, 0.f, tid < L2 ? w[tid] * xw[slotR(0, 0) * L2 + tid] : 0.f);
        __syncthreads();
        if (tid == 0) {
            py[0] = 0.f;
            pd[0] = 0.f;
            pw[0] = total(2);
        }
        __syncthreads();
        for (int n = 0; n < S; ++n, sW = ring_slot(sW, 1, W), sR = ring_slot(sR, 1, WR)) {
            const int jlo = max(0, n - W + 1), nJ = n - jlo + 1, jn = n + 1;
            const float mq = nJ == W ? mqW : a.mu / (float)nJ;
            const float b_jn = bn;
            if (warp == NW - 1) bn = target_at(tid == T - 1 && jn + 1 < S, jn + 1);
            // the next sample's prediction from the live centres, before this step's update
            if (jn < S) {
                if (tid <= W) {
                    band_store(bp, kg, kd, kl, S, W, jn, jn - W, slotR(n, jn), slotR(n, jn - W));
                    band_fetch(bp, a, S, W, jn + 1, jn + 1 - W);
                }
                float ws = 0.f;
                if (tid < L2) {
                    const float x = xsign(jn, xn);
                    xw[slotR(n, jn) * L2 + tid] = x;
                    ws = w[tid] * x;
                    xn = xc(jn + 1);
                }
                const int lo = first_centre(jn);
                const float *grow = a.gtab + (size_t)jn * a.Sp, *drow = a.gdtab + (size_t)jn * a.Sp;
                float ys = 0.f, ds = 0.f;
#pragma unroll
                for (int q = 0; q < kPf; ++q) {
                    const int i = lo + tid + q * T;
                    if (i < jn) {
                        ys = fmaf(gam[i], pf.g[q], ys);
                        ds = fmaf(gam[i], pf.d[q], ds);
                    }
                }
                for (int i = lo + tid + kPf * T; i < jn; i += T) {
                    ys = fmaf(gam[i], __ldg(grow + i), ys);
                    ds = fmaf(gam[i], __ldg(drow + i), ds);
                }
                reduce3(ys, ds, ws);
                if (jn + 1 < S)
                    row_fetch(pf, a.gtab + (size_t)(jn + 1) * a.Sp, a.gdtab + (size_t)(jn + 1) * a.Sp,
                              first_centre(jn + 1), jn + 1);
            }
            // the window's projections (Eq. beta), all from f_n
            if (tid < nJ) {
                const int j = jlo + tid, r = slotW(n, j);
                const float dw = pw[r], yg = py[r], gd = pd[r];
                const float y = fmaf(a.wL, dw, a.wG * yg);
                const float e = y - pb[r];
                const float kap = fmaf(a.wL, nrm[j], a.wG);
                float beta = 0.f, s = 0.f;
                if (kap != 0.f) {
                    if (e < -a.eps) { s = 1.f; beta = (-e - a.eps) / kap; }
                    else if (e > a.eps) { s = -1.f; beta = (-e + a.eps) / kap; }
                }
                tape[(size_t)n * W + tid] = Tape{beta, s, kap, dw, yg, gd};
                ca[tid] = mq * beta;
                cb[tid] = gam[j] + mq * beta;  // the coefficient after the step
            }
            __syncthreads();
            // Eq. apsm: coefficients, linear part, and the carried predictions of J_{n+1}.  With
            // 2D = W + 1 the oldest centre of J_n leaves before step n+1: the arrival jn takes no term
            // of it, and the other samples drop its coefficient after this step's update.
            if (tid < nJ) gam[jlo + tid] = cb[tid];
            if (tid == T - 1 && jn < S) pb[slotW(n, jn)] = b_jn;
            const int t_lo = max(0, n - W + 2), n_t = jn < S ? jn - t_lo + 1 : 0;
            const int e_lo = first_centre(n), e_hi = jn < S ? first_centre(jn) : e_lo;  // leave before step n+1
            const int s_lo = slotR(n, jlo);
            for (int u = tid; u < L2 + n_t; u += T) {
                if (u < L2) {
                    float acc = w[u];
                    int si = s_lo;
#pragma unroll 4
                    for (int o = 0; o < nJ; ++o, si = ring_slot(si, 1, WR)) acc = fmaf(ca[o], xw[si * L2 + u], acc);
                    w[u] = acc;
                } else {
                    const int j = t_lo + (u - L2), r = slotW(n, j), sj = slotR(n, j) * WR;
                    float ay, ad, aw;
                    if (j == jn) {
                        ay = total(0);
                        ad = total(1);
                        aw = total(2);
                    } else {
                        ay = py[r];
                        ad = pd[r];
                        aw = pw[r];
                    }
                    const int o_lo = j == jn ? max(0, e_hi - jlo) : 0;  // sources still live at jn
                    int si = s_lo;
#pragma unroll 4
                    for (int o = 0; o < nJ; ++o, si = ring_slot(si, 1, WR)) {
                        const float c = ca[o];
                        aw = fmaf(c, kl[sj + si], aw);
                        if (o >= o_lo) {
                            ay = fmaf(c, kg[sj + si], ay);
                            ad = fmaf(c, kd[sj + si], ad);
                        }
                    }
                    if (j != jn) {
                        const float *grow = a.gtab + (size_t)j * a.Sp, *drow = a.gdtab + (size_t)j * a.Sp;
                        for (int i = e_lo; i < e_hi; ++i) {  // centres leaving before step n+1
                            const float gi = i >= jlo ? cb[i - jlo] : gam[i];
                            ay = fmaf(-gi, __ldg(grow + i), ay);
                            ad = fmaf(-gi, __ldg(drow + i), ad);
                        }
                    }
                    py[r] = ay;
                    pd[r] = ad;
                    pw[r] = aw;
                }
            }
            __syncthreads();
        }

    }  // forward
    if (!(a.mode & 2)) return;

    // ---- reverse sweep: R = 0, wbar = dL/dw of the final state ------------------------------------
    __syncthreads();
    {  // kernel values and components of the last W + 1 samples (as the forward left them)
        const int j0 = max(0, S - W - 1), nr = S - j0;
        for (int t = tid; t < nr * nr; t += T) {
            const int i = j0 + t / nr, j = j0 + t % nr;
            const size_t x = (size_t)i * a.Sp + j;
            const int u = (i % WR) * WR + j % WR;
            kg[u] = a.gtab[x];
            kl[u] = a.ltab[x];
        }
        for (int t = tid; t < nr * L2; t += T) {
            const int j = j0 + t / L2, m = t % L2;
            xw[(j % WR) * L2 + m] = xcomp(a.rx, M, j, m);
        }
    }
    for (int i = tid; i < S; i += T) gam[i] = 0.f;
    for (int m = tid; m < M; m += T) {
        const float2 d = a.dclin[m * K + k];
        w[m] = d.x;
        w[M + m] = d.y;
    }
    const int alive0 = max(0, P - D);  // first pilot whose entry is held at the end
    auto final_at = [&](int j) {       // adjoint of the final coefficient of sample j (0 if evicted)
        const bool ok = j >= 0 && (j >> 1) >= alive0;
        return ldg_if(ok, a.dgamma + (ok ? ((size_t)((j >> 1) % D) * 2 + (j & 1)) * K + k : 0));
    };
    // centres with a nonzero R when the entrant n - W is pulled at step n (none when it is not alive
    // in any step after n)
    auto pull_hi = [&](int n) {
        const int e = evict_step(n - W);
        return e > n + 1 ? min(e, S) : n - W + 2;
    };
    __syncthreads();
    for (int j = max(0, S - W) + tid; j < S; j += T) {  // abar of the last window
        float d = 0.f;
        for (int m = 0; m < L2; ++m) d = fmaf(w[m], xcomp(a.rx, M, j, m), d);
        py[j % W] = d + final_at(j);
    }
    const int je0 = S - 1 - W;  // the first entrant
    if (je0 >= 0) row_fetch(pf, a.gtab + (size_t)je0 * a.Sp, nullptr, je0 + 2, pull_hi(S - 1));
    band_fetch(bp, a, S, W, je0, je0);
    xn = xc(je0);
    const int t_fa = L2 % T;  // the thread that updates the entrant's abar
    float fa = tid == t_fa ? final_at(je0) : 0.f;  // the entrant's final adjoint, a step early
    Tape tnext;
    auto tape_at = [&](Tape &t, bool ok, int n) {
        const float *f = reinterpret_cast<const float *>(tape + (ok ? (size_t)n * W + tid : 0));
        const float2 u0 = ld2_if(ok, f), u1 = ld2_if(ok, f + 2), u2 = ld2_if(ok, f + 4);
        t = Tape{u0.x, u0.y, u1.x, u1.y, u2.x, u2.y};
    };
    if (tid < W) tape_at(tnext, tid < S - max(0, S - W), S - 1);
    sW = pmod(S - 1 - W - 1, W);
    sR = pmod(S - 1 - W - 1, WR);
    __syncthreads();
    // scalar adjoints: thread o sums the terms of window slot o over all steps (fixed order)
    float sig_bar = 0.f, mu_bar = 0.f, eps_bar = 0.f, wl_bar = 0.f;
    for (int n = S - 1; n >= 0; --n, sW = ring_slot(sW, W - 1, W), sR = ring_slot(sR, WR - 1, WR)) {
        const int jlo = max(0, n - W + 1), nJ = n - jlo + 1, je = n - W;
        const float q = nJ == W ? qW : 1.f / (float)nJ;
        float fa_je = 0.f;
        if (tid == t_fa) {
            fa_je = fa;
            fa = final_at(je - 1);
        }
        // R after the steps >= e, kept for the centres whose entry leaves at step e = n + 1
        if (((n + 1) & 1) == 0 && n + 1 <= S - 1 && ((n + 1) >> 1) >= D && tid < W - 1) {
            const int e = n + 1;
            snap[(size_t)((e >> 1) - D) * W + tid] = gam[e - W + 1 + tid];
        }
        // the entrant's pull: sum_j R_j kappa_G(x_je, x_j) over the steps after n in which it is alive,
        // and <wbar, x_je>, both before this step's terms
        if (je >= 0) {
            if (tid <= W) {
                band_store(bp, kg, kd, kl, S, W, je, je, slotR(n, je), slotR(n, je));
                band_fetch(bp, a, S, W, je - 1, je - 1);
            }
            float ls = 0.f;
            if (tid < L2) {
                const float x = xsign(je, xn);
                xw[slotR(n, je) * L2 + tid] = x;
                ls = w[tid] * x;
                xn = xc(je - 1);
            }
            const int lo = je + 2, hi = pull_hi(n), e = evict_step(je);
            const int s_lo = e <= S - 1 ? e - W + 1 : S;  // centres whose R holds steps >= e
            const float *sv = snap + (size_t)((e >> 1) - D) * W;
            const float *grow = a.gtab + (size_t)je * a.Sp;
            float gs = 0.f;
#pragma unroll
            for (int qq = 0; qq < kPf; ++qq) {
                const int i = lo + tid + qq * T;
                if (i < hi) gs = fmaf(i >= s_lo ? gam[i] - sv[i - s_lo] : gam[i], pf.g[qq], gs);
            }
            for (int i = lo + tid + kPf * T; i < hi; i += T)
                gs = fmaf(i >= s_lo ? gam[i] - sv[i - s_lo] : gam[i], __ldg(grow + i), gs);
            reduce3(gs, ls, 0.f);
            if (je - 1 >= 0) row_fetch(pf, a.gtab + (size_t)(je - 1) * a.Sp, nullptr, je + 1, pull_hi(n - 1));
        }
        if (tid < nJ) {  // slot tid: its scalar terms and its coefficients for the state adjoint
            const Tape tp = tnext;
            tape_at(tnext, n > 0 && tid < n - max(0, n - W), n - 1);
            const int o = tid, j = jlo + o;
            const float ab = py[slotW(n, j)];
            mu_bar += q * tp.beta * ab;
            const float bbar = a.mu * q * ab;
            float cwo = 0.f, cgo = 0.f;
            if (tp.s != 0.f) {  // inside the slab beta does not depend on the state
                const float ybar = -bbar / tp.kappa;
                eps_bar += tp.s * ybar;
                wl_bar += (ybar * tp.beta) * (nrm[j] - 1.f);
                wl_bar += ybar * (tp.dotw - tp.gauss);
                sig_bar += ybar * a.wG * tp.gd2 * inv_s3;
                cwo = ybar * a.wL;
                cgo = ybar * a.wG;
            }
            ca[o] = cwo;
            cb[o] = cgo;
        } else if (tid < W) {
            tape_at(tnext, n > 0 && tid < n - max(0, n - W), n - 1);
        }
        __syncthreads();
        // adjoint of S_n: R, wbar, and abar of the samples of J_{n-1}
        if (tid < nJ) gam[jlo + tid] += cb[tid];
        const int t_lo = max(0, n - W), n_t = n - t_lo;
        const int s_lo = slotR(n, jlo);
        for (int u = tid; u < L2 + n_t; u += T) {
            if (u < L2) {
                float acc = w[u];
                int si = s_lo;
#pragma unroll 4
                for (int o = 0; o < nJ; ++o, si = ring_slot(si, 1, WR)) acc = fmaf(ca[o], xw[si * L2 + u], acc);
                w[u] = acc;
            } else {
                const int j = t_lo + (u - L2), r = slotW(n, j), sj = slotR(n, j) * WR;
                float acc;
                bool alive = true;  // centres of J_{n-1} other than the entrant are alive at step n
                if (j == je) {
                    acc = fa_je + total(0) + total(1);
                    alive = n < evict_step(j);
                } else {
                    acc = py[r];
                }
                int si = s_lo;
#pragma unroll 4
                for (int o = 0; o < nJ; ++o, si = ring_slot(si, 1, WR)) {
                    acc = fmaf(ca[o], kl[sj + si], acc);
                    if (alive) acc = fmaf(cb[o], kg[sj + si], acc);
                }
                py[r] = acc;
            }
        }
        __syncthreads();
    }

    // ---- results -------------------------------------------------------------------------------------
    for (int m = tid; m < M; m += T) a.dclin0[m * K + k] = make_float2(w[m], w[M + m]);
    float *red = py;  // py, pd, pw, ca: 4 W floats, free now
    if (tid < W) {
        red[4 * tid + 0] = sig_bar;
        red[4 * tid + 1] = mu_bar;
        red[4 * tid + 2] = eps_bar;
        red[4 * tid + 3] = wl_bar;
    }
    __syncthreads();
    if (tid < 4) {
        float s = 0.f;
        for (int o = 0; o < W; ++o) s += red[4 * o + tid];
        a.scal[k * 4 + tid] = s;
    }
}

// ---- one warp per user -------------------------------------------------------------------------
// The same recurrence and adjoint as train_bwd_kernel, for windows of at most 32 slots: one warp
// per user (lane o = window slot o), the users of one instance in one CTA, and no block barrier
// inside the step loop -- each step synchronises one warp only.  The O(S) sums of a step take
// 4 kPfV entries per lane (float4 loads) from registers loaded a step ahead (the rest directly).
constexpr int kPfV = 4;  // float4 of a row per lane and table fetched a step ahead (512 entries)

__device__ __forceinline__ float4 ldg4_if(bool c, const float *p) {  // p 16-byte aligned
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %5, 0;\n\t@q ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];\n\t}"
                 : "+f"(v.x), "+f"(v.y), "+f"(v.z), "+f"(v.w)
                 : "l"(p), "r"((int)c));
    return v;
}

// Entries lo4 + 4 (lane + 32 q) + 0..3 (q < kPfV, lo4 = lo rounded down to a multiple of 4, the
// first of the four below hi) of one or two table rows (rows are padded to a multiple of 4 floats).
struct RowPfW {
    float4 g[kPfV], d[kPfV];
};

__device__ __forceinline__ void row_fetch_w(RowPfW &f, const float *grow, const float *drow, int lo, int hi, int lane) {
    const int lo4 = lo & ~3;
#pragma unroll
    for (int q = 0; q < kPfV; ++q) {
        const int i0 = lo4 + 4 * (lane + 32 * q);
        f.g[q] = ldg4_if(i0 < hi, grow + i0);
        f.d[q] = ldg4_if(drow != nullptr && i0 < hi, drow + i0);
    }
}

__device__ __forceinline__ float f4(const float4 &v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }

// band of row r, entries s0 + t for t = lane (and lane + 32 when W = 32), inside [0, S)
template <int NQ>
__device__ __forceinline__ void band_fetch_w(BandPf &b, const TrainBwdArgs &a, int S, int W, int r, int s0, int lane) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int t = lane + 32 * q, j = s0 + t;
        const bool ok = r >= 0 && r < S && t <= W && j >= 0 && j < S;
        const size_t x = ok ? (size_t)r * a.Sp + j : 0;
        b.g[q] = ldg_if(ok, a.gtab + x);
        b.d[q] = ldg_if(ok, a.gdtab + x);
        b.l[q] = ldg_if(ok, a.ltab + x);
    }
}

template <int NQ>
__device__ __forceinline__ void band_store_w(const BandPf &b, float *kg, float *kd, float *kl, int S, int W, int r,
                                             int s0, int sr, int s0r, int lane) {
    const int WR = W + 1;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int t = lane + 32 * q, j = s0 + t;
        if (r >= 0 && r < S && t <= W && j >= 0 && j < S) {
            const int sj = ring_slot(s0r, t, WR);
            const int u = sr * WR + sj, v = sj * WR + sr;
            kg[u] = b.g[q];
            kg[v] = b.g[q];
            kd[u] = b.d[q];
            kd[v] = b.d[q];
            kl[u] = b.l[q];
            kl[v] = b.l[q];
        }
    }
}

// floats of one warp's region: gamma / R [S rounded up to 4, zero padded], kg, kd, kl [(W+1)^2],
// xw [(W+1)][2M], py, pd, pw, pb, ca, cb [W], w / wbar [2M]
__host__ __device__ inline int bwd_warp_floats(int S, int W, int L2) {
    const int WR = W + 1;
    return (((S + 3) & ~3) + 3 * WR * WR + WR * L2 + 6 * W + L2 + 3) & ~3;
}

// WM: a bound on the window (8, 16 or 32) over which the O(W) loops are unrolled, so that their
// shared-memory loads are independent of one another.
template <int WM>
__global__ void __launch_bounds__(32 * kWarpUsersMax) train_bwd_warp_kernel(const TrainBwdArgs a0) {
    extern __shared__ __align__(16) float sm[];
    const TrainBwdArgs a = for_instance(a0, blockIdx.y);
    constexpr int NQ = WM >= 32 ? 2 : 1;  // band entries per lane (W + 1 <= 32 NQ)
    const int lane = threadIdx.x & 31, k = threadIdx.x >> 5;
    const int M = a.M, K = a.K, W = a.W, D = a.D, P = a.P, S = 2 * P, L2 = 2 * M, WR = W + 1;
    float *nrm = sm, *rk = nrm + ((S + 3) & ~3);  // ||x_j||^2 and 1 / kappa_jj, shared by the users
    float *gam = rk + ((S + 3) & ~3) + k * bwd_warp_floats(S, W, L2);
    const int S4 = (S + 3) & ~3;
    float *kg = gam + S4, *kd = kg + WR * WR, *kl = kd + WR * WR, *xw = kl + WR * WR;
    float *py = xw + WR * L2, *pd = py + W, *pw = pd + W, *pb = pw + W, *ca = pb + W, *cb = ca + W, *w = cb + W;
    Tape *tape = a.tape + (size_t)k * S * W;
    float *snap = a.snap + (size_t)k * (P > D ? P - D : 0) * W;
    const float inv_s3 = 1.f / (a.sigma * a.sigma * a.sigma);
    const float mqW = a.mu / (float)W, qW = 1.f / (float)W;
    auto pmod = [](int x, int R) { return ((x % R) + R) % R; };
    int sW = 0, sR = 0;  // slots of the reference sample n - W - 1 (mod W, mod W + 1)
    auto slotW = [&](int n, int j) { return ring_slot(sW, j - (n - W - 1), W); };
    auto slotR = [&](int n, int j) { return ring_slot(sR, j - (n - W - 1), WR); };
    auto first_centre = [&](int n) { return 2 * max(0, (n >> 1) - D + 1); };
    auto evict_step = [&](int i) { return 2 * ((i >> 1) + D); };
    // component m of sample j as stored, and its sign (x_{2t+1}'s upper half is -Re r)
    auto xc = [&](int j, int m) {
        const bool ok = m < L2 && j >= 0 && j < S;
        const bool up = m >= M, odd = j & 1;
        const int mm = up ? m - M : m, comp = up ? (odd ? 0 : 1) : (odd ? 1 : 0);
        return ldg_if(ok, reinterpret_cast<const float *>(a.rx + (ok ? (size_t)(j >> 1) * M + mm : 0)) + comp);
    };
    auto xsign = [&](int j, int m, float v) { return (m >= M && (j & 1)) ? -v : v; };
    auto wrap = [&](int x) { return x >= WR ? x - WR : x; };  // x < 2 (W + 1)
    auto target_at = [&](bool ok, int j) {
        return ldg_if(ok, reinterpret_cast<const float *>(a.sym + (ok ? (size_t)(j >> 1) * K + k : 0)) + (j & 1));
    };

    for (int i = threadIdx.x; i < S; i += blockDim.x) {
        nrm[i] = a.ltab[(size_t)i * a.Sp + i];  // ||x_i||^2
        const float kap = fmaf(a.wL, nrm[i], a.wG);
        rk[i] = kap != 0.f ? 1.f / kap : 0.f;
    }
    __syncthreads();  // the only block barrier: nrm and rk are shared by the users
    for (int i = lane; i < S4; i += 32) gam[i] = 0.f;
    for (int m = lane; m < M; m += 32) {
        const float2 c = a.clin0 ? a.clin0[m * K + k] : make_float2(0.f, 0.f);
        w[m] = c.x;
        w[M + m] = c.y;
    }
    RowPfW pf;
    BandPf bp;
    float xn[4];
    if (a.mode & 1) {
        sW = pmod(-W - 1, W);
        sR = pmod(-W - 1, WR);
        band_fetch_w<NQ>(bp, a, S, W, 0, -W, lane);
        band_store_w<NQ>(bp, kg, kd, kl, S, W, 0, -W, slotR(0, 0), slotR(0, -W), lane);
        band_fetch_w<NQ>(bp, a, S, W, 1, 1 - W, lane);
        if (S > 1) row_fetch_w(pf, a.gtab + a.Sp, a.gdtab + a.Sp, first_centre(1), 1, lane);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int m = lane + 32 * c;
            if (m < L2) xw[slotR(0, 0) * L2 + m] = xcomp(a.rx, M, 0, m);
            xn[c] = xc(1, m);
        }
        float bn = target_at(lane == 0 && S > 1, 1);  // the next arrival's target, a step early
        if (lane == 0) pb[0] = target_at(true, 0);
        __syncwarp();
        {
            float ws = 0.f;
            for (int m = lane; m < L2; m += 32) ws = fmaf(w[m], xw[slotR(0, 0) * L2 + m], ws);
            ws = warp_sum(ws);
            if (lane == 0) {
                py[0] = 0.f;
                pd[0] = 0.f;
                pw[0] = ws;
            }
        }
        __syncwarp();

        // ---- forward ---------------------------------------------------------------------------------------
        for (int n = 0; n < S; ++n, sW = ring_slot(sW, 1, W), sR = ring_slot(sR, 1, WR)) {
            const int jlo = max(0, n - W + 1), nJ = n - jlo + 1, jn = n + 1;
            const float mq = nJ == W ? mqW : a.mu / (float)nJ;
            const float b_jn = bn;
            bn = target_at(lane == 0 && jn + 1 < S, jn + 1);
            float ys = 0.f, ds = 0.f, ws = 0.f;  // the arrival's sums from the state before this step
            if (jn < S) {
                band_store_w<NQ>(bp, kg, kd, kl, S, W, jn, jn - W, slotR(n, jn), slotR(n, jn - W), lane);
                band_fetch_w<NQ>(bp, a, S, W, jn + 1, jn + 1 - W, lane);
                const int sx = slotR(n, jn) * L2;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int m = lane + 32 * c;
                    if (m < L2) {
                        const float x = xsign(jn, m, xn[c]);
                        xw[sx + m] = x;
                        ws = fmaf(w[m], x, ws);
                        xn[c] = xc(jn + 1, m);
                    }
                }
                const int lo = first_centre(jn), lo4 = lo & ~3;
                float y2[2] = {0.f, 0.f}, d2[2] = {0.f, 0.f};  // two chains of sums
                if (lo == 0) {  // nothing evicted yet: gamma is zero from jn on (padding included)
#pragma unroll
                    for (int q = 0; q < kPfV; ++q) {
                        const int i0 = 4 * (lane + 32 * q);
                        if (i0 < jn) {
                            const float4 gm = *reinterpret_cast<const float4 *>(gam + i0);
                            y2[0] = fmaf(gm.x, pf.g[q].x, fmaf(gm.z, pf.g[q].z, y2[0]));
                            y2[1] = fmaf(gm.y, pf.g[q].y, fmaf(gm.w, pf.g[q].w, y2[1]));
                            d2[0] = fmaf(gm.x, pf.d[q].x, fmaf(gm.z, pf.d[q].z, d2[0]));
                            d2[1] = fmaf(gm.y, pf.d[q].y, fmaf(gm.w, pf.d[q].w, d2[1]));
                        }
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < kPfV; ++q) {
                        const int i0 = lo4 + 4 * (lane + 32 * q);
                        if (i0 < jn) {
                            const float4 gm = *reinterpret_cast<const float4 *>(gam + i0);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int i = i0 + e;
                                if (i >= lo && i < jn) {
                                    y2[e & 1] = fmaf(f4(gm, e), f4(pf.g[q], e), y2[e & 1]);
                                    d2[e & 1] = fmaf(f4(gm, e), f4(pf.d[q], e), d2[e & 1]);
                                }
                            }
                        }
                    }
                }
                const float *grow = a.gtab + (size_t)jn * a.Sp, *drow = a.gdtab + (size_t)jn * a.Sp;
                for (int i = max(lo, lo4 + 4 * 32 * kPfV) + lane; i < jn; i += 32) {
                    y2[0] = fmaf(gam[i], __ldg(grow + i), y2[0]);
                    d2[0] = fmaf(gam[i], __ldg(drow + i), d2[0]);
                }
                ys = y2[0] + y2[1];
                ds = d2[0] + d2[1];
                if (jn + 1 < S)
                    row_fetch_w(pf, a.gtab + (size_t)(jn + 1) * a.Sp, a.gdtab + (size_t)(jn + 1) * a.Sp,
                                first_centre(jn + 1), jn + 1, lane);
                ys = warp_sum(ys);
                ds = warp_sum(ds);
                ws = warp_sum(ws);
            }
            if (lane < nJ) {  // the window's projections (Eq. beta), all from f_n
                const int j = jlo + lane, r = slotW(n, j);
                const float dw = pw[r], yg = py[r], gd = pd[r];
                const float y = fmaf(a.wL, dw, a.wG * yg);
                const float e = y - pb[r];
                const float kap = fmaf(a.wL, nrm[j], a.wG), r_k = rk[j];
                float beta = 0.f, s = 0.f;
                if (kap != 0.f) {
                    if (e < -a.eps) { s = 1.f; beta = (-e - a.eps) * r_k; }
                    else if (e > a.eps) { s = -1.f; beta = (-e + a.eps) * r_k; }
                }
                tape[(size_t)n * W + lane] = Tape{beta, s, kap, dw, yg, gd};
                ca[lane] = mq * beta;
                cb[lane] = gam[j] + mq * beta;  // the coefficient after the step
            }
            __syncwarp();
            // Eq. apsm: coefficients, linear part, carried predictions of J_{n+1} (2D = W + 1: the oldest
            // centre of J_n leaves before step n+1)
            if (lane < nJ) gam[jlo + lane] = cb[lane];
            if (lane == 0 && jn < S) pb[slotW(n, jn)] = b_jn;
            const int s_lo = slotR(n, jlo);
            for (int m = lane; m < L2; m += 32) {
                float acc = w[m];
#pragma unroll
                for (int o = 0; o < WM; ++o)
                    if (o < nJ) acc = fmaf(ca[o], xw[wrap(s_lo + o) * L2 + m], acc);
                w[m] = acc;
            }
            const int t_lo = max(0, n - W + 2), n_t = jn < S ? jn - t_lo + 1 : 0;
            const int e_lo = first_centre(n), e_hi = jn < S ? first_centre(jn) : e_lo;
            if (lane < n_t) {
                const int j = t_lo + lane, r = slotW(n, j), sj = slotR(n, j) * WR;
                float ay, ad, aw;
                if (j == jn) {
                    ay = ys;
                    ad = ds;
                    aw = ws;
                } else {
                    ay = py[r];
                    ad = pd[r];
                    aw = pw[r];
                }
                const int o_lo = j == jn ? max(0, e_hi - jlo) : 0;
#pragma unroll
                for (int o = 0; o < WM; ++o) {
                    if (o < nJ) {
                        const int si = sj + wrap(s_lo + o);
                        const float c = ca[o];
                        aw = fmaf(c, kl[si], aw);
                        if (o >= o_lo) {
                            ay = fmaf(c, kg[si], ay);
                            ad = fmaf(c, kd[si], ad);
                        }
                    }
                }
                if (j != jn) {
                    const float *grow = a.gtab + (size_t)j * a.Sp, *drow = a.gdtab + (size_t)j * a.Sp;
                    for (int i = e_lo; i < e_hi; ++i) {
                        const float gi = i >= jlo ? cb[i - jlo] : gam[i];
                        ay = fmaf(-gi, __ldg(grow + i), ay);
                        ad = fmaf(-gi, __ldg(drow + i), ad);
                    }
                }
                py[r] = ay;
                pd[r] = ad;
                pw[r] = aw;
            }
            __syncwarp();
        }

    }  // forward
    if (!(a.mode & 2)) return;

    // ---- reverse sweep ---------------------------------------------------------------------------------
    {  // kernel values and components of the last W + 1 samples (as the forward left them)
        const int j0 = max(0, S - W - 1), nr = S - j0;
        for (int t = lane; t < nr * nr; t += 32) {
            const int i = j0 + t / nr, j = j0 + t % nr;
            const size_t x = (size_t)i * a.Sp + j;
            const int u = (i % WR) * WR + j % WR;
            kg[u] = a.gtab[x];
            kl[u] = a.ltab[x];
        }
        for (int t = lane; t < nr * L2; t += 32) {
            const int j = j0 + t / L2, m = t % L2;
            xw[(j % WR) * L2 + m] = xcomp(a.rx, M, j, m);
        }
    }
    __syncwarp();
    for (int i = lane; i < S4; i += 32) gam[i] = 0.f;  // R
    for (int m = lane; m < M; m += 32) {
        const float2 d = a.dclin[m * K + k];
        w[m] = d.x;
        w[M + m] = d.y;
    }
    const int alive0 = max(0, P - D);
    auto final_at = [&](int j) {
        const bool ok = j >= 0 && (j >> 1) >= alive0;
        int t = j >> 1;  // its ring slot: t mod D (t < D unless entries were evicted)
        if (P > D) t %= D;
        return ldg_if(ok, a.dgamma + (ok ? ((size_t)t * 2 + (j & 1)) * K + k : 0));
    };
    auto pull_hi = [&](int n) {
        const int e = evict_step(n - W);
        return e > n + 1 ? min(e, S) : n - W + 2;
    };
    __syncwarp();
    for (int j = max(0, S - W) + lane; j < S; j += 32) {  // abar of the last window (xw holds them)
        float d = 0.f;
        const int sx = pmod(j, WR) * L2;
        for (int m = 0; m < L2; ++m) d = fmaf(w[m], xw[sx + m], d);
        py[j % W] = d + final_at(j);
    }
    const int je0 = S - 1 - W;
    if (je0 >= 0) row_fetch_w(pf, a.gtab + (size_t)je0 * a.Sp, nullptr, je0 + 2, pull_hi(S - 1), lane);
    band_fetch_w<NQ>(bp, a, S, W, je0, je0, lane);
#pragma unroll
    for (int c = 0; c < 4; ++c) xn[c] = xc(je0, lane + 32 * c);
    float fa = final_at(je0);  // every lane: the entrant's final adjoint, a step early
    Tape tnext;
    auto tape_at = [&](Tape &t, bool ok, int n) {
        const float *f = reinterpret_cast<const float *>(tape + (ok ? (size_t)n * W + lane : 0));
        const float2 u0 = ld2_if(ok, f), u1 = ld2_if(ok, f + 2), u2 = ld2_if(ok, f + 4);
        t = Tape{u0.x, u0.y, u1.x, u1.y, u2.x, u2.y};
    };
    tape_at(tnext, lane < S - max(0, S - W), S - 1);
    sW = pmod(S - 1 - W - 1, W);
    sR = pmod(S - 1 - W - 1, WR);
    __syncwarp();
    float sig_bar = 0.f, mu_bar = 0.f, eps_bar = 0.f, wl_bar = 0.f;  // lane o: window slot o's terms
    for (int n = S - 1; n >= 0; --n, sW = ring_slot(sW, W - 1, W), sR = ring_slot(sR, WR - 1, WR)) {
        const int jlo = max(0, n - W + 1), nJ = n - jlo + 1, je = n - W;
        const float q = nJ == W ? qW : 1.f / (float)nJ;
        const float fa_je = fa;
        fa = final_at(je - 1);
        if (((n + 1) & 1) == 0 && n + 1 <= S - 1 && ((n + 1) >> 1) >= D && lane < W - 1) {
            const int e = n + 1;  // R after the steps >= e, for the centres whose entry leaves at e
            snap[(size_t)((e >> 1) - D) * W + lane] = gam[e - W + 1 + lane];
        }
        float gs = 0.f, ls = 0.f;
        if (je >= 0) {
            band_store_w<NQ>(bp, kg, kd, kl, S, W, je, je, slotR(n, je), slotR(n, je), lane);
            band_fetch_w<NQ>(bp, a, S, W, je - 1, je - 1, lane);
            const int sx = slotR(n, je) * L2;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int m = lane + 32 * c;
                if (m < L2) {
                    const float x = xsign(je, m, xn[c]);
                    xw[sx + m] = x;
                    ls = fmaf(w[m], x, ls);
                    xn[c] = xc(je - 1, m);
                }
            }
            const int lo = je + 2, hi = pull_hi(n), e = evict_step(je);
            const int s_lo = e <= S - 1 ? e - W + 1 : S;
            const float *sv = snap + (size_t)((e >> 1) - D) * W;
            const float *grow = a.gtab + (size_t)je * a.Sp;
            const int lo4 = lo & ~3;
            float g2[2] = {0.f, 0.f};
            if (hi == S && s_lo >= S) {  // no eviction after the entrant: R is zero below lo and past S
#pragma unroll
                for (int qq = 0; qq < kPfV; ++qq) {
                    const int i0 = lo4 + 4 * (lane + 32 * qq);
                    if (i0 < hi) {
                        const float4 rm = *reinterpret_cast<const float4 *>(gam + i0);
                        g2[0] = fmaf(rm.x, pf.g[qq].x, fmaf(rm.z, pf.g[qq].z, g2[0]));
                        g2[1] = fmaf(rm.y, pf.g[qq].y, fmaf(rm.w, pf.g[qq].w, g2[1]));
                    }
                }
            } else {
#pragma unroll
                for (int qq = 0; qq < kPfV; ++qq) {
                    const int i0 = lo4 + 4 * (lane + 32 * qq);
                    if (i0 < hi) {
                        const float4 rm = *reinterpret_cast<const float4 *>(gam + i0);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int i = i0 + e;
                            if (i >= lo && i < hi) {
                                const float r = i >= s_lo ? f4(rm, e) - sv[i - s_lo] : f4(rm, e);
                                g2[e & 1] = fmaf(r, f4(pf.g[qq], e), g2[e & 1]);
                            }
                        }
                    }
                }
            }
            for (int i = max(lo, lo4 + 4 * 32 * kPfV) + lane; i < hi; i += 32)
                g2[0] = fmaf(i >= s_lo ? gam[i] - sv[i - s_lo] : gam[i], __ldg(grow + i), g2[0]);
            gs = g2[0] + g2[1];
            if (je - 1 >= 0) row_fetch_w(pf, a.gtab + (size_t)(je - 1) * a.Sp, nullptr, je + 1, pull_hi(n - 1), lane);
            gs = warp_sum(gs);
            ls = warp_sum(ls);
        }
        if (lane < nJ) {
            const Tape tp = tnext;
            tape_at(tnext, n > 0 && lane < n - max(0, n - W), n - 1);
            const int j = jlo + lane;
            const float ab = py[slotW(n, j)];
            mu_bar += q * tp.beta * ab;
            const float bbar = a.mu * q * ab;
            float cwo = 0.f, cgo = 0.f;
            if (tp.s != 0.f) {
                const float ybar = -bbar * rk[j];
                eps_bar += tp.s * ybar;
                wl_bar += (ybar * tp.beta) * (nrm[j] - 1.f);
                wl_bar += ybar * (tp.dotw - tp.gauss);
                sig_bar += ybar * a.wG * tp.gd2 * inv_s3;
                cwo = ybar * a.wL;
                cgo = ybar * a.wG;
            }
            ca[lane] = cwo;
            cb[lane] = cgo;
        }
        __syncwarp();
        if (lane < nJ) gam[jlo + lane] += cb[lane];
        const int s_lo = slotR(n, jlo);
        for (int m = lane; m < L2; m += 32) {
            float acc = w[m];
#pragma unroll
            for (int o = 0; o < WM; ++o)
                if (o < nJ) acc = fmaf(ca[o], xw[wrap(s_lo + o) * L2 + m], acc);
            w[m] = acc;
        }
        const int t_lo = max(0, n - W), n_t = n - t_lo;
        if (lane < n_t) {
            const int j = t_lo + lane, r = slotW(n, j), sj = slotR(n, j) * WR;
            float acc;
            bool alive = true;
            if (j == je) {
                acc = fa_je + gs + ls;
                alive = n < evict_step(j);
            } else {
                acc = py[r];
            }
#pragma unroll
            for (int o = 0; o < WM; ++o) {
                if (o < nJ) {
                    const int si = sj + wrap(s_lo + o);
                    acc = fmaf(ca[o], kl[si], acc);
                    if (alive) acc = fmaf(cb[o], kg[si], acc);
                }
            }
            py[r] = acc;
        }
        __syncwarp();
    }

    for (int m = lane; m < M; m += 32) a.dclin0[m * K + k] = make_float2(w[m], w[M + m]);
    // slot partials combined in slot order
    float *red = py;  // py, pd, pw, pb: 4 W floats
    if (lane < W) {
        red[4 * lane + 0] = sig_bar;
        red[4 * lane + 1] = mu_bar;
        red[4 * lane + 2] = eps_bar;
        red[4 * lane + 3] = wl_bar;
    }
    __syncwarp();
    if (lane < 4) {
        float s = 0.f;
        for (int o = 0; o < W; ++o) s += red[4 * o + lane];
        a.scal[k * 4 + lane] = s;
    }
}

__global__ void train_bwd_sum_kernel(const TrainBwdArgs a0) {
    const TrainBwdArgs a = for_instance(a0, blockIdx.y);
    if (threadIdx.x < 4) {
        float s = 0.f;
        for (int k = 0; k < a.K; ++k) s += a.scal[k * 4 + threadIdx.x];  // users in order
        a.dscalars[threadIdx.x] = s;
    }
}

size_t train_bwd_smem(int M, int W, int P) {
    return sizeof(float) * (size_t)(2 * 2 * P + 2 * M + 6 * W + 3 * (kBwdThreads / 32) + 3 * (W + 1) * (W + 1) +
                                    (W + 1) * 2 * M);
}

}  // namespace apsm

using namespace apsm;

namespace {

struct BwdLayout {
    size_t ltab, gtab, gdtab, tape, snap, scal, total;
};

BwdLayout bwd_layout(const apsm_params *p, int P) {
    BwdLayout b;
    const size_t S = 2 * (size_t)P;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t off = 0;
    const size_t Sp = (S + 3) & ~size_t(3);
    b.ltab = off;
    off = al(off + sizeof(float) * S * Sp);
    b.gtab = off;
    off = al(off + sizeof(float) * S * Sp);
    b.gdtab = off;
    off = al(off + sizeof(float) * S * Sp);
    b.tape = off;
    off = al(off + sizeof(Tape) * (size_t)p->K * S * p->window);
    b.snap = off;
    off = al(off + sizeof(float) * (size_t)p->K * (size_t)std::max(0, P - p->dict_cap) * p->window);
    b.scal = off;
    off = al(off + sizeof(float) * 4 * (size_t)p->K);
    b.total = off;
    return b;
}

}  // namespace

namespace {

// The calls of one batch of n instances (n = 1 for apsm_train_backward).  mode 1: the tables and
// the forward pass (the tape, kept in the workspace); 2: the reverse sweep over a workspace that
// mode 1 filled; 3: both.
apsm_status train_bwd_run(const apsm_params *p, int n, const float *rx_pilot, const float *sym_pilot, int32_t P,
                          const float *clin0, const float *dgamma, const float *dclin, float *dscalars, float *dclin0,
                          void *workspace, size_t workspace_bytes, void *stream, int mode) {
    size_t dummy = 0;
    apsm_status s = apsm_train_workspace_bytes(p, 0, &dummy);
    if (s != APSM_OK) return s;
    if (n < 1 || n > 65535 || P < 1 || !rx_pilot) return APSM_ERR_INVALID_ARG;
    if ((mode & 1) && !sym_pilot) return APSM_ERR_INVALID_ARG;
    if ((mode & 2) && (!dgamma || !dclin || !dscalars || !dclin0)) return APSM_ERR_INVALID_ARG;
    if (P > 8192) return APSM_ERR_UNSUPPORTED;
    if (p->weights != APSM_Q_UNIFORM) return APSM_ERR_UNSUPPORTED;  // the adjoint of q = 1/|J_n| only
    const BwdLayout b = bwd_layout(p, P);
    if (!workspace || workspace_bytes < b.total * (size_t)n) return APSM_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return APSM_ERR_INVALID_ARG;
    const size_t smem = train_bwd_smem(p->M, p->window, P);
    // one warp per user when the window fits the lanes and every user's rings fit one CTA
    const size_t smem_w =
        sizeof(float) * (2 * (size_t)((2 * P + 3) & ~3) + (size_t)p->K * bwd_warp_floats(2 * P, p->window, 2 * p->M));
    const bool warp_form = p->window <= 32 && smem_w <= 227 * 1024;
    if (!warp_form && smem > 227 * 1024) return APSM_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return APSM_ERR_CUDA;
    }
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return APSM_ERR_NOT_SM103;
    cudaStream_t strm = static_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    TrainBwdArgs a{};
    a.M = p->M;
    a.K = p->K;
    a.W = p->window;
    a.D = p->dict_cap;
    a.P = P;
    a.Sp = (2 * P + 3) & ~3;
    a.sigma = p->sigma;
    a.mu = p->mu;
    a.eps = p->eps;
    a.wL = p->w_L;
    a.wG = 1.f - p->w_L;
    a.k2 = kLog2e / (2.f * p->sigma * p->sigma);
    a.rx = reinterpret_cast<const float2 *>(rx_pilot);
    a.sym = reinterpret_cast<const float2 *>(sym_pilot);
    a.clin0 = reinterpret_cast<const float2 *>(clin0);
    a.dgamma = dgamma;
    a.dclin = reinterpret_cast<const float2 *>(dclin);
    a.ltab = reinterpret_cast<float *>(ws + b.ltab);
    a.gtab = reinterpret_cast<float *>(ws + b.gtab);
    a.gdtab = reinterpret_cast<float *>(ws + b.gdtab);
    a.tape = reinterpret_cast<Tape *>(ws + b.tape);
    a.snap = reinterpret_cast<float *>(ws + b.snap);
    a.scal = reinterpret_cast<float *>(ws + b.scal);
    a.dclin0 = reinterpret_cast<float2 *>(dclin0);
    a.dscalars = dscalars;
    a.st_rx = (size_t)P * p->M;
    a.st_sym = (size_t)P * p->K;
    a.st_clin0 = (size_t)p->M * p->K;
    a.st_dgamma = (size_t)round_up(p->dict_cap, kTileEntries) * 2 * p->K;
    a.st_mk = (size_t)p->M * p->K;
    a.ws_stride = b.total;
    a.mode = mode;
    const long long pairs = 2LL * P * a.Sp;
    const int blocks = (int)std::min<long long>(std::max(1, 4096 / n), (pairs + 255) / 256);
    if (mode & 1) train_bwd_tables_kernel<<<dim3(blocks, n), 256, 0, strm>>>(a);
    if (warp_form) {
        auto kern = p->window <= 8 ? train_bwd_warp_kernel<8>
                    : p->window <= 16 ? train_bwd_warp_kernel<16> : train_bwd_warp_kernel<32>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_w) != cudaSuccess)
            return APSM_ERR_CUDA;
        kern<<<dim3(1, n), 32 * p->K, smem_w, strm>>>(a);
    } else {
        if (cudaFuncSetAttribute(train_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return APSM_ERR_CUDA;
        train_bwd_kernel<<<dim3(p->K, n), kBwdThreads, smem, strm>>>(a);
    }
    if (mode & 2) train_bwd_sum_kernel<<<dim3(1, n), 32, 0, strm>>>(a);
    g_launches += 1 + (mode & 1) + ((mode & 2) >> 1);
    return cudaGetLastError() == cudaSuccess ? APSM_OK : APSM_ERR_CUDA;
}

}  // namespace

extern "C" {

apsm_status apsm_train_backward_workspace_bytes(const apsm_params *p, int32_t P, size_t *bytes) {
    return apsm_train_backward_batched_workspace_bytes(p, P, 1, bytes);
}

apsm_status apsm_train_backward_batched_workspace_bytes(const apsm_params *p, int32_t P, int32_t n, size_t *bytes) {
    size_t dummy = 0;
    apsm_status s = apsm_train_workspace_bytes(p, 0, &dummy);  // parameter validation
    if (s != APSM_OK) return s;
    if (!bytes || P < 0 || n < 1) return APSM_ERR_INVALID_ARG;
    *bytes = bwd_layout(p, P).total * (size_t)n;
    return APSM_OK;
}

apsm_status apsm_train_backward(const apsm_params *p, const float *rx_pilot, const float *sym_pilot, int32_t P,
                                const float *clin0, const float *dgamma, const float *dclin, float *dscalars,
                                float *dclin0, void *workspace, size_t workspace_bytes, void *stream) {
    return train_bwd_run(p, 1, rx_pilot, sym_pilot, P, clin0, dgamma, dclin, dscalars, dclin0, workspace,
                         workspace_bytes, stream, 3);
}

apsm_status apsm_train_backward_batched(const apsm_params *p, int32_t n, const float *rx_pilot, const float *sym_pilot,
                                        int32_t P, const float *clin0, const float *dgamma, const float *dclin,
                                        float *dscalars, float *dclin0, void *workspace, size_t workspace_bytes,
                                        void *stream) {
    return train_bwd_run(p, n, rx_pilot, sym_pilot, P, clin0, dgamma, dclin, dscalars, dclin0, workspace,
                         workspace_bytes, stream, 3);
}

apsm_status apsm_train_backward_batched_forward(const apsm_params *p, int32_t n, const float *rx_pilot,
                                                const float *sym_pilot, int32_t P, const float *clin0,
                                                void *workspace, size_t workspace_bytes, void *stream) {
    return train_bwd_run(p, n, rx_pilot, sym_pilot, P, clin0, nullptr, nullptr, nullptr, nullptr, workspace,
                         workspace_bytes, stream, 1);
}

apsm_status apsm_train_backward_batched_reverse(const apsm_params *p, int32_t n, const float *rx_pilot, int32_t P,
                                                const float *dgamma, const float *dclin, float *dscalars,
                                                float *dclin0, void *workspace, size_t workspace_bytes,
                                                void *stream) {
    return train_bwd_run(p, n, rx_pilot, nullptr, P, nullptr, dgamma, dclin, dscalars, dclin0, workspace,
                         workspace_bytes, stream, 2);
}

}  // extern "C"
