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
// Checkpointing: a first forward pass stores (w, every gamma) at the start of every segment of
// 32 pilots (64 steps); the reverse sweep restores each segment, re-runs its forward recording a
// per-step tape (beta, branch, kappa, <w, x_j>, gauss_j, its sigma weight), then walks it back.
// Kernel values between samples come from tables built once per call.  One CTA of 8 warps per
// user: a warp per window slot for the inner products, a thread per centre for the state
// adjoint's update, a thread per slot for the scalar terms (summed in slot order at the end).
#include <algorithm>
#include <atomic>
#include <cmath>

#include "apsm_common.cuh"
#include "train_f32.cuh"

namespace apsm {

extern std::atomic<long long> g_launches;  // apsm_api.cu

constexpr int kBwdSeg = 64;  // steps per checkpoint segment (32 pilots)

struct TrainBwdArgs {
    int M, K, W, D, P;
    float sigma, mu, eps, wL, wG, k2;
    const float2 *rx;       // [P][M]
    const float2 *sym;      // [P][K]
    const float2 *clin0;    // [M][K] or null
    const float *dgamma;    // [A][2][K] adjoint of the final coefficients (ring layout)
    const float2 *dclin;    // [M][K] adjoint of the final linear filter
    float *ltab;            // [2P][2P] x_i . x_j
    float *gtab;            // [2P][2P] kappa_G(x_i, x_j)
    float *ckpt;            // [K][n_seg][2M + 2P]
    float *scal;            // [K][4] per-user sigma, mu, eps, w_L adjoints
    float2 *dclin0;         // [M][K] out
    float *dscalars;        // [4] out
    int n_seg;
};

__global__ void train_bwd_tables_kernel(const TrainBwdArgs a) {
    const int S = 2 * a.P;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)S * S;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / S), j = (int)(idx % S);
        float dot, d2;
        sample_pair(a.rx + (size_t)(i >> 1) * a.M, a.rx + (size_t)(j >> 1) * a.M, a.M, i & 1, j & 1, dot, d2);
        a.ltab[idx] = dot;
        a.gtab[idx] = ex2(-a.k2 * d2);
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

struct Tape {  // one window slot of one step
    float beta, s, kappa, dotw, gauss, gd2;
};

constexpr int kBwdThreads = 256;  // 8 warps per user: one window slot per warp

// smem: gamma [2P], gbar [2P], norms [2P], w [2M], wbar [2M], abar [W], cw [W], cg [W],
//       tape [kBwdSeg][W]
__global__ void __launch_bounds__(kBwdThreads) train_bwd_kernel(const TrainBwdArgs a) {
    extern __shared__ __align__(16) float sm[];
    const int k = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kBwdThreads / 32;
    const int M = a.M, K = a.K, W = a.W, D = a.D, P = a.P, S = 2 * P, L2 = 2 * M;
    float *gam = sm, *gbar = gam + S, *nrm = gbar + S, *w = nrm + S, *wbar = w + L2, *abar = wbar + L2;
    float *cw = abar + W, *cg = cw + W;
    Tape *tape = reinterpret_cast<Tape *>(cg + W);
    const float inv_s3 = 1.f / (a.sigma * a.sigma * a.sigma);

    auto target = [&](int j) {
        const float2 b = __ldg(a.sym + (size_t)(j >> 1) * K + k);
        return (j & 1) ? b.y : b.x;
    };
    auto first_centre = [&](int n) { return 2 * max(0, (n >> 1) - D + 1); };
    for (int i = tid; i < S; i += kBwdThreads) nrm[i] = a.ltab[(size_t)i * S + i];  // ||x_i||^2

    // ---- forward over one segment (warp o takes window slots o, o + 8, ...); records the tape --
    auto forward = [&](int n0, int n1) {
        for (int n = n0; n < n1; ++n) {
            const int c_lo = first_centre(n), c_hi = 2 * (n >> 1) + 2;
            const int jlo = max(0, n - W + 1), nJ = n - jlo + 1;
            for (int o = warp; o < nJ; o += NW) {
                const int j = jlo + o;
                float dw = 0.f;
                for (int m = lane; m < L2; m += 32) dw = fmaf(w[m], xcomp(a.rx, M, j, m), dw);
                const float nj = nrm[j];
                const float *grow = a.gtab + (size_t)j * S, *lrow = a.ltab + (size_t)j * S;
                float gs[4] = {0.f, 0.f, 0.f, 0.f}, gd[4] = {0.f, 0.f, 0.f, 0.f};
                int i = c_lo + lane;
                for (; i + 96 < c_hi; i += 128) {  // four centres per lane in flight
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int ii = i + 32 * q;
                        const float g = __ldg(grow + ii), lt = __ldg(lrow + ii), gi = gam[ii];
                        gs[q] = fmaf(gi, g, gs[q]);
                        gd[q] = fmaf(gi * g, fmaxf(nrm[ii] + nj - 2.f * lt, 0.f), gd[q]);
                    }
                }
                for (; i < c_hi; i += 32) {
                    const float g = __ldg(grow + i), lt = __ldg(lrow + i), gi = gam[i];
                    gs[0] = fmaf(gi, g, gs[0]);
                    gd[0] = fmaf(gi * g, fmaxf(nrm[i] + nj - 2.f * lt, 0.f), gd[0]);
                }
                dw = warp_sum(dw);
                const float gsum = warp_sum((gs[0] + gs[1]) + (gs[2] + gs[3]));
                const float gdsum = warp_sum((gd[0] + gd[1]) + (gd[2] + gd[3]));
                const float y = fmaf(a.wL, dw, a.wG * gsum);
                const float e = y - target(j);
                const float kap = fmaf(a.wL, nj, a.wG);
                float beta = 0.f, s = 0.f;
                if (kap != 0.f) {
                    if (e < -a.eps) { s = 1.f; beta = (-e - a.eps) / kap; }
                    else if (e > a.eps) { s = -1.f; beta = (-e + a.eps) / kap; }
                }
                if (lane == 0) tape[(n - n0) * W + o] = Tape{beta, s, kap, dw, gsum, gdsum};
            }
            __syncthreads();
            // all projections of the step from the same f_n (Eq. apsm), then applied together
            const float mq = a.mu / (float)nJ;
            if (tid < nJ) gam[jlo + tid] += mq * tape[(n - n0) * W + tid].beta;
            for (int m = tid; m < L2; m += kBwdThreads) {
                float acc = w[m];
                for (int o = 0; o < nJ; ++o) acc = fmaf(mq * tape[(n - n0) * W + o].beta, xcomp(a.rx, M, jlo + o, m), acc);
                w[m] = acc;
            }
            __syncthreads();
        }
    };

    // ---- pass 1: forward, checkpoint at every segment start ------------------------------------------
    for (int i = tid; i < S; i += kBwdThreads) gam[i] = 0.f;
    for (int m = tid; m < M; m += kBwdThreads) {
        const float2 c = a.clin0 ? a.clin0[m * K + k] : make_float2(0.f, 0.f);
        w[m] = c.x;      // w = [Re c; Im c]
        w[M + m] = c.y;
    }
    __syncthreads();
    float *ck = a.ckpt + (size_t)k * a.n_seg * (L2 + S);
    for (int sg = 0; sg < a.n_seg; ++sg) {
        float *dst = ck + (size_t)sg * (L2 + S);
        for (int m = tid; m < L2; m += kBwdThreads) dst[m] = w[m];
        for (int i = tid; i < S; i += kBwdThreads) dst[L2 + i] = gam[i];
        forward(sg * kBwdSeg, min(S, (sg + 1) * kBwdSeg));
    }

    // ---- initial adjoint: the final coefficients and linear filter --------------------------------
    for (int i = tid; i < S; i += kBwdThreads) {
        const int t = i >> 1;
        const bool alive = P > 0 && t >= max(0, P - D);
        gbar[i] = alive ? a.dgamma[((size_t)(t % D) * 2 + (i & 1)) * K + k] : 0.f;
    }
    for (int m = tid; m < M; m += kBwdThreads) {
        const float2 d = a.dclin[m * K + k];
        wbar[m] = d.x;
        wbar[M + m] = d.y;
    }
    __syncthreads();
    // scalar adjoints: thread o sums the terms of window slot o over all steps (fixed order)
    float sig_bar = 0.f, mu_bar = 0.f, eps_bar = 0.f, wl_bar = 0.f;

    // ---- reverse sweep, one segment at a time -------------------------------------------------------
    for (int sg = a.n_seg - 1; sg >= 0; --sg) {
        const int n0 = sg * kBwdSeg, n1 = min(S, (sg + 1) * kBwdSeg);
        const float *src = ck + (size_t)sg * (L2 + S);
        for (int m = tid; m < L2; m += kBwdThreads) w[m] = src[m];
        for (int i = tid; i < S; i += kBwdThreads) gam[i] = src[L2 + i];
        __syncthreads();
        forward(n0, n1);
        for (int n = n1 - 1; n >= n0; --n) {
            const int c_lo = first_centre(n), c_hi = 2 * (n >> 1) + 2;
            const int jlo = max(0, n - W + 1), nJ = n - jlo + 1;
            const float q = 1.f / (float)nJ;
            // abar_j from the adjoint of S_{n+1}, for every j, before any update
            for (int o = warp; o < nJ; o += NW) {
                const int j = jlo + o;
                float d = 0.f;
                for (int m = lane; m < L2; m += 32) d = fmaf(wbar[m], xcomp(a.rx, M, j, m), d);
                d = warp_sum(d) + gbar[j];
                if (lane == 0) abar[o] = d;
            }
            __syncthreads();
            if (tid < nJ) {  // slot tid: its scalar terms and its coefficients for the state adjoint
                const int o = tid, j = jlo + o;
                const float ab = abar[o];
                const Tape tp = tape[(n - n0) * W + o];
                mu_bar += q * tp.beta * ab;
                const float bbar = a.mu * q * ab;
                float cwo = 0.f, cgo = 0.f;
                if (tp.s != 0.f) {  // inside the slab beta does not depend on the state
                    const float ybar = -bbar / tp.kappa;
                    eps_bar += -tp.s * bbar / tp.kappa;
                    wl_bar += (-bbar * tp.beta / tp.kappa) * (nrm[j] - 1.f);
                    wl_bar += ybar * (tp.dotw - tp.gauss);
                    sig_bar += ybar * a.wG * tp.gd2 * inv_s3;
                    cwo = ybar * a.wL;
                    cgo = ybar * a.wG;
                }
                cw[o] = cwo;
                cg[o] = cgo;
            }
            __syncthreads();
            for (int m = tid; m < L2; m += kBwdThreads) {
                float acc = wbar[m];
                for (int o = 0; o < nJ; ++o) acc = fmaf(cw[o], xcomp(a.rx, M, jlo + o, m), acc);
                wbar[m] = acc;
            }
            for (int i = c_lo + tid; i < c_hi; i += kBwdThreads) {
                float acc = gbar[i];
                for (int o = 0; o < nJ; ++o) acc = fmaf(cg[o], __ldg(a.gtab + (size_t)(jlo + o) * S + i), acc);
                gbar[i] = acc;
            }
            __syncthreads();
        }
    }

    // ---- results -------------------------------------------------------------------------------------
    for (int m = tid; m < M; m += kBwdThreads) a.dclin0[m * K + k] = make_float2(wbar[m], wbar[M + m]);
    // per-slot partial sums, combined in slot order
    __syncthreads();
    float *red = reinterpret_cast<float *>(tape);  // free now (kBwdSeg * W tapes >= 4 W floats)
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

__global__ void train_bwd_sum_kernel(const TrainBwdArgs a) {
    if (threadIdx.x < 4) {
        float s = 0.f;
        for (int k = 0; k < a.K; ++k) s += a.scal[k * 4 + threadIdx.x];  // users in order
        a.dscalars[threadIdx.x] = s;
    }
}

size_t train_bwd_smem(int M, int W, int P) {
    return sizeof(float) * (size_t)(3 * 2 * P + 2 * 2 * M + 3 * W) + sizeof(Tape) * (size_t)kBwdSeg * W;
}

}  // namespace apsm

using namespace apsm;

namespace {

struct BwdLayout {
    size_t ltab, gtab, ckpt, scal, total;
    int n_seg;
};

BwdLayout bwd_layout(const apsm_params *p, int P) {
    BwdLayout b;
    const size_t S = 2 * (size_t)P;
    b.n_seg = P > 0 ? (int)((S + kBwdSeg - 1) / kBwdSeg) : 0;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t off = 0;
    b.ltab = off;
    off = al(off + sizeof(float) * S * S);
    b.gtab = off;
    off = al(off + sizeof(float) * S * S);
    b.ckpt = off;
    off = al(off + sizeof(float) * (size_t)p->K * b.n_seg * (2 * p->M + S));
    b.scal = off;
    off = al(off + sizeof(float) * 4 * (size_t)p->K);
    b.total = off;
    return b;
}

}  // namespace

extern "C" {

apsm_status apsm_train_backward_workspace_bytes(const apsm_params *p, int32_t P, size_t *bytes) {
    size_t dummy = 0;
    apsm_status s = apsm_train_workspace_bytes(p, 0, &dummy);  // parameter validation
    if (s != APSM_OK) return s;
    if (!bytes || P < 0) return APSM_ERR_INVALID_ARG;
    *bytes = bwd_layout(p, P).total;
    return APSM_OK;
}

apsm_status apsm_train_backward(const apsm_params *p, const float *rx_pilot, const float *sym_pilot, int32_t P,
                                const float *clin0, const float *dgamma, const float *dclin, float *dscalars,
                                float *dclin0, void *workspace, size_t workspace_bytes, void *stream) {
    size_t dummy = 0;
    apsm_status s = apsm_train_workspace_bytes(p, 0, &dummy);
    if (s != APSM_OK) return s;
    if (P < 1 || !rx_pilot || !sym_pilot || !dgamma || !dclin || !dscalars || !dclin0) return APSM_ERR_INVALID_ARG;
    if (P > 8192) return APSM_ERR_UNSUPPORTED;
    if (p->weights != APSM_Q_UNIFORM) return APSM_ERR_UNSUPPORTED;  // the adjoint of q = 1/|J_n| only
    const BwdLayout b = bwd_layout(p, P);
    if (!workspace || workspace_bytes < b.total) return APSM_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return APSM_ERR_INVALID_ARG;
    const size_t smem = train_bwd_smem(p->M, p->window, P);
    if (smem > 227 * 1024) return APSM_ERR_UNSUPPORTED;
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
    a.ckpt = reinterpret_cast<float *>(ws + b.ckpt);
    a.scal = reinterpret_cast<float *>(ws + b.scal);
    a.dclin0 = reinterpret_cast<float2 *>(dclin0);
    a.dscalars = dscalars;
    a.n_seg = b.n_seg;
    const long long pairs = 4LL * P * P;
    const int blocks = (int)std::min<long long>(4096, (pairs + 255) / 256);
    train_bwd_tables_kernel<<<blocks, 256, 0, strm>>>(a);
    if (cudaFuncSetAttribute(train_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return APSM_ERR_CUDA;
    train_bwd_kernel<<<p->K, kBwdThreads, smem, strm>>>(a);
    train_bwd_sum_kernel<<<1, 32, 0, strm>>>(a);
    g_launches += 3;
    return cudaGetLastError() == cudaSuccess ? APSM_OK : APSM_ERR_CUDA;
}

}  // extern "C"
