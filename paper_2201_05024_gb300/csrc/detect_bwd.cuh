// detect_bwd.cuh -- adjoint of detection (apsm_detect_backward).
//
// For the loss L = sum_{s,k} dy1[s][k] y1[s][k] + dy2[s][k] y2[s][k] (dy = dsoft, the gradient
// of any scalar loss with respect to soft = y1 + i y2), with
//   y1 = w_L Re(c_k^H r_s) + w_G sum_t [g1_t E_A + g2_t E_C],
//   y2 = w_L Im(c_k^H r_s) + w_G sum_t [g1_t E_B + g2_t E_A]       (detection, Sec. III-B)
// the partial derivatives are
//   dL/dg1_t = w_G sum_s (dy1 E_A + dy2 E_B)          dL/dg2_t = w_G sum_s (dy1 E_C + dy2 E_A)
//   dL/dc_k  = w_L sum_s conj(dy_s^k) r_s             (c = Re c + i Im c, as one complex number)
//   dL/dsigma = (w_G / sigma^3) sum_{s,t,k} [g1 (dy1 E_A d_A + dy2 E_B d_B) + g2 (dy1 E_C d_C + dy2 E_A d_A)]
//   dL/dw_L  = sum_{s,k} dy . (c^H r_s) - sum_{s,k} dy . (unweighted Gaussian sums)
// (d_A, d_B, d_C the squared distances behind E_A, E_B, E_C; dE/dsigma = E d / sigma^3).  The
// last term equals sum_t sum_k (g1 G1 + g2 G2) with G the unweighted coefficient gradients, so
// every scalar follows from per-entry sums.  Exponentials are recomputed, not stored.
//
// Kernels:
//   detect_bwd_entry_kernel   entry-stationary: each thread owns one dictionary entry (vector in
//                             registers) and streams a slice of the queries past it through
//                             shared memory; writes per-slice sums G (coefficient gradient) and
//                             H (sigma weights) -- no atomics.
//   detect_bwd_clin_kernel    per query slice, sum_s conj(dy) r for every (m, k).
//   detect_bwd_finalize_kernel  one thread per (entry, coefficient): fixed-order sums over the
//                             slices -> dgamma and its scalar terms.
//   detect_bwd_scalars_kernel one CTA: fixed-order sums -> dclin, dsigma, dw_L.
#pragma once

#include "apsm_common.cuh"

namespace apsm {

constexpr int kBwdEntriesPerCta = 64;
constexpr int kBwdQueryTile = 32;

struct DetectBwdArgs {
    const float2 *rx;         // [N][M]
    const float2 *dsoft;      // [N][K]
    int N;
    const float2 *dict;       // [A][M]
    const float *dict_norm;   // [A]
    const float *gamma;       // [A][2][K]
    const float2 *clin;       // [M][K]
    const int *meta;          // meta[0] = entries held
    int n_entries;            // host bound (dict_cap)
    int A;                    // slots
    int q_per_slice;          // queries per slice (multiple of kBwdQueryTile)
    int n_qslices;
    int n_cslices;            // slices of the linear-filter reduction
    float k2, wL, wG, sigma;
    float *gh;                // workspace [n_qslices][A][4K]: G1, G2, H1, H2
    float2 *cpart;            // workspace [n_cslices][M][K]
    float *scal;              // workspace [A][2K][2]: per-coefficient sigma and Gaussian terms
    float *dgamma;            // out [A][2][K]
    float2 *dclin;            // out [M][K]
    float *dscalars;          // out [2]: dL/dsigma, dL/dw_L
};

template <int M, int K>
__global__ void __launch_bounds__(kBwdEntriesPerCta) detect_bwd_entry_kernel(const DetectBwdArgs a) {
    __shared__ __align__(16) float2 s_r[kBwdQueryTile * M];
    __shared__ __align__(16) float2 s_dy[kBwdQueryTile * K];
    __shared__ float s_n[kBwdQueryTile];
    const int n_ent = min(a.n_entries, max(__ldg(a.meta), 0));
    const int t = blockIdx.x * kBwdEntriesPerCta + threadIdx.x;
    const bool valid = t < n_ent;
    float2 rt[M];
    float nt = 0.f, G1[K], G2[K], H1[K], H2[K];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        rt[m] = valid ? __ldg(a.dict + (size_t)t * M + m) : make_float2(0.f, 0.f);
        nt = fmaf(rt[m].x, rt[m].x, fmaf(rt[m].y, rt[m].y, nt));
    }
#pragma unroll
    for (int k = 0; k < K; ++k) G1[k] = G2[k] = H1[k] = H2[k] = 0.f;

    const int q0 = blockIdx.y * a.q_per_slice, q1 = min(a.N, q0 + a.q_per_slice);
    for (int qt = q0; qt < q1; qt += kBwdQueryTile) {
        const int cnt = min(kBwdQueryTile, q1 - qt);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt * M; i += blockDim.x) s_r[i] = a.rx[(size_t)qt * M + i];
        for (int i = threadIdx.x; i < cnt * K; i += blockDim.x) s_dy[i] = a.dsoft[(size_t)qt * K + i];
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            float n = 0.f;
            for (int m = 0; m < M; ++m) n = fmaf(s_r[i * M + m].x, s_r[i * M + m].x, fmaf(s_r[i * M + m].y, s_r[i * M + m].y, n));
            s_n[i] = n;
        }
        __syncthreads();
        if (!valid) continue;
#pragma unroll 1
        for (int s = 0; s < cnt; ++s) {
            float zr = 0.f, zi = 0.f;  // z = r_t^H r_s
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const float2 x = s_r[s * M + m];
                zr = fmaf(rt[m].x, x.x, fmaf(rt[m].y, x.y, zr));
                zi = fmaf(rt[m].x, x.y, fmaf(-rt[m].y, x.x, zi));
            }
            const float nn = nt + s_n[s];
            const float dA = fmaxf(fmaf(-2.f, zr, nn), 0.f);
            const float dB = fmaxf(fmaf(-2.f, zi, nn), 0.f);
            const float dC = fmaxf(fmaf(2.f, zi, nn), 0.f);
            const float eA = ex2(-a.k2 * dA), eB = ex2(-a.k2 * dB), eC = ex2(-a.k2 * dC);
            const float fA = eA * dA, fB = eB * dB, fC = eC * dC;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float2 g = s_dy[s * K + k];  // (dy1, dy2)
                G1[k] = fmaf(g.x, eA, fmaf(g.y, eB, G1[k]));
                G2[k] = fmaf(g.x, eC, fmaf(g.y, eA, G2[k]));
                H1[k] = fmaf(g.x, fA, fmaf(g.y, fB, H1[k]));
                H2[k] = fmaf(g.x, fC, fmaf(g.y, fA, H2[k]));
            }
        }
    }
    if (t < a.A) {
        float *dst = a.gh + ((size_t)blockIdx.y * a.A + t) * 4 * K;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            dst[k] = G1[k];
            dst[K + k] = G2[k];
            dst[2 * K + k] = H1[k];
            dst[3 * K + k] = H2[k];
        }
    }
}

// Partial sums of conj(dy_s^k) r_s[m] over one query slice; thread = (m, k) pair.
template <int M, int K>
__global__ void detect_bwd_clin_kernel(const DetectBwdArgs a) {
    const int mk = threadIdx.x;
    if (mk >= M * K) return;
    const int m = mk / K, k = mk % K;
    const int per = (a.N + a.n_cslices - 1) / a.n_cslices;
    const int q0 = blockIdx.x * per, q1 = min(a.N, q0 + per);
    float re = 0.f, im = 0.f;
#pragma unroll 8
    for (int s = q0; s < q1; ++s) {
        const float2 r = __ldg(a.rx + (size_t)s * M + m), g = __ldg(a.dsoft + (size_t)s * K + k);
        re = fmaf(g.x, r.x, fmaf(g.y, r.y, re));   // Re(conj(g) r)
        im = fmaf(g.x, r.y, fmaf(-g.y, r.x, im));  // Im(conj(g) r)
    }
    a.cpart[(size_t)blockIdx.x * M * K + mk] = make_float2(re, im);
}

template <int K>
__global__ void detect_bwd_finalize_kernel(const DetectBwdArgs a) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.A * 2 * K) return;
    const int t = idx / (2 * K), j = idx % (2 * K);
    const int n_ent = min(a.n_entries, max(__ldg(a.meta), 0));
    float G = 0.f, H = 0.f;
    if (t < n_ent) {
        const float *src = a.gh + (size_t)t * 4 * K + j;
        const size_t stride = (size_t)a.A * 4 * K;
        for (int sl0 = 0; sl0 < a.n_qslices; sl0 += 8) {  // eight slices' loads in flight, summed in order
            float g[8], h[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const bool in = sl0 + q < a.n_qslices;
                g[q] = in ? src[(sl0 + q) * stride] : 0.f;
                h[q] = in ? src[(sl0 + q) * stride + 2 * K] : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                G += g[q];
                H += h[q];
            }
        }
    }
    const float g = t < n_ent ? a.gamma[(size_t)t * 2 * K + j] : 0.f;
    a.dgamma[(size_t)t * 2 * K + j] = a.wG * G;
    a.scal[2 * (size_t)idx] = g * H;
    a.scal[2 * (size_t)idx + 1] = g * G;
}

// One CTA of 256 threads: fixed-order reductions for dclin, dsigma, dw_L.
template <int M, int K>
__global__ void __launch_bounds__(256) detect_bwd_scalars_kernel(const DetectBwdArgs a) {
    __shared__ float s_sig[256], s_gau[256], s_lin[256];
    float sig = 0.f, gau = 0.f, lin = 0.f;
    for (int t = threadIdx.x; t < a.A * 2 * K; t += blockDim.x) {
        sig += a.scal[2 * t];
        gau += a.scal[2 * t + 1];
    }
    for (int mk = threadIdx.x; mk < M * K; mk += blockDim.x) {
        float re = 0.f, im = 0.f;
        for (int sl = 0; sl < a.n_cslices; ++sl) {
            const float2 v = a.cpart[(size_t)sl * M * K + mk];
            re += v.x;
            im += v.y;
        }
        a.dclin[mk] = make_float2(a.wL * re, a.wL * im);
        const float2 c = a.clin[mk];
        lin = fmaf(c.x, re, fmaf(c.y, im, lin));  // Re(conj(c) Gc)
    }
    s_sig[threadIdx.x] = sig;
    s_gau[threadIdx.x] = gau;
    s_lin[threadIdx.x] = lin;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s_sig[threadIdx.x] += s_sig[threadIdx.x + w];
            s_gau[threadIdx.x] += s_gau[threadIdx.x + w];
            s_lin[threadIdx.x] += s_lin[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float s3 = a.sigma * a.sigma * a.sigma;
        a.dscalars[0] = a.wG * s_sig[0] / s3;
        a.dscalars[1] = s_lin[0] - s_gau[0];
    }
}

template <int M, int K>
cudaError_t launch_detect_bwd(const DetectBwdArgs &a, cudaStream_t stream) {
    if (a.N > 0) {
        const dim3 grid((a.n_entries + kBwdEntriesPerCta - 1) / kBwdEntriesPerCta, a.n_qslices);
        detect_bwd_entry_kernel<M, K><<<grid, kBwdEntriesPerCta, 0, stream>>>(a);
        detect_bwd_clin_kernel<M, K><<<a.n_cslices, round_up(M * K, 32), 0, stream>>>(a);
    }
    detect_bwd_finalize_kernel<K><<<(a.A * 2 * K + 127) / 128, 128, 0, stream>>>(a);
    detect_bwd_scalars_kernel<M, K><<<1, 256, 0, stream>>>(a);
    return cudaGetLastError();
}

using DetectBwdLauncher = cudaError_t (*)(const DetectBwdArgs &, cudaStream_t);

}  // namespace apsm
