// linear_init.cu -- apsm_linear_init: a conventional linear detector as the start f_0 of the
// APSM recurrence (Sec. I: start from a linear filter; f_0 is arbitrary in Eq. apsm).
//
// From P pilots r(t) (columns of Y, M x P) and their symbols s(t) (columns of S, K x P):
//   least-squares channel estimate   H = Y S^H (S S^H)^-1                    (M x K)
//   MMSE filter                      W = H (H^H H + N0 I_K)^-1               (M x K; N0 = 0: ZF)
// whose soft estimates are W^H r.  The push-through identity gives the same W as the textbook
// (H H^H + N0 I_M)^-1 H with a K x K instead of an M x M system.  Both K x K systems are
// Hermitian positive definite when the pilot symbols span K directions; they are solved by
// Cholesky factorisation.  The library's linear part evaluates w_L c^H r, so the output is
// clin0 = W / w_L.
//
// One CTA: the two sums over the pilots take one thread per output element with four
// interleaved partial sums (fixed order, deterministic), the factorisations and solves are a few
// thousand complex operations in shared memory.
#include <atomic>
#include <cmath>

#include "apsm_common.cuh"

namespace apsm {
namespace {

constexpr int kLinThreads = 512;
constexpr int kMaxM = 64, kMaxK = 16;

struct cplx {
    float x, y;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cplx cmulc(cplx a, cplx b) { return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y}; }  // a conj(b)
__device__ __forceinline__ cplx cconjmul(cplx a, cplx b) { return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x}; }  // conj(a) b

// In-place Cholesky A = L L^H of the n x n Hermitian matrix A (row-major, stride n) by one warp;
// returns false on a non-positive (or non-finite) pivot.  The strictly upper part is not read.
__device__ bool chol_warp(cplx *A, int n) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < n; ++j) {
        float d = A[j * n + j].x;
        for (int k = 0; k < j; ++k) d -= A[j * n + k].x * A[j * n + k].x + A[j * n + k].y * A[j * n + k].y;
        if (!(d > 0.f) || !isfinite(d)) return false;
        const float ljj = sqrtf(d);
        __syncwarp();
        // column j below the diagonal: L[i][j] = (A[i][j] - sum_k L[i][k] conj(L[j][k])) / L[j][j]
        for (int i = j + 1 + lane; i < n; i += 32) {
            cplx v = A[i * n + j];
            for (int k = 0; k < j; ++k) {
                const cplx t = cmulc(A[i * n + k], A[j * n + k]);
                v.x -= t.x;
                v.y -= t.y;
            }
            A[i * n + j] = {v.x / ljj, v.y / ljj};
        }
        __syncwarp();
        if (lane == 0) A[j * n + j] = {ljj, 0.f};
        __syncwarp();
    }
    return true;
}

// Solve L L^H x = b for one right-hand side (b overwritten by x), by one thread.
__device__ void chol_solve(const cplx *L, int n, cplx *b) {
    for (int i = 0; i < n; ++i) {  // L y = b
        cplx v = b[i];
        for (int k = 0; k < i; ++k) {
            const cplx t = cmul(L[i * n + k], b[k]);
            v.x -= t.x;
            v.y -= t.y;
        }
        b[i] = {v.x / L[i * n + i].x, v.y / L[i * n + i].x};
    }
    for (int i = n - 1; i >= 0; --i) {  // L^H x = y
        cplx v = b[i];
        for (int k = i + 1; k < n; ++k) {
            const cplx t = cconjmul(L[k * n + i], b[k]);
            v.x -= t.x;
            v.y -= t.y;
        }
        b[i] = {v.x / L[i * n + i].x, v.y / L[i * n + i].x};
    }
}

__global__ void __launch_bounds__(kLinThreads) linear_init_kernel(const float2 *__restrict__ rx,
                                                                 const float2 *__restrict__ sym, int P, int M, int K,
                                                                 float noise_var, float inv_wL, float2 *clin0) {
    __shared__ cplx G[kMaxK * kMaxK];   // S S^H, then its factor; later H^H H + N0 I and its factor
    __shared__ cplx B[kMaxM * kMaxK];   // Y S^H, then H (row m = h_m), then W
    __shared__ int ok;
    pdl_enter();
    const int tid = threadIdx.x;
    if (tid == 0) ok = 1;
    // the two sums over the pilots: G[i][j] = sum_t s_i(t) conj(s_j(t)), B[m][j] = sum_t r_m(t) conj(s_j(t))
    for (int o = tid; o < K * K + M * K; o += kLinThreads) {
        const bool g = o < K * K;
        const int row = g ? o / K : (o - K * K) / K, col = g ? o % K : (o - K * K) % K;
        cplx acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        for (int t = 0; t < P; ++t) {
            const float2 a = g ? sym[(size_t)t * K + row] : rx[(size_t)t * M + row];
            const float2 s = sym[(size_t)t * K + col];
            const cplx v = cmulc({a.x, a.y}, {s.x, s.y});
            acc[t & 3].x += v.x;
            acc[t & 3].y += v.y;
        }
        const cplx r = {(acc[0].x + acc[1].x) + (acc[2].x + acc[3].x), (acc[0].y + acc[1].y) + (acc[2].y + acc[3].y)};
        if (g) G[row * K + col] = r;
        else B[row * K + col] = r;
    }
    __syncthreads();
    if (tid < 32 && !chol_warp(G, K) && tid == 0) ok = 0;
    __syncthreads();
    // H: row h_m solves h_m (S S^H) = b_m, i.e. (S S^H) h_m^H = b_m^H (Hermitian system)
    if (ok && tid < M) {
        cplx x[kMaxK];
        for (int j = 0; j < K; ++j) x[j] = {B[tid * K + j].x, -B[tid * K + j].y};
        chol_solve(G, K, x);
        for (int j = 0; j < K; ++j) B[tid * K + j] = {x[j].x, -x[j].y};
    }
    __syncthreads();
    // C = H^H H + N0 I  (C[i][j] = sum_m conj(H[m][i]) H[m][j])
    if (ok) {
        for (int o = tid; o < K * K; o += kLinThreads) {
            const int i = o / K, j = o % K;
            cplx acc = {0.f, 0.f};
            for (int m = 0; m < M; ++m) {
                const cplx t = cconjmul(B[m * K + i], B[m * K + j]);
                acc.x += t.x;
                acc.y += t.y;
            }
            if (i == j) acc.x += noise_var;
            G[o] = acc;
        }
    }
    __syncthreads();
    if (ok && tid < 32 && !chol_warp(G, K) && tid == 0) ok = 0;
    __syncthreads();
    // W: row w_m solves w_m C = h_m, i.e. C w_m^H = h_m^H; output clin0 = W / w_L
    if (tid < M) {
        cplx x[kMaxK];
        for (int j = 0; j < K; ++j) x[j] = {B[tid * K + j].x, -B[tid * K + j].y};
        if (ok) chol_solve(G, K, x);
        for (int j = 0; j < K; ++j)
            clin0[(size_t)tid * K + j] = ok ? make_float2(x[j].x * inv_wL, -x[j].y * inv_wL) : make_float2(0.f, 0.f);
    }
}

}  // namespace

extern std::atomic<long long> g_launches;

}  // namespace apsm

extern "C" apsm_status apsm_linear_init(const apsm_params *p, const float *rx_pilot, const float *sym_pilot,
                                        int32_t P, float noise_var, float *clin0, void *stream) {
    if (!p || !rx_pilot || !sym_pilot || !clin0) return APSM_ERR_INVALID_ARG;
    size_t dummy = 0;
    apsm_status s = apsm_train_workspace_bytes(p, 0, &dummy);  // parameter validation
    if (s != APSM_OK) return s;
    if (P < p->K || P > (1 << 26) || !(noise_var >= 0.f) || !std::isfinite(noise_var) || !(p->w_L > 0.f))
        return APSM_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(rx_pilot) & 15) || (reinterpret_cast<uintptr_t>(sym_pilot) & 7) ||
        (reinterpret_cast<uintptr_t>(clin0) & 7))
        return APSM_ERR_INVALID_ARG;
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
        cudaGetLastError();
        return APSM_ERR_CUDA;
    }
    if (major != 10 || minor != 3) return APSM_ERR_NOT_SM103;
    const cudaError_t e = apsm::launch_pdl(apsm::linear_init_kernel, dim3(1), dim3(apsm::kLinThreads), 0,
                                           static_cast<cudaStream_t>(stream),
                                           reinterpret_cast<const float2 *>(rx_pilot),
                                           reinterpret_cast<const float2 *>(sym_pilot), (int)P, p->M, p->K, noise_var,
                                           1.f / p->w_L, reinterpret_cast<float2 *>(clin0));
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return APSM_ERR_CUDA;
    apsm::g_launches++;
    return APSM_OK;
}
