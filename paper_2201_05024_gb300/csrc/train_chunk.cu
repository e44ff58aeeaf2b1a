// train_chunk.cu -- the training kernel-table kernel (train_gram_kernel) and the host-side
// launcher table of the phase-B kernel (instantiated per live-range warp count S in
// train_chunk_s*.cu, so that the build compiles them in parallel).
#include "train_f32.cuh"

namespace apsm {

// One CTA per (chunk, 32 x 32 sample tile of one table).  The tile's 16 row and 16 column pilots
// are staged in shared memory with their norms; each thread takes one pilot pair, whose complex
// inner product z = r_a^H r_b gives all four real-split sample pairs:
//   r1(a).r1(b) = r2(a).r2(b) = Re z,  r1(a).r2(b) = Im z,  r2(a).r1(b) = -Im z,
//   ||x_a - x_b||^2 = ||r_a||^2 + ||r_b||^2 - 2 x_a.x_b.
// Tables: 0 = kmat (live range x live range, sum kernel), 1 = gev (dropped entries x live range,
// Gaussian), 2 = kx (live range x next chunk's samples, sum kernel).
// Row and column vectors come from the extended pilot sequence rx; an entry dropped in the chunk
// whose running index is below t_base (trained on in an earlier call) comes from its dictionary
// slot, which holds it until the chunk kernels overwrite it (they run after this kernel).
__global__ void __launch_bounds__(256) train_gram_kernel(const float2 *__restrict__ rx, const float2 *__restrict__ dict,
                                                         TrainGeom g, float k2, float wL, float wG,
                                                         float *__restrict__ kmat, float *__restrict__ gev,
                                                         float *__restrict__ kx) {
    extern __shared__ __align__(16) float2 s_gram[];
    pdl_enter();
    const int c = blockIdx.y;
    int t0, Tc, s0, s1, l0;
    chunk_range(g, c, t0, Tc, s0, s1, l0);
    const int M = g.M, MS = g.M + 1;  // padded row of a staged pilot (bank spread)
    float2 *s_row = s_gram, *s_col = s_gram + 16 * MS;
    float *s_nrm = reinterpret_cast<float *>(s_gram + 32 * MS);  // [0,16) rows, [16,32) columns
    const int RT = g.RS / 32, ET = (2 * g.T + 31) / 32, XT = g.KXS / 32;
    const int n_ev = g.evict ? ET * RT : 0;
    const int n_next = c + 1 < g.n_chunks ? 2 * min(g.T, g.P - t0 - Tc) : 0;
    int job = blockIdx.x, table, rt, ct;
    if (job < RT * RT) {
        table = 0; rt = job / RT; ct = job % RT;
    } else if ((job -= RT * RT) < n_ev) {
        table = 1; rt = job / RT; ct = job % RT;
    } else {
        job -= n_ev;
        if (!g.track || job >= RT * XT) return;
        table = 2; rt = job / XT; ct = job % XT;
    }
    // vector of staged row / column i (nullptr: outside the table's valid range)
    auto row_src = [&](int i) -> const float2 * {
        if (table == 1) {  // entry dropped at step 2(t0 + e): running index tb + t0 + e - D
            const int e = 16 * rt + i, run = g.t_base + t0 + e - g.D;
            if (e >= Tc || run < 0) return nullptr;
            return run >= g.t_base ? rx + (size_t)(run - g.t_base) * g.M : dict + (size_t)(run % g.D) * g.M;
        }
        const int smp = l0 + 32 * rt + 2 * i;
        return smp < s1 ? rx + (size_t)(smp >> 1) * g.M : nullptr;
    };
    auto col_src = [&](int j) -> const float2 * {
        if (table == 2) {
            const int v = 32 * ct + 2 * j;
            return v < n_next ? rx + (size_t)(t0 + Tc + (v >> 1)) * g.M : nullptr;
        }
        const int smp = l0 + 32 * ct + 2 * j;
        return smp < s1 ? rx + (size_t)(smp >> 1) * g.M : nullptr;
    };
    for (int idx = threadIdx.x; idx < 32 * M; idx += blockDim.x) {
        const int i = idx / M, mm = idx % M;
        const float2 *src = i < 16 ? row_src(i) : col_src(i - 16);
        const float2 v = src ? __ldcg(src + mm) : make_float2(0.f, 0.f);
        (i < 16 ? s_row + i * MS : s_col + (i - 16) * MS)[mm] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const float2 *r = threadIdx.x < 16 ? s_row + threadIdx.x * MS : s_col + (threadIdx.x - 16) * MS;
        float n = 0.f;
        for (int mm = 0; mm < M; ++mm) n = fmaf(r[mm].x, r[mm].x, fmaf(r[mm].y, r[mm].y, n));
        s_nrm[threadIdx.x] = n;
    }
    __syncthreads();
    const int i = threadIdx.x >> 4, j = threadIdx.x & 15;
    const bool ok = row_src(i) != nullptr && col_src(j) != nullptr;
    const float2 *ra = s_row + i * MS, *rb = s_col + j * MS;
    float zr = 0.f, zi = 0.f;
    for (int mm = 0; mm < M; ++mm) {
        const float2 x = ra[mm], y = rb[mm];
        zr = fmaf(x.x, y.x, fmaf(x.y, y.y, zr));
        zi = fmaf(x.x, y.y, fmaf(-x.y, y.x, zi));
    }
    const float nn = s_nrm[i] + s_nrm[16 + j];
    float out[2][2];
#pragma unroll
    for (int la = 0; la < 2; ++la)
#pragma unroll
        for (int lb = 0; lb < 2; ++lb) {
            const float dot = (la == lb) ? zr : (la == 0 ? zi : -zi);
            const float ge = ex2(-k2 * fmaxf(nn - 2.f * dot, 0.f));
            const float val = table == 1 ? ge : fmaf(wL, dot, wG * ge);  // sum kernel (Fact 1)
            out[la][lb] = ok ? val : 0.f;
        }
    const int row0 = 32 * rt + 2 * i, col = 32 * ct + 2 * j;
#pragma unroll
    for (int la = 0; la < 2; ++la) {
        const float2 v = make_float2(out[la][0], out[la][1]);
        if (table == 0) {
            reinterpret_cast<float2 *>(kmat + ((size_t)c * g.RS + row0 + la) * g.RS + col)[0] = v;
        } else if (table == 1) {
            if (row0 + la < 2 * g.T)
                reinterpret_cast<float2 *>(gev + ((size_t)c * 2 * g.T + row0 + la) * g.RS + col)[0] = v;
        } else {
            reinterpret_cast<float2 *>(kx + ((size_t)c * g.RS + row0 + la) * g.KXS + col)[0] = v;
        }
    }
}

cudaError_t launch_train_gram(const float2 *rx, const float2 *dict, const TrainGeom &g, float k2, float wL, float wG,
                              float *kmat, float *gev, float *kx, cudaStream_t stream) {
    const int RT = g.RS / 32, ET = (2 * g.T + 31) / 32, XT = g.KXS / 32;
    const int jobs = RT * RT + (g.evict ? ET * RT : 0) + (g.track ? RT * XT : 0);
    const size_t smem = (size_t)32 * (g.M + 1) * sizeof(float2) + 32 * sizeof(float);
    cudaError_t e = launch_pdl(train_gram_kernel, dim3(jobs, g.n_chunks), dim3(256), smem, stream, rx, dict, g, k2,
                               wL, wG, kmat, gev, kx);
    return e != cudaSuccess ? e : cudaGetLastError();
}

using ChunkLauncher = cudaError_t (*)(const ChunkArgs &, int, cudaStream_t);
ChunkLauncher chunk_launcher_s1_x0(int WP);
ChunkLauncher chunk_launcher_s1_x1(int WP);  // train_chunk_s*{p,x}.cu: one translation unit per (S, plain or extended)
ChunkLauncher chunk_launcher_s2_x0(int WP);
ChunkLauncher chunk_launcher_s2_x1(int WP);
ChunkLauncher chunk_launcher_s3_x0(int WP);
ChunkLauncher chunk_launcher_s3_x1(int WP);
ChunkLauncher chunk_launcher_s4_x0(int WP);
ChunkLauncher chunk_launcher_s4_x1(int WP);
ChunkLauncher chunk_launcher_s5_x0(int WP);
ChunkLauncher chunk_launcher_s5_x1(int WP);

// Smallest supported padded window >= W (0 if W is too large).
int padded_window(int W) {
    static const int kWP[] = {4, 8, 12, 16, 20, 24, 32, 48, 64, 96, 128};
    for (int wp : kWP)
        if (wp >= W) return wp;
    return 0;
}

ChunkLauncher chunk_launcher(int S, int WP, bool ext) {
    switch (S) {
        case 1: return ext ? chunk_launcher_s1_x1(WP) : chunk_launcher_s1_x0(WP);
        case 2: return ext ? chunk_launcher_s2_x1(WP) : chunk_launcher_s2_x0(WP);
        case 3: return ext ? chunk_launcher_s3_x1(WP) : chunk_launcher_s3_x0(WP);
        case 4: return ext ? chunk_launcher_s4_x1(WP) : chunk_launcher_s4_x0(WP);
        case 5: return ext ? chunk_launcher_s5_x1(WP) : chunk_launcher_s5_x0(WP);
        default: return nullptr;
    }
}

}  // namespace apsm
