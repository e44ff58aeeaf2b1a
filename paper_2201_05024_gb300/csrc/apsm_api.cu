// apsm_api.cu -- host side of the C ABI declared in include/apsm.h.
//
// Validates arguments before any CUDA call, checks for an sm_103 device, picks launch
// shapes and enqueues the kernels on the caller's stream.  Nothing is allocated here: state
// and workspace are caller-owned device memory.
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "apsm_common.cuh"
#include "detect_bwd.cuh"
#include "detect_f32.cuh"
#include "detect_tc.cuh"
#include "detect_tcc.cuh"
#include "detect_tma.cuh"
#include "train_f32.cuh"

namespace apsm {

std::atomic<long long> g_launches{0};

DetectLauncher detect_f32_launcher(int M, int K);  // detect_f32_m*.cu
DetectBwdLauncher detect_bwd_launcher(int M, int K);  // detect_f32_m*.cu
TcLauncher detect_tc_launcher(int M, int K, int prec);  // detect_tc_m*.cu
TmaLauncher detect_tma_launcher(int M, int K);         // detect_tma_m*.cu
TccLauncher detect_tcc_launcher(int M, int K);         // detect_tc_m*.cu (BF16/FP16, coefficient sums on tcgen05)
size_t detect_tcc_workspace(int M, int K, int D);
using ChunkLauncher = cudaError_t (*)(const ChunkArgs &, int, cudaStream_t);
ChunkLauncher chunk_launcher(int S, int WP, bool ext);  // train_chunk.cu
int padded_window(int W);                           // train_chunk.cu

namespace {

bool supported_M(int M) { return M == 2 || M == 4 || M == 8 || M == 16 || M == 32 || M == 64; }

apsm_status check_params(const apsm_params *p) {
    if (!p) return APSM_ERR_INVALID_ARG;
    if (p->M < 1 || p->K < 1 || p->window < 1 || p->dict_cap < 1) return APSM_ERR_INVALID_ARG;
    if (!(p->sigma > 0.f) || !std::isfinite(p->sigma)) return APSM_ERR_INVALID_ARG;
    if (!(p->mu > 0.f) || !(p->mu <= 2.f)) return APSM_ERR_INVALID_ARG;
    if (!(p->eps >= 0.f) || !std::isfinite(p->eps)) return APSM_ERR_INVALID_ARG;
    if (!(p->w_L >= 0.f) || !(p->w_L <= 1.f)) return APSM_ERR_INVALID_ARG;
    if (2LL * p->dict_cap <= p->window) return APSM_ERR_INVALID_ARG;
    if (p->dtype != APSM_FP32 && p->dtype != APSM_BF16 && p->dtype != APSM_FP16) return APSM_ERR_INVALID_ARG;
    if (p->dict_cap > (1 << 26)) return APSM_ERR_INVALID_ARG;
    if (p->modulation != 0 && p->modulation != 2 && p->modulation != 4 && p->modulation != 6)
        return APSM_ERR_INVALID_ARG;
    if (p->weights != APSM_Q_UNIFORM && p->weights != APSM_Q_VIOLATED) return APSM_ERR_INVALID_ARG;
    if (!supported_M(p->M) || p->K > 16 || p->window > 128) return APSM_ERR_UNSUPPORTED;
    return APSM_OK;
}

bool aligned16(const void *ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15) == 0; }

apsm_status check_state(const apsm_state *st) {
    if (!st || !st->dict || !st->dict_norm || !st->gamma || !st->clin || !st->meta || !st->target)
        return APSM_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(st->target) & 7) return APSM_ERR_INVALID_ARG;
    // dictionary tiles are moved by the bulk-copy engine: 16-byte aligned sources
    if (!aligned16(st->dict) || !aligned16(st->dict_norm) || !aligned16(st->gamma)) return APSM_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(st->clin) & 7) || (reinterpret_cast<uintptr_t>(st->meta) & 3))
        return APSM_ERR_INVALID_ARG;
    return APSM_OK;
}

int current_device() {
    int dev = 0;
    return cudaGetDevice(&dev) == cudaSuccess ? dev : 0;
}

// sm_103 check, cached per device.
apsm_status check_device() {
    static std::mutex mu;
    static int cached[64];  // 0 unknown, 1 ok, 2 not sm_103
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return APSM_ERR_CUDA;
    }
    if (dev < 0 || dev >= 64) return APSM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (cached[dev] == 0) {
        int major = 0, minor = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
            cudaGetLastError();
            return APSM_ERR_CUDA;
        }
        cached[dev] = (major == 10 && minor == 3) ? 1 : 2;
    }
    return cached[dev] == 1 ? APSM_OK : APSM_ERR_NOT_SM103;
}

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
    }
    return sms;
}

constexpr int kMaxChunkThreads = 160;      // phase-B CTA size limit (S <= 5 warps)
constexpr int kMaxSmemBytes = 227 * 1024;  // opt-in shared memory per CTA

// ---- process-wide launch options (apsm_set_option) -------------------------------------------
std::atomic<int> g_opt_train_chunk{64};  // pilots per training chunk
std::atomic<int> g_opt_train_track{1};   // next-chunk tracking form (1) or sequential form (0)
std::atomic<int> g_opt_detect_tma{1};     // TMA-staged FP32 detection where it applies (1) or not (0)
std::atomic<int> g_opt_half_tc_coef{1};   // BF16/FP16: coefficient sums on the tensor cores (1) or FP32 pipe (0)

inline apsm_status cuda_status(cudaError_t e) { return e == cudaSuccess ? APSM_OK : APSM_ERR_CUDA; }

float k2_of(float sigma) { return kLog2e / (2.f * sigma * sigma); }

// ---- launch-choice table filled by the autotuner (apsm_tune_set) ----------------------------
struct TuneEntry {
    int set, engine, threads, split, qpt;
};
std::mutex g_tune_mu;
TuneEntry g_tune[7][17][3];  // [log2 M][K][dtype]

int m_slot(int M) {
    switch (M) {
        case 2: return 1;
        case 4: return 2;
        case 8: return 3;
        case 16: return 4;
        case 32: return 5;
        case 64: return 6;
        default: return 0;
    }
}

TuneEntry tune_get(int M, int K, int dtype) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (m_slot(M) == 0 || K < 1 || K > 16 || dtype < 0 || dtype > 2) return TuneEntry{};
    return g_tune[m_slot(M)][K][dtype];
}

// ---- detection launch shape -------------------------------------------------------------
DetectShape detect_shape(int M, int K, int dtype) {
    const TuneEntry te = tune_get(M, K, dtype);
    if (te.set && te.engine == 1) return DetectShape{te.threads, te.split, te.qpt};
    return DetectShape{64, 2, 1};  // 64 query lanes x 2 entry groups, one query per lane
}

// ---- training geometry --------------------------------------------------------------------
// Geometry of one training call: P new vectors after n_prev earlier ones (of which the last
// nc0 = min(n_prev, W/2) pilots are carried, because the first new window reaches back into
// them).  evict: -1 = decide from the counts, 0/1 = forced (workspace bounds over both cases).
TrainGeom train_geom(const apsm_params *p, int P, int n_prev, int evict = -1) {
    TrainGeom g;
    g.M = p->M;
    g.K = p->K;
    g.W = p->window;
    g.D = p->dict_cap;
    g.nc0 = std::min(n_prev, g.W / 2);
    g.t_base = n_prev - g.nc0;
    g.P = g.nc0 + P;
    g.evict = evict >= 0 ? evict : (g.t_base + g.P > g.D ? 1 : 0);
    // Entries dropped inside a chunk must be older than the chunk's live range, whose first pilot
    // is t0 - floor(W/2): D >= T + floor(W/2).  The same bound keeps a chunk's live range in the
    // dictionary at the next chunk's start (needed by the tracked form).
    int T = g_opt_train_chunk.load();
    T = std::min(T, g.D - g.W / 2);
    T = std::min(T, (kMaxChunkThreads - g.W) / 2);  // one thread per live-range sample
    T = std::max(T, 1);
    g.WP = padded_window(g.W);
    g.slice = kTileEntries;
    const bool want_track = g_opt_train_track.load() != 0;
    for (;; --T) {  // the largest chunk whose phase-B tables fit in shared memory
        g.T = T;
        g.RMAX = 2 * T + g.W;
        g.RS = round_up(g.RMAX, 32);
        g.KXS = round_up(2 * T, 32);
        // tracking needs the blocked form (padded window <= 24) and a warp besides the window warp
        g.track = want_track && g.WP <= 24 && g.RS >= 64 && 2 * T <= 2 * (g.RS - 32) ? 1 : 0;
        if (T == 1 || ChunkSmem(g).bytes <= kMaxSmemBytes) break;
    }
    g.n_chunks = P > 0 ? (P + T - 1) / T : 0;
    return g;
}

struct TrainWs {
    size_t kmat, gev, kx, partial[2], track[2], carry, ext_rx, ext_sym, total;
    int max_slices, part_rows;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Workspace layout; ext: room for the extended sequence (carried pilots + new vectors and their
// targets) of a continuation or of decision-directed training.
TrainWs train_ws(const TrainGeom &g, bool ext) {
    TrainWs w;
    size_t off = 0;
    w.kmat = off;
    off = align256(off + sizeof(float) * (size_t)g.n_chunks * g.RS * g.RS);
    w.gev = off;
    off = align256(off + sizeof(float) * (size_t)g.n_chunks * g.T * 2 * g.RS);
    w.kx = off;
    if (g.track) off = align256(off + sizeof(float) * (size_t)g.n_chunks * g.RS * g.KXS);
    // slot segments of the frozen entries start at a tile boundary: up to two extra slices; the
    // first chunk of a continuation also evaluates its carried pilots (up to W/2 more rows)
    w.max_slices = (g.D + g.slice - 1) / g.slice + 2;
    w.part_rows = g.T + g.W / 2;
    for (int i = 0; i < 2; ++i) {
        w.partial[i] = off;
        if (i == 0 || g.track) off = align256(off + sizeof(float) * (size_t)w.max_slices * w.part_rows * 2 * g.K);
    }
    for (int i = 0; i < 2; ++i) {
        w.track[i] = off;
        if (g.track) off = align256(off + sizeof(float) * (size_t)g.KXS * g.K);
    }
    w.carry = off;
    off = align256(off + sizeof(float) * (size_t)g.W * g.K);
    w.ext_rx = off;
    if (ext) off = align256(off + sizeof(float2) * (size_t)g.P * g.M);
    w.ext_sym = off;
    if (ext) off = align256(off + sizeof(float2) * (size_t)g.P * g.K);
    w.total = g.n_chunks > 0 ? off : 0;
    return w;
}

// Workspace bound of a continuation of P vectors, whatever n_prev (carried pilots at most W/2,
// with or without eviction).
size_t continue_ws_bytes(const apsm_params *p, int P) {
    const int n_prev = p->window / 2;  // the largest carried count
    const size_t a = train_ws(train_geom(p, P, n_prev, 0), true).total;
    const size_t b = train_ws(train_geom(p, P, n_prev, 1), true).total;
    return std::max(a, b);
}

// The extended sequence of a training call: rows [0, nc0) are the carried pilots, read from
// their dictionary slots with the targets they were trained on; rows [nc0, nc0 + P) are the new
// vectors and their targets (zero when they are to be decided).
__global__ void train_ext_kernel(const float2 *__restrict__ rx, const float2 *__restrict__ sym, int P, int nc0,
                                 int t_base, int D, int M, int K, const float2 *__restrict__ dict,
                                 const float2 *__restrict__ target, float2 *ext_rx, float2 *ext_sym) {
    pdl_enter();
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    for (int i = tid; i < (nc0 + P) * M; i += nthr) {
        const int e = i / M, m = i % M;
        ext_rx[i] = e < nc0 ? __ldcg(dict + (size_t)((t_base + e) % D) * M + m) : rx[(size_t)(e - nc0) * M + m];
    }
    for (int i = tid; i < (nc0 + P) * K; i += nthr) {
        const int e = i / K, k = i % K;
        ext_sym[i] = e < nc0 ? __ldcg(target + (size_t)((t_base + e) % D) * K + k)
                             : (sym ? sym[(size_t)(e - nc0) * K + k] : make_float2(0.f, 0.f));
    }
}

int qam_half_of(const apsm_params *p) { return (p->modulation == 0 ? 2 : p->modulation) / 2; }
float qam_a_of(const apsm_params *p) {
    const int L = 1 << qam_half_of(p);
    return (float)std::sqrt(3.0 / (2.0 * ((double)L * L - 1.0)));
}

// Gray square-QAM labels of soft outputs (the same FP32 values the detection wrote).
__global__ void qam_label_kernel(const float2 *__restrict__ soft, uint8_t *__restrict__ hard, long long n, int half,
                                 float a) {
    pdl_enter();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float2 y = __ldcg(soft + i);
        hard[i] = qam_label(y.x, y.y, half, a);
    }
}

apsm_status qam_labels(float *soft, uint8_t *hard, int N, const apsm_params *p, cudaStream_t strm) {
    const long long n = (long long)N * p->K;
    const int blocks = (int)std::max<long long>(1, std::min<long long>(4 * num_sms(), (n + 255) / 256));
    if (launch_pdl(qam_label_kernel, dim3(blocks), dim3(256), 0, strm, reinterpret_cast<const float2 *>(soft), hard,
                   n, qam_half_of(p), qam_a_of(p)) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess)
        return APSM_ERR_CUDA;
    g_launches++;
    return APSM_OK;
}

__global__ void state_set_kernel(const float2 *__restrict__ entries, const float *__restrict__ gamma,
                                 const float2 *__restrict__ clin, const float2 *__restrict__ target, int n, int M,
                                 int K, float2 *dict, float *dict_norm, float *gam_out, float2 *clin_out,
                                 float2 *tgt_out, int *meta) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    for (int i = tid; i < n * M; i += nthr) dict[i] = entries[i];
    for (int i = tid; i < n * K; i += nthr) tgt_out[i] = target ? target[i] : make_float2(0.f, 0.f);
    for (int i = tid; i < n * 2 * K; i += nthr) gam_out[i] = gamma[i];
    for (int i = tid; i < M * K; i += nthr) clin_out[i] = clin[i];
    for (int t = tid; t < n; t += nthr) {
        float s = 0.f;
        for (int m = 0; m < M; ++m) {
            const float2 v = entries[(size_t)t * M + m];
            s = fmaf(v.x, v.x, fmaf(v.y, v.y, s));
        }
        dict_norm[t] = s;
    }
    if (tid == 0) {
        meta[0] = n;
        meta[1] = 0;
        meta[2] = n;
        meta[3] = 0;
    }
}

// ---- detection adjoint geometry -----------------------------------------------------------
struct BwdGeom {
    int A, n_qslices, q_per_slice, n_cslices;
    size_t gh, cpart, scal, total;
};

BwdGeom bwd_geom(const apsm_params *p, int N) {
    BwdGeom b;
    b.A = round_up(p->dict_cap, kTileEntries);
    const int entry_ctas = (p->dict_cap + kBwdEntriesPerCta - 1) / kBwdEntriesPerCta;
    const int want = std::max(1, (2 * 152 + entry_ctas - 1) / entry_ctas);  // ~2 CTAs per SM
    b.n_qslices = N > 0 ? std::min(want, (N + kBwdQueryTile - 1) / kBwdQueryTile) : 0;
    b.q_per_slice = b.n_qslices ? round_up((N + b.n_qslices - 1) / b.n_qslices, kBwdQueryTile) : 0;
    if (b.q_per_slice) b.n_qslices = (N + b.q_per_slice - 1) / b.q_per_slice;
    b.n_cslices = N > 0 ? std::min(256, (N + 127) / 128) : 0;
    size_t off = 0;
    b.gh = off;
    off = align256(off + sizeof(float) * (size_t)b.n_qslices * b.A * 4 * p->K);
    b.cpart = off;
    off = align256(off + sizeof(float) * 2 * (size_t)b.n_cslices * p->M * p->K);
    b.scal = off;
    off = align256(off + sizeof(float) * 2 * (size_t)b.A * 2 * p->K);
    b.total = off;
    return b;
}

// apsm_read_status: the status word is exchanged with 0 and the old value parked in a
// library-owned device slot, from which the host copies it.
__device__ int32_t g_status_slot;
std::mutex g_status_mu;
__global__ void status_take_kernel(int *status) { g_status_slot = atomicExch(status, 0); }

// Failure-detection self-check: one CTA waits on an mbarrier that no thread arrives at (its
// phase 0 never completes), through the bounded wait of every kernel; when the wait budget runs
// out the status word gets APSM_ERR_TIMEOUT and the CTA returns.
__global__ void wait_timeout_check_kernel(int *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();  // the initialisation is visible before any thread waits
    const bool done = mbar_wait_bounded(&bar, 0);
    if (!done && threadIdx.x == 0) report(status, APSM_ERR_TIMEOUT);
}

}  // namespace

// The launch-choice table forces the FMA engine for this class (batch.cu follows it).
bool tune_forces_ffma(int M, int K, int dtype) {
    const TuneEntry te = tune_get(M, K, dtype);
    return te.set && te.engine == 1;
}

}  // namespace apsm

using namespace apsm;

extern "C" {

apsm_status apsm_dict_alloc(const apsm_params *p, int32_t *dict_alloc) {
    apsm_status s = check_params(p);
    if (s != APSM_OK) return s;
    if (!dict_alloc) return APSM_ERR_INVALID_ARG;
    *dict_alloc = round_up(p->dict_cap, kTileEntries);
    return APSM_OK;
}

apsm_status apsm_train_workspace_bytes(const apsm_params *p, int32_t P, size_t *bytes) {
    apsm_status s = check_params(p);
    if (s != APSM_OK) return s;
    if (!bytes || P < 0) return APSM_ERR_INVALID_ARG;
    *bytes = train_ws(train_geom(p, P, 0), false).total;
    return APSM_OK;
}

apsm_status apsm_train_continue_workspace_bytes(const apsm_params *p, int32_t P, size_t *bytes) {
    apsm_status s = check_params(p);
    if (s != APSM_OK) return s;
    if (!bytes || P < 0) return APSM_ERR_INVALID_ARG;
    *bytes = continue_ws_bytes(p, P);
    return APSM_OK;
}

}  // extern "C"

namespace apsm {
namespace {

// One training call (apsm_train: fresh = true, n_prev = 0; apsm_train_continue otherwise): P new
// vectors rx with targets sym (NULL: decided at arrival) after n_prev earlier ones.
apsm_status train_run(const apsm_params *p, const float *rx_in, const float *sym_in, int P, int n_prev,
                      const apsm_state *st, void *workspace, size_t workspace_bytes, float *soft, uint8_t *hard,
                      int8_t *case_log, cudaStream_t strm) {
    const bool decide = sym_in == nullptr;
    const TrainGeom g = train_geom(p, P, n_prev);
    const bool ext = g.nc0 > 0 || decide;
    const TrainWs ws = train_ws(g, ext);
    if (ws.total > 0 && (!workspace || workspace_bytes < ws.total)) return APSM_ERR_WORKSPACE;
    if (ws.total > 0 && (reinterpret_cast<uintptr_t>(workspace) & 255)) return APSM_ERR_INVALID_ARG;
    if (P == 0) return APSM_OK;

    unsigned char *wsb = static_cast<unsigned char *>(workspace);
    float *kmat = reinterpret_cast<float *>(wsb + ws.kmat);
    float *gev = reinterpret_cast<float *>(wsb + ws.gev);
    float *kx = reinterpret_cast<float *>(wsb + ws.kx);
    float *partial[2] = {reinterpret_cast<float *>(wsb + ws.partial[0]), reinterpret_cast<float *>(wsb + ws.partial[1])};
    float *track[2] = {reinterpret_cast<float *>(wsb + ws.track[0]), reinterpret_cast<float *>(wsb + ws.track[1])};
    float *carry = reinterpret_cast<float *>(wsb + ws.carry);
    const float k2 = k2_of(p->sigma);
    const float wL = p->w_L, wG = 1.f - p->w_L;
    const float2 *rx = reinterpret_cast<const float2 *>(rx_in);
    float2 *sym = const_cast<float2 *>(reinterpret_cast<const float2 *>(sym_in));  // written only when decided
    if (ext) {  // the extended sequence: carried pilots (from their slots) + the new vectors
        float2 *erx = reinterpret_cast<float2 *>(wsb + ws.ext_rx);
        float2 *esym = reinterpret_cast<float2 *>(wsb + ws.ext_sym);
        const int work = g.P * std::max(g.M, g.K);
        const int blocks = std::max(1, std::min(2 * num_sms(), (work + 255) / 256));
        if (launch_pdl(train_ext_kernel, dim3(blocks), dim3(256), 0, strm, rx, reinterpret_cast<const float2 *>(sym_in),
                       P, g.nc0, g.t_base, g.D, g.M, g.K, reinterpret_cast<const float2 *>(st->dict),
                       reinterpret_cast<const float2 *>(st->target), erx, esym) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess)
            return APSM_ERR_CUDA;
        g_launches++;
        rx = erx;
        sym = esym;
    }

    {   // kernel values of every chunk's live range, of dropped entries against it, and against
        // the next chunk's samples
        if (launch_train_gram(rx, reinterpret_cast<const float2 *>(st->dict), g, k2, wL, wG, kmat, gev, kx, strm) !=
            cudaSuccess)
            return APSM_ERR_CUDA;
        g_launches++;
    }

    DetectLauncher det = detect_f32_launcher(p->M, p->K);
    if (!det) return APSM_ERR_UNSUPPORTED;
    const ChunkSmem layout(g);
    // the extended instantiation only for the modes that need it
    const bool ext_modes = decide || soft != nullptr || hard != nullptr || p->weights == APSM_Q_VIOLATED;
    const ChunkLauncher chunk = chunk_launcher(g.RS / 32, g.WP, ext_modes);
    if (!chunk) return APSM_ERR_UNSUPPORTED;

    // phase A: the partial Gaussian sums of f, at the extended pilots [q0, q0 + nq), over the
    // dictionary entries with running indices [lo, lo + n) (their slots mod D) -- the whole
    // dictionary, or its frozen entries
    auto phase_a = [&](int q0, int nq, int lo, int n, float *dst, int &n_slices, bool late) -> bool {
        DetectArgs da{};
        da.rx = rx + (size_t)q0 * g.M;
        da.N = nq;
        da.dict = reinterpret_cast<const float2 *>(st->dict);
        da.dict_norm = st->dict_norm;
        da.gamma = st->gamma;
        da.clin = reinterpret_cast<const float2 *>(st->clin);
        da.meta = nullptr;
        da.n_entries = g.D;
        da.slice_entries = g.slice;
        da.k2 = k2;
        da.wL = wL;
        da.wG = wG;
        da.partial = dst;
        da.pdl_late = late ? 1 : 0;
        da.status = st->meta + 3;
        const int first = lo % g.D, hi0 = std::min(g.D, first + n), hi1 = first + n - g.D;
        da.seg0_lo = first;
        da.seg0_hi = hi0;
        const int ns0 = (hi0 - first / g.slice * g.slice + g.slice - 1) / g.slice;
        int ns1 = 0;
        if (hi1 > 0) {
            da.seg1_lo = 0;
            da.seg1_hi = hi1;
            ns1 = (hi1 + g.slice - 1) / g.slice;
        }
        da.seg_slices = ns0;
        n_slices = ns0 + ns1;
        const int thr = std::min(256, round_up(nq, 32));
        const DetectShape sh{thr, std::max(1, 256 / thr), 1};  // entry groups share each tile
        if (det(da, n_slices, sh, strm) != cudaSuccess) return false;
        g_launches++;
        return true;
    };

    const int tb = g.t_base;
    int slices_of[2] = {0, 0};  // phase-A slices waiting in partial[c & 1]
    for (int c = 0; c < g.n_chunks; ++c) {
        int t0, Tc, s0, s1, l0;
        chunk_range(g, c, t0, Tc, s0, s1, l0);
        int mode = 0, part_p0 = t0, part_rows = Tc, fresh_carry = 0;
        const bool cont0 = c == 0 && n_prev > 0;  // first chunk of a continuation: dictionary not empty
        if (cont0 || !g.track) {
            // f at the chunk start over the whole dictionary, between the chunks (in the first chunk
            // of a continuation also at the carried pilots, whose predictions start from it)
            const int held = std::min(tb + t0, g.D);
            if (cont0) {
                part_p0 = l0 / 2;
                part_rows = t0 + Tc - part_p0;
                fresh_carry = g.nc0 > 0 ? 1 : 0;
            }
            slices_of[0] = 0;
            if (held > 0) {
                if (!phase_a(part_p0, part_rows, tb + t0 - held, held, partial[0], slices_of[0], false))
                    return APSM_ERR_CUDA;
                mode = 2;
            }
        } else {
            // the previous launch is the previous chunk's phase B or this chunk's frozen-entry
            // phase A; either way the kernel tables are complete
            mode = c > 0 ? 1 : 0;
        }
        ChunkArgs ca{};
        ca.g = g;
        ca.chunk = c;
        ca.mu = p->mu;
        ca.eps = p->eps;
        ca.wL = wL;
        ca.wG = wG;
        ca.rx = rx;
        ca.sym = sym;
        ca.dict = reinterpret_cast<float2 *>(st->dict);
        ca.dict_norm = st->dict_norm;
        ca.gamma = st->gamma;
        ca.clin = reinterpret_cast<float2 *>(st->clin);
        ca.meta = st->meta;
        ca.kmat = kmat;
        ca.gev = gev;
        const int pb = (g.track && !cont0) ? (c & 1) : 0;  // the tracked form alternates two phase-A buffers
        ca.partial = partial[pb];
        ca.n_slices = slices_of[pb];
        ca.part_p0 = part_p0;
        ca.part_rows = part_rows;
        ca.fresh_carry = fresh_carry;
        ca.carry = carry;
        ca.case_log = case_log;
        ca.target = st->target;
        ca.soft_out = soft;
        ca.hard_out = hard;
        ca.decide = decide ? 1 : 0;
        ca.qviol = p->weights == APSM_Q_VIOLATED ? 1 : 0;
        ca.qam_half = qam_half_of(p);
        ca.qam_a = qam_a_of(p);
        if (g.track) {
            ca.kx = kx + (size_t)c * g.RS * g.KXS;
            ca.track_in = (c > 0) ? track[c & 1] : nullptr;
            ca.track_out = c + 1 < g.n_chunks ? track[(c + 1) & 1] : nullptr;
        }
        ca.pdl_mode = mode;
        if (chunk(ca, layout.bytes, strm) != cudaSuccess) return APSM_ERR_CUDA;
        g_launches++;
        if (g.track && c + 1 < g.n_chunks) {
            // frozen part of the next chunk's starting filter: entries older than this chunk's live
            // range still held at the next chunk's start.  Their coefficients are final once the
            // previous chunk's phase B completed, which this chunk's phase B waits for before it
            // lets this launch start; it runs beside this chunk's phase B.
            int t0n, Tcn, s0n, s1n, l0n;
            chunk_range(g, c + 1, t0n, Tcn, s0n, s1n, l0n);
            const int f0 = std::max(0, tb + t0n - g.D), f1 = tb + l0 / 2;
            slices_of[(c + 1) & 1] = 0;
            if (f1 > f0 &&
                !phase_a(t0n, Tcn, f0, f1 - f0, partial[(c + 1) & 1], slices_of[(c + 1) & 1], true))
                return APSM_ERR_CUDA;
        }
    }
    return APSM_OK;
}

apsm_status check_train_args(const apsm_params *p, const float *rx, const float *sym, int P, const apsm_state *st,
                             bool sym_required) {
    apsm_status s = check_params(p);
    if (s != APSM_OK) return s;
    if ((s = check_state(st)) != APSM_OK) return s;
    if (P < 0 || (P > 0 && (!rx || (sym_required && !sym)))) return APSM_ERR_INVALID_ARG;
    if (P > (1 << 26)) return APSM_ERR_INVALID_ARG;
    if (P > 0 && (!aligned16(rx) || (reinterpret_cast<uintptr_t>(sym) & 7))) return APSM_ERR_INVALID_ARG;
    return APSM_OK;
}

}  // namespace
}  // namespace apsm

extern "C" {

apsm_status apsm_train(const apsm_params *p, const float *rx_pilot, const float *sym_pilot, int32_t P,
                       const float *clin0, const apsm_state *st, void *workspace, size_t workspace_bytes,
                       int8_t *case_log, void *stream) {
    apsm_status s = check_train_args(p, rx_pilot, sym_pilot, P, st, true);
    if (s != APSM_OK) return s;
    if (clin0 && (reinterpret_cast<uintptr_t>(clin0) & 7)) return APSM_ERR_INVALID_ARG;
    const TrainWs ws = train_ws(train_geom(p, P, 0), false);
    if (ws.total > 0 && (!workspace || workspace_bytes < ws.total)) return APSM_ERR_WORKSPACE;
    if (ws.total > 0 && (reinterpret_cast<uintptr_t>(workspace) & 255)) return APSM_ERR_INVALID_ARG;
    if ((s = check_device()) != APSM_OK) return s;
    cudaStream_t strm = static_cast<cudaStream_t>(stream);

    // f_0: linear part clin0 (or zero), empty Gaussian part
    const size_t clin_bytes = sizeof(float) * 2 * (size_t)p->M * p->K;
    cudaError_t ce = clin0 == nullptr ? cudaMemsetAsync(st->clin, 0, clin_bytes, strm)
                     : clin0 != st->clin ? cudaMemcpyAsync(st->clin, clin0, clin_bytes, cudaMemcpyDeviceToDevice, strm)
                                         : cudaSuccess;
    if (ce != cudaSuccess) return APSM_ERR_CUDA;
    if (P == 0) return cuda_status(cudaMemsetAsync(st->meta, 0, 3 * sizeof(int32_t), strm));
    return train_run(p, rx_pilot, sym_pilot, P, 0, st, workspace, workspace_bytes, nullptr, nullptr, case_log, strm);
}

apsm_status apsm_train_continue(const apsm_params *p, const float *rx, const float *sym, int32_t P, int32_t n_prev,
                                const apsm_state *st, void *workspace, size_t workspace_bytes, float *soft,
                                uint8_t *hard, int8_t *case_log, void *stream) {
    apsm_status s = check_train_args(p, rx, sym, P, st, false);
    if (s != APSM_OK) return s;
    if (n_prev < 0 || n_prev > (1 << 30) - P) return APSM_ERR_INVALID_ARG;
    if ((soft && (reinterpret_cast<uintptr_t>(soft) & 7))) return APSM_ERR_INVALID_ARG;
    if (P > 0 && (!workspace || continue_ws_bytes(p, P) > workspace_bytes)) return APSM_ERR_WORKSPACE;
    if (P > 0 && (reinterpret_cast<uintptr_t>(workspace) & 255)) return APSM_ERR_INVALID_ARG;
    if ((s = check_device()) != APSM_OK) return s;
    return train_run(p, rx, sym, P, n_prev, st, workspace, workspace_bytes, soft, hard, case_log,
                     static_cast<cudaStream_t>(stream));
}

apsm_status apsm_detect_ws(const apsm_params *p, const apsm_state *st, const float *rx, int32_t N, float *soft,
                           uint8_t *hard, void *workspace, size_t workspace_bytes, void *stream) {
    apsm_status s = check_params(p);
    if (s != APSM_OK) return s;
    if ((s = check_state(st)) != APSM_OK) return s;
    if (N < 0 || (N > 0 && (!rx || !soft))) return APSM_ERR_INVALID_ARG;
    if (N > 0 && (!aligned16(rx) || (reinterpret_cast<uintptr_t>(soft) & 7))) return APSM_ERR_INVALID_ARG;
    if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255)) return APSM_ERR_INVALID_ARG;
    if ((s = check_device()) != APSM_OK) return s;
    if (N == 0) return APSM_OK;
    cudaStream_t strm = static_cast<cudaStream_t>(stream);
    // square-QAM labels: the detection kernel writes QPSK decisions only; labels of larger
    // constellations are formed from the soft outputs by one extra pass
    const bool qam_pass = hard != nullptr && qam_half_of(p) > 1;
    // Engine: the Gram on the tensor cores (TF32 x3 for FP32, BF16/FP16 as requested) where a
    // kernel exists for (M, K); FFMA otherwise, or where the tuning table chose it for FP32.
    const TuneEntry te = tune_get(p->M, p->K, p->dtype);
    const bool force_ffma = te.set && te.engine == 1;
    if (p->dtype != APSM_FP32 || !force_ffma) {
        const int prec = p->dtype == APSM_FP32 ? kTF32x3 : kHalf;
        TcLauncher tc = detect_tc_launcher(p->M, p->K, prec);
        // BF16/FP16 with a workspace: the coefficient sums on the tensor cores too
        TccLauncher tcc = (prec == kHalf && workspace && g_opt_half_tc_coef.load()) ? detect_tcc_launcher(p->M, p->K)
                                                                                     : nullptr;
        TmaLauncher tma = (p->dtype == APSM_FP32 && g_opt_detect_tma.load()) ? detect_tma_launcher(p->M, p->K) : nullptr;
        if (tc || tma) {
            TcArgs ta{};
            ta.rx = reinterpret_cast<const float2 *>(rx);
            ta.N = N;
            ta.dict = reinterpret_cast<const float2 *>(st->dict);
            ta.dict_norm = st->dict_norm;
            ta.gamma = st->gamma;
            ta.clin = reinterpret_cast<const float2 *>(st->clin);
            ta.meta = st->meta;
            ta.n_entries = p->dict_cap;
            ta.K = p->K;
            ta.half_fmt = p->dtype == APSM_BF16 ? 1 : 0;
            ta.k2 = k2_of(p->sigma);
            ta.wL = p->w_L;
            ta.wG = 1.f - p->w_L;
            ta.soft = reinterpret_cast<float2 *>(soft);
            ta.hard = hard;
            ta.status = st->meta + 3;
            if (qam_pass) ta.hard = nullptr;
            // the TMA-staged form where it applies (shape, alignment; balanced over the SMs with a
            // workspace), else the converter form
            int sms = 0;
            if (tma && workspace && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, current_device()) != cudaSuccess)
                return APSM_ERR_CUDA;
            const int r = tma ? tma(ta, workspace, workspace_bytes, sms, strm) : 1;
            if (r < 0) return APSM_ERR_CUDA;
            if (r > 0 && tcc) {
                if (tcc(ta, workspace, workspace_bytes, strm) != cudaSuccess) return APSM_ERR_CUDA;
                g_launches++;  // (the packing launch)
            } else if (r > 0 && (!tc || tc(ta, strm) != cudaSuccess)) {
                return tc ? APSM_ERR_CUDA : APSM_ERR_UNSUPPORTED;
            }
            g_launches++;
            return qam_pass ? qam_labels(soft, hard, N, p, strm) : APSM_OK;
        }
        if (p->dtype != APSM_FP32) return APSM_ERR_UNSUPPORTED;
    }
    DetectLauncher det = detect_f32_launcher(p->M, p->K);
    if (!det) return APSM_ERR_UNSUPPORTED;
    DetectArgs da{};
    da.rx = reinterpret_cast<const float2 *>(rx);
    da.N = N;
    da.dict = reinterpret_cast<const float2 *>(st->dict);
    da.dict_norm = st->dict_norm;
    da.gamma = st->gamma;
    da.clin = reinterpret_cast<const float2 *>(st->clin);
    da.meta = st->meta;
    da.n_entries = p->dict_cap;
    da.slice_entries = round_up(p->dict_cap, kTileEntries);
    da.k2 = k2_of(p->sigma);
    da.wL = p->w_L;
    da.wG = 1.f - p->w_L;
    da.soft = reinterpret_cast<float2 *>(soft);
    da.hard = hard;
    da.partial = nullptr;
    da.status = st->meta + 3;
    if (qam_pass) da.hard = nullptr;
    const DetectShape sh = detect_shape(p->M, p->K, p->dtype);
    if (det(da, 1, sh, strm) != cudaSuccess) return APSM_ERR_CUDA;
    g_launches++;
    return qam_pass ? qam_labels(soft, hard, N, p, strm) : APSM_OK;
}

apsm_status apsm_detect(const apsm_params *p, const apsm_state *st, const float *rx, int32_t N, float *soft,
                        uint8_t *hard, void *stream) {
    return apsm_detect_ws(p, st, rx, N, soft, hard, nullptr, 0, stream);
}

apsm_status apsm_detect_workspace_bytes(const apsm_params *p, int32_t N, size_t *bytes) {
    if (!bytes) return APSM_ERR_INVALID_ARG;
    *bytes = 0;
    apsm_status s = check_params(p);
    if (s != APSM_OK) return s;
    if (N < 0) return APSM_ERR_INVALID_ARG;
    if (N == 0) return APSM_OK;
    if (p->dtype != APSM_FP32) {  // the packed operands of the reduced-precision form
        if (g_opt_half_tc_coef.load()) *bytes = detect_tcc_workspace(p->M, p->K, p->dict_cap);
        return APSM_OK;
    }
    if (!detect_tma_launcher(p->M, p->K)) return APSM_OK;
    if ((s = check_device()) != APSM_OK) return s;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, current_device()) != cudaSuccess)
        return APSM_ERR_CUDA;
    *bytes = tma_workspace(N, p->K, 2 * sms).total;
    return APSM_OK;
}

apsm_status apsm_state_set(const apsm_params *p, const float *entries, const float *gamma, const float *clin,
                           const float *target, int32_t n, const apsm_state *st, void *stream) {
    apsm_status s = check_params(p);
    if (s != APSM_OK) return s;
    if ((s = check_state(st)) != APSM_OK) return s;
    if (n < 0 || n > p->dict_cap || !clin || (n > 0 && (!entries || !gamma))) return APSM_ERR_INVALID_ARG;
    if (target && (reinterpret_cast<uintptr_t>(target) & 7)) return APSM_ERR_INVALID_ARG;
    if ((s = check_device()) != APSM_OK) return s;
    const int work = std::max(n * p->M, std::max(n * 2 * p->K, p->M * p->K));
    const int blocks = std::max(1, std::min(1024, (work + 255) / 256));
    state_set_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float2 *>(entries), gamma, reinterpret_cast<const float2 *>(clin),
        reinterpret_cast<const float2 *>(target), n, p->M, p->K, reinterpret_cast<float2 *>(st->dict), st->dict_norm,
        st->gamma, reinterpret_cast<float2 *>(st->clin), reinterpret_cast<float2 *>(st->target), st->meta);
    g_launches++;
    return cuda_status(cudaGetLastError());
}

apsm_status apsm_detect_backward_workspace_bytes(const apsm_params *p, int32_t N, size_t *bytes) {
    apsm_status s = check_params(p);
    if (s != APSM_OK) return s;
    if (!bytes || N < 0) return APSM_ERR_INVALID_ARG;
    *bytes = bwd_geom(p, N).total;
    return APSM_OK;
}

apsm_status apsm_detect_backward(const apsm_params *p, const apsm_state *st, const float *rx, int32_t N,
                                 const float *dsoft, float *dgamma, float *dclin, float *dscalars, void *workspace,
                                 size_t workspace_bytes, void *stream) {
    apsm_status s = check_params(p);
    if (s != APSM_OK) return s;
    if ((s = check_state(st)) != APSM_OK) return s;
    if (N < 0 || (N > 0 && (!rx || !dsoft)) || !dgamma || !dclin || !dscalars) return APSM_ERR_INVALID_ARG;
    if (N > 0 && (!aligned16(rx) || (reinterpret_cast<uintptr_t>(dsoft) & 7))) return APSM_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(dgamma) & 3) || (reinterpret_cast<uintptr_t>(dclin) & 7) ||
        (reinterpret_cast<uintptr_t>(dscalars) & 3))
        return APSM_ERR_INVALID_ARG;
    if (p->dtype != APSM_FP32) return APSM_ERR_UNSUPPORTED;
    const BwdGeom b = bwd_geom(p, N);
    if (!workspace || workspace_bytes < b.total) return APSM_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return APSM_ERR_INVALID_ARG;
    if ((s = check_device()) != APSM_OK) return s;
    DetectBwdLauncher bwd = detect_bwd_launcher(p->M, p->K);
    if (!bwd) return APSM_ERR_UNSUPPORTED;
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    DetectBwdArgs a{};
    a.rx = reinterpret_cast<const float2 *>(rx);
    a.dsoft = reinterpret_cast<const float2 *>(dsoft);
    a.N = N;
    a.dict = reinterpret_cast<const float2 *>(st->dict);
    a.dict_norm = st->dict_norm;
    a.gamma = st->gamma;
    a.clin = reinterpret_cast<const float2 *>(st->clin);
    a.meta = st->meta;
    a.n_entries = p->dict_cap;
    a.A = b.A;
    a.q_per_slice = b.q_per_slice;
    a.n_qslices = b.n_qslices;
    a.n_cslices = b.n_cslices;
    a.k2 = k2_of(p->sigma);
    a.wL = p->w_L;
    a.wG = 1.f - p->w_L;
    a.sigma = p->sigma;
    a.gh = reinterpret_cast<float *>(ws + b.gh);
    a.cpart = reinterpret_cast<float2 *>(ws + b.cpart);
    a.scal = reinterpret_cast<float *>(ws + b.scal);
    a.dgamma = dgamma;
    a.dclin = reinterpret_cast<float2 *>(dclin);
    a.dscalars = dscalars;
    if (bwd(a, static_cast<cudaStream_t>(stream)) != cudaSuccess) return APSM_ERR_CUDA;
    g_launches += N > 0 ? 4 : 2;
    return APSM_OK;
}

apsm_status apsm_tune_set(int32_t M, int32_t K, int32_t dtype, int32_t engine, int32_t threads, int32_t split,
                          int32_t qpt) {
    if (m_slot(M) == 0 || K < 1 || K > 16 || dtype < 0 || dtype > 2 || (engine != 0 && engine != 1))
        return APSM_ERR_INVALID_ARG;
    if (engine == 1 && (threads < 32 || threads > 256 || threads % 32 || split < 1 || split * threads > 256 ||
                        (qpt != 1 && qpt != 2)))
        return APSM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[m_slot(M)][K][dtype] = TuneEntry{1, engine, threads, split, qpt};
    return APSM_OK;
}

apsm_status apsm_set_option(int32_t option, int32_t value) {
    switch (option) {
        case APSM_OPT_TRAIN_CHUNK:
            if (value < 1 || value > 1024) return APSM_ERR_INVALID_ARG;
            g_opt_train_chunk.store(value);
            return APSM_OK;
        case APSM_OPT_TRAIN_TRACK:
            if (value != 0 && value != 1) return APSM_ERR_INVALID_ARG;
            g_opt_train_track.store(value);
            return APSM_OK;
        case APSM_OPT_DETECT_TMA:
            if (value != 0 && value != 1) return APSM_ERR_INVALID_ARG;
            g_opt_detect_tma.store(value);
            return APSM_OK;
        case APSM_OPT_HALF_TC_COEF:
            if (value != 0 && value != 1) return APSM_ERR_INVALID_ARG;
            g_opt_half_tc_coef.store(value);
            return APSM_OK;
        default: return APSM_ERR_INVALID_ARG;
    }
}

apsm_status apsm_tune_clear(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    std::memset(g_tune, 0, sizeof(g_tune));
    return APSM_OK;
}

apsm_status apsm_check_wait_timeout(const apsm_state *st, void *stream) {
    if (!st || !st->meta) return APSM_ERR_INVALID_ARG;
    apsm_status s = check_device();
    if (s != APSM_OK) return s;
    wait_timeout_check_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(st->meta + 3);
    return cudaGetLastError() == cudaSuccess ? APSM_OK : APSM_ERR_CUDA;
}

apsm_status apsm_read_status(const apsm_state *st, int32_t *device_status, void *stream) {
    if (!st || !st->meta || !device_status) return APSM_ERR_INVALID_ARG;
    apsm_status s = check_device();
    if (s != APSM_OK) return s;
    cudaStream_t strm = static_cast<cudaStream_t>(stream);
    // one atomic read-and-clear in stream order (a status a kernel on another stream writes
    // afterwards stays for the next call), then a copy of the read value on the same stream; the
    // slot is library-owned, so concurrent callers are serialised on the host
    std::lock_guard<std::mutex> lock(g_status_mu);
    status_take_kernel<<<1, 1, 0, strm>>>(st->meta + 3);
    int32_t v = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyFromSymbolAsync(&v, g_status_slot, sizeof(v), 0, cudaMemcpyDeviceToHost, strm) != cudaSuccess ||
        cudaStreamSynchronize(strm) != cudaSuccess) {
        cudaGetLastError();
        return APSM_ERR_CUDA;
    }
    *device_status = v;
    return APSM_OK;
}

const char *apsm_status_string(apsm_status s) {
    switch (s) {
        case APSM_OK: return "ok";
        case APSM_ERR_INVALID_ARG: return "invalid argument";
        case APSM_ERR_UNSUPPORTED: return "unsupported shape";
        case APSM_ERR_CUDA: return "CUDA runtime error";
        case APSM_ERR_TIMEOUT: return "device-side wait timed out";
        case APSM_ERR_NOT_SM103: return "device is not sm_103";
        case APSM_ERR_WORKSPACE: return "workspace too small";
    }
    return "unknown status";
}

int64_t apsm_launch_count(void) { return g_launches.load(); }

}  // extern "C"
