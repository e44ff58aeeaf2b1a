/*
 * apsm.h -- C ABI of the GB300 (sm_103a) APSM multiuser detector library (libapsm_gb300.so).
 *
 * The method is the adaptive projected subgradient method (APSM) for partially linear
 * multiuser detection of arXiv 2201.05024:
 *   - filters live in the weighted sum space H = H_L + H_G with reproducing kernel
 *     kappa = w_L kappa_L + w_G kappa_G (Sec. II-A/B, Fact 1), kappa_L(u,v) = u^T v and
 *     kappa_G(u,v) = exp(-||u - v||^2 / (2 sigma^2));
 *   - a complex received vector r in C^M is processed as the two real vectors
 *     r1 = [Re r; Im r] and r2 = [Im r; -Re r]; one real filter f per user gives the
 *     complex soft symbol g(r) = f(r1) + i f(r2) (Sec. II-D);
 *   - training runs the concurrent hyperslab projections of Eq. apsm / Eq. beta over the
 *     window J_n of the last W real-split samples (Sec. II-D); detection evaluates the trained
 *     expansion (Sec. III-B).
 *
 * Conventions shared by every entry point:
 *   - Complex arrays are interleaved (re, im) float32 pairs (the layout of torch.complex64 /
 *     C99 float _Complex).  Every pointer whose comment says "device" must point to memory of
 *     the current CUDA device; the caller allocates and owns all of it -- the library keeps no
 *     allocation between calls and makes none inside them.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls enqueue work on it and
 *     return without synchronising; results are valid once the stream has reached them.
 *   - Arrays of received vectors (rx_pilot, rx) and the state's dict, dict_norm and gamma must be
 *     16-byte aligned (they are read with 16-byte vector loads and bulk copies); other arrays
 *     need the alignment of their element type.  Misaligned pointers give APSM_ERR_INVALID_ARG.
 *   - Host-side argument errors return at once, before any CUDA call.  A device-side error
 *     (a bounded wait that ran out) is written to meta[3] of the state and reported by
 *     apsm_read_status().
 *   - No C++ exception crosses this boundary.  The library runs on sm_103 devices only and
 *     returns APSM_ERR_NOT_SM103 elsewhere; it has no CPU fallback.
 *   - Results are deterministic: no floating-point atomics, fixed reduction orders.
 */
#ifndef APSM_GB300_H
#define APSM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    APSM_OK = 0,
    APSM_ERR_INVALID_ARG = 1,  /* a size, pointer or parameter outside its documented range   */
    APSM_ERR_UNSUPPORTED = 2,  /* a valid shape this build has no kernel for (see apsm_params) */
    APSM_ERR_CUDA = 3,         /* a CUDA runtime call failed (no device, launch failure, ...)  */
    APSM_ERR_TIMEOUT = 4,      /* a device-side bounded wait ran out (reported via meta[3])    */
    APSM_ERR_NOT_SM103 = 5,    /* the current device is not compute capability 10.3            */
    APSM_ERR_WORKSPACE = 6     /* the workspace passed is smaller than the size queried        */
} apsm_status;

typedef enum { APSM_FP32 = 0, APSM_BF16 = 1, APSM_FP16 = 2 } apsm_dtype;

/*
 * Algorithm parameters (Sec. II-D and Sec. V of the paper; the readings of open points are
 * stated per field).
 *   M        antennas, i.e. complex dimension of r(t); the real-split dimension is 2M.
 *            Supported: 2, 4, 8, 16, 32, 64.
 *   K        users (one filter per user, all trained on the same received vectors, Sec. III-B).
 *            Supported: 1..16.
 *   window   W >= 1: number of hyperslabs projected concurrently, counted in real-split samples
 *            (J_n = {n-W+1, .., n}, Sec. II-D).  Supported: 1..128.
 *   dict_cap D: Gaussian dictionary capacity in entries; one entry is one complex pilot r(t)
 *            and carries both centres r1(t), r2(t).  The paper's dictionary grows without
 *            bound; here the oldest entry is dropped (FIFO) once D are held.  Requires 2D > W.
 *   sigma    Gaussian kernel width sigma > 0 (kappa_G uses 2 sigma^2; the paper's default
 *            variance sigma^2 = 0.05).
 *   mu       relaxation of the projection step, 0 < mu <= 2; mu = 1 is Eq. apsm as printed.
 *   eps      hyperslab half-width epsilon >= 0 (Eq. convex_set).
 *   w_L      weight of the linear kernel in [0, 1]; the Gaussian weight is w_G = 1 - w_L.
 *   dtype    apsm_dtype of the detection contractions; training always runs in FP32.
 *   modulation  bits per symbol of the Gray square QAM used for hard decisions and for the
 *            decision-directed targets of apsm_train_continue: 2 (QPSK; 0 is read as 2), 4
 *            (16-QAM) or 6 (64-QAM), unit mean energy (Sec. V, Fig. modulation).  One axis has
 *            L = 2^(modulation/2) levels (2i - (L-1)) a, a = sqrt(3 / (2 (L^2 - 1))); the
 *            decision is the number of boundaries (2i - L) a at or below the value (a value on a
 *            boundary takes the upper level; QPSK: the sign, 0 counting as non-negative); the
 *            label is the Gray code of (L-1-level) per axis, real axis in the low bits.
 *   weights  APSM_Q_UNIFORM: q_j = 1/|J_n| over the window; APSM_Q_VIOLATED: q_j = 1/|V_n| over
 *            the violated slabs V_n = {j in J_n : |e_j| > eps}, 0 elsewhere (Sec. II-D: the
 *            weights may adaptively prioritise).  The adjoint supports APSM_Q_UNIFORM only.
 */
typedef enum { APSM_Q_UNIFORM = 0, APSM_Q_VIOLATED = 1 } apsm_weights;

typedef struct {
    int32_t M;
    int32_t K;
    int32_t window;
    int32_t dict_cap;
    float sigma;
    float mu;
    float eps;
    float w_L;
    int32_t dtype;
    int32_t modulation;
    int32_t weights;
} apsm_params;

/*
 * Detector state: the trained filters f^k of all users (Sec. II-D decomposition
 * f_n = f_L,n + f_G,n).  All DEVICE pointers, caller-allocated with the sizes below, where
 * A = apsm_dict_alloc() >= dict_cap.
 *   dict       [A][M] complex  ring buffer of dictionary entries r(t); entry t sits in slot t % D
 *   dict_norm  [A]     float   ||r(t)||^2 of each slot
 *   gamma      [A][2][K] float Gaussian coefficients of centre r1(t) (index 0) and r2(t)
 *                               (index 1), unweighted (w_G is applied when evaluating)
 *   clin       [M][K] complex  linear part as complex filter c_k = w_k[0:M] + i w_k[M:2M], so
 *                               that w_k^T r1 = Re(c_k^H r) and w_k^T r2 = Im(c_k^H r)
 *                               (unweighted: w_L is applied when evaluating).
 *   meta       [4] int32       [0] entries held, [1] slot of the oldest entry,
 *                               [2] vectors consumed, [3] device status (apsm_status code)
 *   target     [A][K] complex  the target each held entry was trained on (its pilot symbol, or
 *                               the decision taken in decision-directed mode); read when
 *                               training continues, to carry the window across calls.
 * Slot of the vector with running index t (counted over all training calls since the state was
 * emptied) is t % D.  Slots at or beyond meta[0] are never read by the kernels.
 */
typedef struct {
    float *dict;
    float *dict_norm;
    float *gamma;
    float *clin;
    int32_t *meta;
    float *target;
} apsm_state;

/* Number of dictionary slots A (>= dict_cap) the state arrays must hold. */
apsm_status apsm_dict_alloc(const apsm_params *p, int32_t *dict_alloc);

/* Bytes of device workspace apsm_train needs for P pilots (0 is possible). */
apsm_status apsm_train_workspace_bytes(const apsm_params *p, int32_t P, size_t *bytes);

/*
 * Training (Eq. apsm with Eq. beta over the window J_n, Sec. II-D; Fig. training of Sec. III-B).
 * Runs the recurrence over the 2P real-split samples of P pilots, starting from f_0 whose
 * linear part is clin0 (zero when NULL; Sec. I/II-D: f_0 is arbitrary, e.g. a conventional
 * linear filter) and whose Gaussian part is empty; on return (stream order) the state holds
 * f_{2P}: at most D entries, their coefficients, clin and meta.  Every state array is
 * overwritten, so a state can be retrained without clearing it.
 *   rx_pilot   device [P][M] complex  received pilot vectors r(t)
 *   sym_pilot  device [P][K] complex  transmitted pilot symbols b_k(t) (targets: b_{2t} = Re,
 *                                     b_{2t+1} = Im, Sec. II-D)
 *   P          pilots, >= 0
 *   clin0      device [M][K] complex, initial linear filter, or NULL for zero; may alias st->clin
 *   st         state (output)
 *   workspace  device scratch of at least apsm_train_workspace_bytes(p, P) bytes (may be NULL
 *              when that size is 0), 256-byte aligned
 *   case_log   optional device [2P][W][K] int8: for step n and window slot o (sample
 *              j = n - W + 1 + o) the branch of Eq. beta taken: -1 (residual < -eps),
 *              0 (inside the slab), +1 (residual > eps); slots with j < 0 are left untouched.
 * Errors: APSM_ERR_INVALID_ARG (null pointer, P < 0, parameter out of range, 2D <= W),
 * APSM_ERR_UNSUPPORTED (M, K or W outside the supported sets), APSM_ERR_WORKSPACE,
 * APSM_ERR_NOT_SM103, APSM_ERR_CUDA.
 */
apsm_status apsm_train(const apsm_params *p, const float *rx_pilot, const float *sym_pilot, int32_t P,
                       const float *clin0, const apsm_state *st, void *workspace, size_t workspace_bytes,
                       int8_t *case_log, void *stream);

/* Bytes of device workspace apsm_train_continue needs for P further vectors (any n_prev). */
apsm_status apsm_train_continue_workspace_bytes(const apsm_params *p, int32_t P, size_t *bytes);

/*
 * Continue training a state on P further vectors (Eq. apsm / Eq. beta over the window J_n,
 * Sec. II-D): the recurrence goes on from the state exactly as if these vectors had followed the
 * earlier ones in one apsm_train call -- the window reaches back into the previous call's last
 * samples (their targets are kept in st->target), the dictionary ring and its FIFO eviction go on.
 * With sym == NULL the targets are decided (decision-directed tracking through the data symbols,
 * Sec. II-D): the target of real-split sample n is the Gray-QAM decision (p->modulation) on the
 * filter's own output at its arrival, b_n = Q(f_n(x_n)).
 *   rx       device [P][M] complex    received vectors
 *   sym      device [P][K] complex    their targets, or NULL for decision-directed targets
 *   P        >= 0
 *   n_prev   vectors the state has consumed so far (its meta[2]): the caller's count of every
 *            vector trained on since the state was emptied (0 continues an empty Gaussian part
 *            whose linear part is st->clin as it stands)
 *   st       state, updated in place
 *   workspace  apsm_train_continue_workspace_bytes(p, P) bytes, 256-byte aligned
 *   soft     device [P][K] complex, or NULL: the filter's output at each vector's arrival,
 *            f_{2t}(r1(t)) + i f_{2t+1}(r2(t)) (each half before its own projection; for tracking
 *            these are the detector's outputs)
 *   hard     device [P][K] uint8, or NULL: the Gray-QAM labels of the targets trained on (the
 *            decisions, in decision-directed mode)
 *   case_log as for apsm_train, for the P new vectors' steps.
 * Errors as for apsm_train; APSM_ERR_INVALID_ARG also for n_prev < 0.
 */
apsm_status apsm_train_continue(const apsm_params *p, const float *rx, const float *sym, int32_t P, int32_t n_prev,
                                const apsm_state *st, void *workspace, size_t workspace_bytes, float *soft,
                                uint8_t *hard, int8_t *case_log, void *stream);

/*
 * Conventional linear start of the filter (Sec. I: start from a linear MMSE/ZF detector; f_0 is
 * arbitrary in Eq. apsm).  From P pilots it forms the least-squares channel estimate
 *   H = Y S^H (S S^H)^-1        (Y = [r(0) .. r(P-1)] M x P, S = pilot symbols K x P)
 * and the MMSE filter W = H (H^H H + noise_var I)^-1 (zero-forcing for noise_var = 0), whose soft
 * estimates are W^H r, and writes clin0 = W / w_L, so that the linear part of f_0 (weighted by
 * w_L) detects exactly as W.  One CTA, FP32, fixed-order sums.
 *   rx_pilot, sym_pilot  device, as for apsm_train; P >= K
 *   noise_var            >= 0 (per receive antenna, relative to unit symbol energy)
 *   clin0                device [M][K] complex output (pass it to apsm_train)
 * Errors: APSM_ERR_INVALID_ARG (P < K, w_L = 0, noise_var < 0 or not finite, null or misaligned
 * pointers), APSM_ERR_NOT_SM103, APSM_ERR_CUDA.  When S S^H or H^H H + noise_var I is not
 * positive definite in FP32 (the pilot symbols do not span K independent directions) clin0 is
 * set to zero.
 */
apsm_status apsm_linear_init(const apsm_params *p, const float *rx_pilot, const float *sym_pilot, int32_t P,
                             float noise_var, float *clin0, void *stream);

/*
 * apsm_train_noalloc -- apsm_train for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a deployment variant of apsm_train, not part of the
 * method.  Callers such as a real-time receive loop that must not allocate once it runs, or a
 * plug-in whose host framework owns all device memory, cannot provide apsm_train's workspace;
 * this entry point uses scratch memory that is part of the library instead: a fixed array of
 * APSM_NOALLOC_SCRATCH_BYTES that every device loading the library holds until process exit.
 * Arguments and results are those of apsm_train without workspace/workspace_bytes.
 *   - It calls no cudaMalloc, cudaFree or other allocating routine.
 *   - Training that needs more scratch than the array holds (apsm_train_workspace_bytes(p, P)
 *     > APSM_NOALLOC_SCRATCH_BYTES) is rejected with APSM_ERR_WORKSPACE before any work.
 *   - The first call in a CUDA context (one per device in the usual case of the primary
 *     context), with that device current, looks up the array's device address there
 *     (cudaGetSymbolAddress) and caches it for that context, so a context created anew after
 *     cudaDeviceReset gets a fresh lookup; make that first call before any stream capture.
 *   - All calls on a device share the one array, which keeps the last call's contents (the
 *     training writes every scratch word before reading it).  Calls whose GPU work overlaps --
 *     on different streams, or from different threads -- race on it: serialise them.
 */
#define APSM_NOALLOC_SCRATCH_BYTES (8u << 20)
apsm_status apsm_train_noalloc(const apsm_params *p, const float *rx_pilot, const float *sym_pilot, int32_t P,
                               const float *clin0, const apsm_state *st, int8_t *case_log, void *stream);

/*
 * Detection (Sec. III-B, Fig. detection): for every data vector r and user k,
 *   soft[n][k] = f^k(r1) + i f^k(r2),
 *   f^k(x) = w_L <w_k, x> + w_G sum_{alive centres i} gamma_i^k kappa_G(c_i, x),
 * and the Gray square-QAM decision hard[n][k] of soft[n][k] (p->modulation; QPSK:
 * (Re soft < 0) | (Im soft < 0) << 1, an exact zero counting as non-negative).  The number of
 * alive entries is read from st->meta[0] on the device, so a detection queued behind apsm_train
 * on the same stream needs no host synchronisation.
 * The squared distances are formed from one complex inner product per (vector, entry) pair
 * (norm expansion).  Where that cancels -- the smallest of a pair's three distances below
 * theta k2 (||r||^2 + ||r_t||^2), theta = 2^-4 for BF16/FP16 contractions and 2^-12 for FP32 with
 * inputs outside the factored range -- the pair's distances are recomputed by direct
 * differences in FP32 (direct-difference fallback).
 *   rx    device [N][M] complex      data vectors
 *   N     >= 0
 *   soft  device [N][K] complex      output
 *   hard  device [N][K] uint8        output, may be NULL
 * p->dtype selects the contraction precision (APSM_FP32 here).
 * Errors as for apsm_train.
 */
apsm_status apsm_detect(const apsm_params *p, const apsm_state *st, const float *rx, int32_t N, float *soft,
                        uint8_t *hard, void *stream);

/*
 * Detection with a workspace (the same results as apsm_detect up to rounding order; Sec. III-B
 * detection).  FP32 detection with 4, 8 or 16 antennas and an even user count in
 * {2, 4, 6, 8, 12, 16} splits its (query tile, dictionary tile) work evenly over a persistent
 * grid; a query tile split between CTAs leaves each part's sums in the workspace and the CTA
 * that brings its last part adds the parts in a fixed order (results do not depend on timing).
 * BF16/FP16 detection with 16, 32 or 64 antennas packs the dictionary's operands into the
 * workspace once per call and forms the coefficient sums on the tensor cores too (see
 * APSM_OPT_HALF_TC_COEF): the exponentials rounded to BF16 against the coefficients as a BF16
 * hi + lo pair, accumulated in FP32.
 *   apsm_detect_workspace_bytes: bytes for N data vectors on the current device; 0 where the
 *     balanced form does not apply (apsm_detect_ws then runs apsm_detect).
 *   workspace  device, 256-byte aligned, at least that many bytes, ZERO-FILLED before its first
 *     use.  It starts with one arrival counter per 128 data vectors (int32); every call that
 *     completes without a status error leaves them at zero again (the rest is scratch).  After
 *     a status error, fill the workspace with zeros again before the next call.  One workspace
 *     per call in flight (calls that overlap on different streams need different workspaces).
 *     NULL: apsm_detect.
 * Other arguments and errors as for apsm_detect; APSM_ERR_INVALID_ARG for an unaligned
 * workspace.  A workspace smaller than the balanced form needs runs apsm_detect.
 */
apsm_status apsm_detect_workspace_bytes(const apsm_params *p, int32_t N, size_t *bytes);
apsm_status apsm_detect_ws(const apsm_params *p, const apsm_state *st, const float *rx, int32_t N, float *soft,
                           uint8_t *hard, void *workspace, size_t workspace_bytes, void *stream);

/* Bytes of device workspace apsm_detect_backward needs for N data vectors. */
apsm_status apsm_detect_backward_workspace_bytes(const apsm_params *p, int32_t N, size_t *bytes);

/*
 * Adjoint of apsm_detect (not in the paper: the gradient of the detection of Sec. III-B with
 * respect to the filter and the kernel parameters).  Given dsoft = dL/d(soft) for a real loss L
 * (as complex numbers: dL/dRe + i dL/dIm), with soft = f(r1) + i f(r2) and
 * f(x) = w_L <w, x> + w_G sum_i gamma_i kappa_G(c_i, x) (Fact 1, Sec. II-D):
 *   dgamma[t][l][k] = w_G sum_s (dRe_s^k kappa_G(c_tl, r1(s)) + dIm_s^k kappa_G(c_tl, r2(s)))
 *   dclin[m][k]     = w_L sum_s conj(dsoft[s][k]) r_s[m]      (gradient with respect to Re c + i Im c)
 *   dscalars[0]     = dL/dsigma,  dscalars[1] = dL/dw_L  (with w_G = 1 - w_L)
 * Exponentials are recomputed.  Deterministic (fixed-order reductions, no atomics).
 *   rx        device [N][M] complex, the data vectors of the forward call
 *   dsoft     device [N][K] complex
 *   dgamma    device [A][2][K] float out (slots beyond the entries held are set to 0)
 *   dclin     device [M][K] complex out
 *   dscalars  device [2] float out
 *   workspace device scratch of apsm_detect_backward_workspace_bytes(p, N) bytes, 256-byte aligned
 * Errors as for apsm_detect, plus APSM_ERR_WORKSPACE.
 */
apsm_status apsm_detect_backward(const apsm_params *p, const apsm_state *st, const float *rx, int32_t N,
                                 const float *dsoft, float *dgamma, float *dclin, float *dscalars, void *workspace,
                                 size_t workspace_bytes, void *stream);

/* Bytes of device workspace apsm_train_backward needs for P pilots. */
apsm_status apsm_train_backward_workspace_bytes(const apsm_params *p, int32_t P, size_t *bytes);

/*
 * Adjoint of apsm_train (not in the paper: gradients through the unrolled recurrence of Eq. apsm
 * with Eq. beta, Sec. II-D).  Given the gradient of a loss with respect to the trained state --
 * dgamma [A][2][K] (ring layout of apsm_state.gamma, e.g. from apsm_detect_backward) and
 * dclin [M][K] complex (dL/dRe c + i dL/dIm c) -- it returns
 *   dscalars[4] = {dL/dsigma, dL/dmu, dL/deps, dL/dw_L} through the training only, and
 *   dclin0 [M][K] complex = dL/d(initial linear filter c_0).
 * The derivative of Eq. beta is taken piecewise: -1/kappa_jj with respect to the residual and
 * -+1/kappa_jj with respect to eps outside the slab, 0 inside it (and at |e| = eps exactly).
 * The forward recurrence is run once, carrying the window's predictions from step to step, and
 * its per-step terms are kept in the workspace; the reverse sweep forms a centre's adjoint when
 * the centre enters the window, so both passes cost O(W^2 + P) per step.
 *   rx_pilot, sym_pilot, P, clin0: as given to apsm_train (clin0 may be NULL for zero), P >= 1
 *   workspace: apsm_train_backward_workspace_bytes(p, P) bytes, 256-byte aligned
 * All pointers DEVICE.  Deterministic.  Errors as for apsm_train.
 */
apsm_status apsm_train_backward(const apsm_params *p, const float *rx_pilot, const float *sym_pilot, int32_t P,
                                const float *clin0, const float *dgamma, const float *dclin, float *dscalars,
                                float *dclin0, void *workspace, size_t workspace_bytes, void *stream);

/* Bytes of device workspace apsm_train_backward_batched needs for n instances of P pilots. */
apsm_status apsm_train_backward_batched_workspace_bytes(const apsm_params *p, int32_t P, int32_t n, size_t *bytes);

/*
 * apsm_train_backward for n independent instances with the same parameters and pilot count, in
 * one launch per kernel (users x instances thread blocks).  Instance i's arrays follow instance
 * i-1's, each in the layout of apsm_train_backward:
 *   rx_pilot [n][P][M], sym_pilot [n][P][K] complex; clin0 [n][M][K] complex or NULL (zero);
 *   dgamma [n][A][2][K]; dclin [n][M][K] complex; dscalars [n][4] out; dclin0 [n][M][K] out.
 * Each instance's results equal those of its own apsm_train_backward call bit for bit.
 *   n: 1..65535; workspace: apsm_train_backward_batched_workspace_bytes(p, P, n) bytes, 256-byte aligned.
 * All pointers DEVICE.  Errors as for apsm_train_backward.
 */
apsm_status apsm_train_backward_batched(const apsm_params *p, int32_t n, const float *rx_pilot, const float *sym_pilot,
                                        int32_t P, const float *clin0, const float *dgamma, const float *dclin,
                                        float *dscalars, float *dclin0, void *workspace, size_t workspace_bytes,
                                        void *stream);

/*
 * apsm_train_backward_batched in two calls on one workspace, so that the first can run before
 * the loss gradient exists (e.g. beside the detection and its adjoint):
 *   _forward: the kernel tables and the forward pass of the recurrence of every instance, whose
 *             per-step terms it keeps in the workspace (arguments as for apsm_train_backward_batched);
 *   _reverse: the reverse sweep over that workspace, given dgamma and dclin; the same results, bit
 *             for bit, as apsm_train_backward_batched.
 * rx_pilot, P, n and the parameters must be those of the _forward call on the same workspace, and
 * _forward must precede _reverse in stream order.  All pointers DEVICE.
 */
apsm_status apsm_train_backward_batched_forward(const apsm_params *p, int32_t n, const float *rx_pilot,
                                                const float *sym_pilot, int32_t P, const float *clin0,
                                                void *workspace, size_t workspace_bytes, void *stream);
apsm_status apsm_train_backward_batched_reverse(const apsm_params *p, int32_t n, const float *rx_pilot, int32_t P,
                                                const float *dgamma, const float *dclin, float *dscalars,
                                                float *dclin0, void *workspace, size_t workspace_bytes,
                                                void *stream);

/*
 * Load a given filter into a state (detection with fixed, externally trained coefficients):
 * entries [n][M] complex, gamma [n][2][K], clin [M][K] complex and target [n][K] complex (the
 * entries' training targets, read only if training continues from this state; NULL: zero), all
 * DEVICE, in age order (oldest first), 0 <= n <= dict_cap.  Writes slots 0..n-1, their norms
 * ||r||^2, clin, the targets and meta = {n, 0, n, 0}, so that training can continue with
 * n_prev = n.  Same expansion as Sec. II-D: f^k = w_L <w_k, .> + w_G sum gamma kappa_G.
 */
apsm_status apsm_state_set(const apsm_params *p, const float *entries, const float *gamma, const float *clin,
                           const float *target, int32_t n, const apsm_state *st, void *stream);

/*
 * Detection launch choice for one class (M, K, dtype), set by the autotuner
 * (paper_2201_05024_gb300/autotune.py, not part of the method): engine 0 = Gram on the tensor
 * cores, 1 = FP32 FMA pipe with `threads` query lanes x `split` entry groups per CTA and `qpt`
 * queries per lane (ignored for engine 0).  Classes never set use built-in defaults.  The table
 * is process-wide; apsm_tune_clear empties it.
 */
apsm_status apsm_tune_set(int32_t M, int32_t K, int32_t dtype, int32_t engine, int32_t threads, int32_t split,
                          int32_t qpt);
apsm_status apsm_tune_clear(void);

/*
 * Batched form (not in the paper: many independent detectors -- cells, resource blocks -- of
 * uneven antenna count, user count, dictionary size and data length).  One instance:
 */
typedef struct {
    apsm_params p;             /* its parameters (M, K, window, dict_cap, kernel parameters)   */
    int32_t P;                 /* pilots                                                       */
    int32_t N;                 /* data vectors                                                 */
    const float *rx_pilot;     /* device [P][M] complex                                        */
    const float *sym_pilot;    /* device [P][K] complex                                        */
    const float *rx;           /* device [N][M] complex                                        */
    float *soft;               /* device [N][K] complex                                        */
    uint8_t *hard;             /* device [N][K] or NULL                                        */
    apsm_state st;             /* its state (apsm_dict_alloc(&p) slots)                        */
    void *workspace;           /* device, apsm_train_workspace_bytes(&p, P) bytes              */
    size_t workspace_bytes;
} apsm_instance;

typedef struct apsm_batch_s *apsm_batch;

/*
 * Bytes of device workspace apsm_batch_create needs for these instances (the work lists of the
 * persistent detection launches; 0 when no instance is in the batched kernel's range).
 */
apsm_status apsm_batch_workspace_bytes(const apsm_instance *inst, int32_t n, size_t *bytes);

/*
 * Record the whole batch into one CUDA graph:
 *   training   -- apsm_train (from f_0 = 0) of every instance, spread over `lanes` (1..64) parallel
 *                 graph branches, longest first, each onto the currently least-loaded branch;
 *   detection  -- per class (antenna count, user bucket of K) ONE persistent launch whose resident
 *                 CTAs take (instance, 128-vector tile) work items from a device counter, listed
 *                 longest instance first, until none is left (the counters are reset by memset
 *                 nodes of the graph).  This covers FP32 detection up to 32 antennas with QPSK
 *                 decisions (or no hard output) in classes the launch-choice table does not give
 *                 to the FMA engine; any other instance is detected by apsm_detect on its
 *                 branch after its training.  Per instance the outputs equal apsm_train followed
 *                 by apsm_detect bit for bit.
 * The descriptors (and the buffers they point to) are bound at creation: apsm_batch_launch replays
 * the same work on new data in the same buffers.  Every instance is validated before anything is
 * recorded.  workspace: apsm_batch_workspace_bytes bytes, 256-byte aligned, caller-owned, kept
 * for the life of the batch (written once here, synchronously).  The handle owns the graphs.
 */
apsm_status apsm_batch_create(const apsm_instance *inst, int32_t n, int32_t lanes, void *workspace,
                              size_t workspace_bytes, apsm_batch *out);
/* Launch the whole batch (one graph launch) on `stream`. */
apsm_status apsm_batch_launch(apsm_batch b, void *stream);
/* Launch only the persistent detection phase (a second graph; for timing it alone). */
apsm_status apsm_batch_launch_detect(apsm_batch b, void *stream);
/* Number of classes detected by persistent launches and of instances in them. */
apsm_status apsm_batch_info(apsm_batch b, int32_t *n_classes, int32_t *n_batched);
apsm_status apsm_batch_destroy(apsm_batch b);

/* Read and clear the device status word meta[3] in one atomic exchange enqueued on `stream`,
 * then wait for `stream` and return the value read in *device_status.  A status that a kernel
 * on another stream writes after the exchange stays for the next call.  Returns APSM_ERR_CUDA if
 * the stream fails. */
apsm_status apsm_read_status(const apsm_state *st, int32_t *device_status, void *stream);

/* Failure-detection self-check.  Enqueues on `stream` one CTA that waits, through the same bounded
 * mbarrier wait every kernel of the library uses, on a barrier that no thread ever arrives at.
 * The wait gives up after the library's wait budget (about two seconds of SM clock), the kernel
 * writes APSM_ERR_TIMEOUT to the state's status word (meta[3]) and returns, so that the context
 * stays usable: apsm_read_status() then reports APSM_ERR_TIMEOUT.  Nothing else of the state is
 * touched.  Returns APSM_ERR_INVALID_ARG for a null state, APSM_ERR_CUDA if the launch fails. */
apsm_status apsm_check_wait_timeout(const apsm_state *st, void *stream);

/*
 * Process-wide launch options (not part of the method; every setting gives the same results up
 * to FP32 rounding order):
 *   APSM_OPT_TRAIN_CHUNK  pilots per training chunk (1..1024, default 64; shared memory may
 *                         lower it further)
 *   APSM_OPT_TRAIN_TRACK  1 (default): the next chunk's starting predictions are tracked during
 *                         the current chunk; 0: they are evaluated between chunks (sequential)
 *   APSM_OPT_DETECT_TMA   1 (default): FP32 detection with 4, 8 or 16 antennas and an even user
 *                         count in {2, 4, 6, 8, 12, 16} stages every operand by TMA (entry rows
 *                         as stored, the real split's rotation on the query side); 0: the
 *                         tensor-core form that converts entry rows in shared memory
 *   APSM_OPT_HALF_TC_COEF 1 (default): BF16/FP16 detection with 16, 32 or 64 antennas forms the
 *                         coefficient sums on the tensor cores too (the exponentials rounded to
 *                         BF16, the coefficients as a BF16 hi + lo pair, FP32 accumulation);
 *                         0: coefficient sums in FP32 on the FMA pipe
 * Returns APSM_ERR_INVALID_ARG for an unknown option or a value out of range.
 */
typedef enum {
    APSM_OPT_TRAIN_CHUNK = 0,
    APSM_OPT_TRAIN_TRACK = 1,
    APSM_OPT_DETECT_TMA = 2,
    APSM_OPT_HALF_TC_COEF = 3
} apsm_option;
apsm_status apsm_set_option(int32_t option, int32_t value);

/* Static description of a status code. */
const char *apsm_status_string(apsm_status s);

/* Number of kernels this library has launched in this process (for launch accounting). */
int64_t apsm_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* APSM_GB300_H */
