/*
 * apsm_oracle.c -- plain FP64 CPU oracle of the APSM partially linear multiuser
 * detector of arXiv 2201.05024 (Sec. II).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file; the product (the CUDA library and its
 * binding) never does, and this file shares no code, header, table or helper
 * with it.
 *
 * It is deliberately slow and literal:
 *   - vectors are the real split of Sec. II-D, formed explicitly
 *     (x_{2t} = [Re r(t); Im r(t)], x_{2t+1} = [Im r(t); -Re r(t)],
 *      b_{2t} = Re s(t), b_{2t+1} = Im s(t));
 *   - Gaussian kernels use the direct difference ||u - v||^2 (Sec. II-A);
 *   - every window prediction is recomputed from the full expansion of f_n at
 *     every step (no incremental update, no Gram trick);
 *   - all projections of one step use the same f_n (Eq. apsm);
 *   - one user at a time, one step at a time, in FP64.
 *
 * Readings of points the paper leaves open (each is a parameter or a choice
 * made once here):
 *   - relaxation mu multiplies the projection step (mu = 1 is Eq. apsm as printed);
 *   - weights q_j are uniform, 1/|J_n|, unless the violated-slab weighting below is chosen;
 *   - W counts real-split samples n (Sec. II-D index);
 *   - the Gaussian dictionary holds at most D entries, one entry per complex
 *     pilot r(t) carrying both centres x_{2t}, x_{2t+1}; when full, the oldest
 *     entry (both centres and their coefficients) is dropped before the new one
 *     joins with zero coefficients; the linear part keeps the dropped samples'
 *     contribution because the linear dictionary is the fixed Euclidean basis
 *     (Sec. II-D, decomposition of f_n); 2D > W is required;
 *   - f_0 has no Gaussian part; its linear part w0 is given (zero by default);
 *   - w_G = 1 - w_L;
 *   - kappa(x_j, x_j) = 0 (only possible when w_L = 1 and x_j = 0) gives beta = 0;
 *   - |e| == eps lies inside the hyperslab (Eq. beta, middle case);
 *   - adaptive weights (Sec. II-D leaves q_j free beyond q_j >= 0, sum q_j = 1): either
 *     uniform over the window, or uniform over the violated slabs V_n = {j in J_n : |e_j| > eps}
 *     and 0 elsewhere (no update when V_n is empty);
 *   - decision-directed targets (Sec. II-D, tracking through the data symbols): a sample's
 *     target is the decision on the filter's own output at its arrival, b_n = Q(f_n(x_n)), with
 *     Q the slicer of one real axis of a Gray square QAM (each real-split sample carries one
 *     axis of the complex symbol);
 *   - continuing a trained filter on further vectors is the same recurrence over the
 *     concatenated sequence, so it needs no separate definition here.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int M;          /* receive antennas; real-split dimension is 2M           */
    int K;          /* users                                                  */
    int W;          /* window size |J_n| for n >= W-1 (Sec. II-D)             */
    int D;          /* dictionary capacity in entries (complex pilots)        */
    double sigma;   /* Gaussian kernel width: exp(-||u-v||^2 / (2 sigma^2))   */
    double mu;      /* relaxation of the concurrent projection step           */
    double eps;     /* hyperslab half-width epsilon (Eq. convex_set)          */
    double w_L;     /* weight of the linear kernel; w_G = 1 - w_L (Fact 1)    */
    int qam_bits;   /* Gray square QAM of decided targets: 2 (QPSK), 4, 6 bits */
    int weights;    /* 0: q_j = 1/|J_n|;  1: q_j = 1/|V_n| on violated slabs  */
} apsm_oracle_params;

/* One real axis of a Gray square QAM with 2^bits points and unit mean energy: L = 2^(bits/2)
 * amplitude levels (2i - (L-1)) a, i = 0..L-1, a = sqrt(3 / (2 (L^2 - 1))), separated by the
 * decision boundaries (2i - L) a, i = 1..L-1.  The slicer returns the nearest level: its index
 * is the number of boundaries at or below y (a value on a boundary takes the upper level; for
 * QPSK this is the sign test with 0 counting as non-negative); it writes the index to *level
 * when level is not NULL. */
double apsm_oracle_pam_slice(double y, int bits, int *level)
{
    const int L = 1 << (bits / 2);
    const double a = sqrt(3.0 / (2.0 * ((double)L * L - 1.0)));
    int i = 0;
    for (int b = 1; b < L; ++b)
        if (y >= (2.0 * b - L) * a) i += 1;
    if (level) *level = i;
    return (2.0 * i - (L - 1)) * a;
}

/* Real split of one complex vector r (interleaved re,im, length M) -- Sec. II-D. */
static void real_split(int M, const double *r, double *x1, double *x2)
{
    for (int m = 0; m < M; ++m) {
        double re = r[2 * m], im = r[2 * m + 1];
        x1[m] = re;      x1[M + m] = im;    /* r1 = [Re r; Im r]  */
        x2[m] = im;      x2[M + m] = -re;   /* r2 = [Im r; -Re r] */
    }
}

/* Linear kernel kappa_L(u, v) = u^T v -- Sec. II-A. */
static double kappa_lin(int L, const double *u, const double *v)
{
    double s = 0.0;
    for (int i = 0; i < L; ++i) s += u[i] * v[i];
    return s;
}

/* Gaussian kernel kappa_G(u, v) = exp(-||u - v||^2 / (2 sigma^2)) -- Sec. II-A. */
static double kappa_gauss(int L, const double *u, const double *v, double sigma)
{
    double d2 = 0.0;
    for (int i = 0; i < L; ++i) {
        double d = u[i] - v[i];
        d2 += d * d;
    }
    return exp(-d2 / (2.0 * sigma * sigma));
}

/* f(x) = w_L <w, x> + w_G sum_i gamma_i kappa_G(c_i, x): the value <f, kappa(x, .)>_H of an
 * element of the sum space H = H_L + H_G (Fact 1, Eq. sum_inner_product, with the
 * decomposition f_n = f_L,n + f_G,n of Sec. II-D).  gamma has stride gstride. */
static double eval_f(int L, const double *w, int n_c, const double *cent, const double *gamma,
                     int gstride, const double *x, double sigma, double w_L)
{
    double lin = kappa_lin(L, w, x);
    double gs = 0.0;
    for (int i = 0; i < n_c; ++i)
        gs += gamma[(size_t)i * gstride] * kappa_gauss(L, cent + (size_t)i * L, x, sigma);
    return w_L * lin + (1.0 - w_L) * gs;
}

/* Real-split centres of complex dictionary entries: entry t holds x_{2t} = r1(t) and
 * x_{2t+1} = r2(t).  entries [n][M][2] -> centres [2n][2M]. */
void apsm_oracle_centres(int M, int n, const double *entries, double *centres)
{
    for (int t = 0; t < n; ++t)
        real_split(M, entries + (size_t)t * 2 * M, centres + (size_t)(2 * t) * 2 * M,
                   centres + (size_t)(2 * t + 1) * 2 * M);
}

/* Evaluate f^k at real vectors x[q] for q in [q0, q1):
 *   y[q][k] = w_L w_k^T x_q + w_G sum_i gamma[i][k] kappa_G(c_i, x_q).
 * cent [n_c][2M], gamma [n_c][K], w [K][2M], x [n_x][2M], y [n_x][K]. */
void apsm_oracle_eval(const apsm_oracle_params *p, int n_c, const double *cent, const double *gamma,
                      const double *w, int q0, int q1, const double *x, double *y)
{
    const int L = 2 * p->M, K = p->K;
    for (int q = q0; q < q1; ++q)
        for (int k = 0; k < K; ++k)
            y[(size_t)q * K + k] = eval_f(L, w + (size_t)k * L, n_c, cent, gamma + k, K,
                                          x + (size_t)q * L, p->sigma, p->w_L);
}

/* Detection (Sec. II-D, Sec. III-B): for complex data vectors r[q] (interleaved [N][M][2]),
 * y[q][k][0] = f^k(r1(q)), y[q][k][1] = f^k(r2(q)); the complex soft estimate of user k is
 * g^k(r) = f^k(r1) + i f^k(r2).  Queries [q0, q1). */
void apsm_oracle_detect(const apsm_oracle_params *p, int n_c, const double *cent,
                        const double *gamma, const double *w, int q0, int q1,
                        const double *rx, double *y)
{
    const int M = p->M, L = 2 * M, K = p->K;
    double *x1 = (double *)malloc(sizeof(double) * (size_t)L);
    double *x2 = (double *)malloc(sizeof(double) * (size_t)L);
    for (int q = q0; q < q1; ++q) {
        real_split(M, rx + (size_t)q * 2 * M, x1, x2);
        for (int k = 0; k < K; ++k) {
            y[((size_t)q * K + k) * 2 + 0] =
                eval_f(L, w + (size_t)k * L, n_c, cent, gamma + k, K, x1, p->sigma, p->w_L);
            y[((size_t)q * K + k) * 2 + 1] =
                eval_f(L, w + (size_t)k * L, n_c, cent, gamma + k, K, x2, p->sigma, p->w_L);
        }
    }
    free(x1);
    free(x2);
}

/*
 * Training (Eq. apsm with Eq. beta, window J_n of Sec. II-D), users k in [k0, k1).
 *
 * Inputs:  rx [P][M][2] pilots, sym [P][K][2] pilot symbols, w0 [K][2M] or NULL.
 *          n_steps = number of real-split steps n = 0 .. n_steps-1 (<= 2P; < 0 means 2P).
 * Outputs: w_out [K][2M]            linear coefficients (rows k0..k1-1 written);
 *          gamma_out [2D][K]        Gaussian coefficients of the alive centres in age order
 *                                   (columns k0..k1-1 written);
 *          alive_out [2]            first alive entry, number of alive entries (written when k0 == 0);
 *          case_log [n_steps][W][K] (nullable) -1: e < -eps, 0: |e| <= eps, +1: e > eps, for window
 *                                   slot o = j - n + W - 1 (slots with j < 0 are left untouched);
 *          margin_log [n_steps][W][K] (nullable) | |e| - eps |;
 *          forced [n_steps][W][K]   (nullable) a value in {-1, 0, 1} forces that case for the slot
 *                                   (replay of a run that took another branch at a tie); any other
 *                                   value leaves the slot free;
 *          decide_from              samples n >= decide_from take the decision b_n = Q(f_n(x_n))
 *                                   as their target (sym is not read for them); n_steps or more:
 *                                   every target comes from sym;
 *          pred_out [P][K][2]       (nullable) f_n(x_n) at each sample's arrival n = 2t + l;
 *          target_out [P][K][2]     (nullable) the target each sample was trained on.
 * Returns 0, or -1 on invalid arguments / allocation failure.
 */
int apsm_oracle_train(const apsm_oracle_params *p, int P, int n_steps, const double *rx,
                      const double *sym, const double *w0, int k0, int k1, double *w_out,
                      double *gamma_out, int *alive_out, signed char *case_log,
                      double *margin_log, const signed char *forced, int decide_from,
                      double *pred_out, double *target_out)
{
    const int M = p->M, L = 2 * M, K = p->K, W = p->W, D = p->D;
    if (M < 1 || K < 1 || W < 1 || D < 1 || P < 0 || 2 * D <= W || p->sigma <= 0.0) return -1;
    if (n_steps < 0 || n_steps > 2 * P) n_steps = 2 * P;
    const double w_G = 1.0 - p->w_L;

    /* Real-split training samples (x_n, b_n), n = 2t + l (Sec. II-D). */
    double *x = (double *)malloc(sizeof(double) * (size_t)(2 * P + 1) * L);
    double *g = (double *)malloc(sizeof(double) * (size_t)(2 * P + 1));
    double *beta = (double *)malloc(sizeof(double) * (size_t)W);
    double *tgt = (double *)malloc(sizeof(double) * (size_t)(2 * P + 1));
    int *cs_win = (int *)malloc(sizeof(int) * (size_t)W);
    if (!x || !g || !beta || !tgt || !cs_win) { free(x); free(g); free(beta); free(tgt); free(cs_win); return -1; }
    for (int t = 0; t < P; ++t)
        real_split(M, rx + (size_t)t * 2 * M, x + (size_t)(2 * t) * L, x + (size_t)(2 * t + 1) * L);

    int first = 0, t_last = 0;
    for (int k = k0; k < k1; ++k) {
        double *w = w_out + (size_t)k * L;
        for (int i = 0; i < L; ++i) w[i] = w0 ? w0[(size_t)k * L + i] : 0.0;
        for (int i = 0; i < 2 * P + 1; ++i) g[i] = 0.0;
        first = 0;
        t_last = 0;
        for (int n = 0; n < n_steps; ++n) {
            const int t = n / 2;
            t_last = t;
            /* A new pilot t arrives at n = 2t: drop the oldest entry if the dictionary is full;
             * entry t joins with both centres at zero coefficient. */
            if (n % 2 == 0 && t - first == D) first += 1;
            const int c_lo = 2 * first, c_hi = 2 * t + 2;   /* alive centres [c_lo, c_hi) */
            const int j0 = (n >= W - 1) ? n - W + 1 : 0;   /* J_n = [j0, n] */
            const int nJ = n - j0 + 1;
            /* All projections of this step are taken from the same f_n (Eq. apsm). */
            for (int j = j0; j <= n; ++j) {
                const double *xj = x + (size_t)j * L;
                const double y = eval_f(L, w, c_hi - c_lo, x + (size_t)c_lo * L, g + c_lo, 1, xj,
                                        p->sigma, p->w_L);
                if (j == n) {   /* the sample arrives: its target is given or decided now */
                    tgt[n] = (n >= decide_from) ? apsm_oracle_pam_slice(y, p->qam_bits, NULL)
                                                : sym[((size_t)(n / 2) * K + k) * 2 + (n % 2)];
                    if (pred_out) pred_out[((size_t)(n / 2) * K + k) * 2 + (n % 2)] = y;
                    if (target_out) target_out[((size_t)(n / 2) * K + k) * 2 + (n % 2)] = tgt[n];
                }
                const double bj = tgt[j];
                const double e = y - bj;
                const double kjj = p->w_L * kappa_lin(L, xj, xj) + w_G;   /* kappa(r_j, r_j) */
                int cs = (e < -p->eps) ? -1 : (e > p->eps ? 1 : 0);
                const int o = j - n + W - 1;
                const size_t li = ((size_t)n * W + o) * K + k;
                if (forced && (forced[li] == -1 || forced[li] == 0 || forced[li] == 1)) cs = forced[li];
                double b = 0.0;                                                    /* Eq. beta */
                if (kjj != 0.0) {
                    if (cs < 0) b = (bj - y - p->eps) / kjj;
                    else if (cs > 0) b = (bj - y + p->eps) / kjj;
                }
                beta[j - j0] = b;
                cs_win[j - j0] = cs;
                if (case_log) case_log[li] = (signed char)cs;
                if (margin_log) margin_log[li] = fabs(fabs(e) - p->eps);
            }
            /* weights q_j: uniform over J_n, or uniform over the violated slabs of J_n */
            double q = 1.0 / (double)nJ;
            if (p->weights == 1) {
                int nv = 0;
                for (int j = j0; j <= n; ++j) nv += (cs_win[j - j0] != 0);
                q = nv > 0 ? 1.0 / (double)nv : 0.0;
            }
            /* f_{n+1} = f_n + mu sum_j q_j beta_j kappa(x_j, .): coefficient of centre j and the
             * linear dictionary (Sec. II-D: kappa_L(x_j, .) = sum_m [x_j]_m kappa_L(e_m, .)).
             * (beta_j = 0 wherever q_j = 0 in the violated-slab weighting.) */
            for (int j = j0; j <= n; ++j) {
                const double a = p->mu * q * beta[j - j0];
                g[j] += a;
                const double *xj = x + (size_t)j * L;
                for (int i = 0; i < L; ++i) w[i] += a * xj[i];
            }
        }
        if (n_steps == 0) { first = 0; t_last = -1; }
        const int n_alive = t_last - first + 1;
        for (int i = 0; i < 2 * n_alive; ++i) gamma_out[(size_t)i * K + k] = g[2 * first + i];
    }
    if (k0 == 0 && alive_out) {
        if (k1 <= k0) {   /* no user trained: still report the dictionary bookkeeping */
            first = 0;
            t_last = (n_steps > 0) ? (n_steps - 1) / 2 : -1;
            for (int n = 0; n < n_steps; n += 2)
                if (n / 2 - first == D) first += 1;
        }
        alive_out[0] = first;
        alive_out[1] = (n_steps > 0) ? t_last - first + 1 : 0;
    }
    free(x);
    free(g);
    free(beta);
    free(tgt);
    free(cs_win);
    return 0;
}

/*
 * Gradient of a linear functional of the detection outputs (for the adjoint of detection):
 *   L = sum_{q,k} dy[q][k][0] f^k(r1(q)) + dy[q][k][1] f^k(r2(q)),
 *   f^k(x) = w_L <w_k, x> + w_G sum_i gamma_i^k kappa_G(c_i, x)      (Fact 1, Sec. II-D)
 * with the plain partial derivatives
 *   dL/dgamma_i^k = w_G sum_q sum_l dy[q][k][l] kappa_G(c_i, x_l(q))
 *   dL/dw_k       = w_L sum_q sum_l dy[q][k][l] x_l(q)
 *   dL/dsigma     = w_G sum_{q,k,l,i} dy[q][k][l] gamma_i^k kappa_G(c_i, x_l(q)) ||c_i - x_l(q)||^2 / sigma^3
 *   dL/dw_L       = sum_{q,k,l} dy[q][k][l] (<w_k, x_l(q)> - sum_i gamma_i^k kappa_G(c_i, x_l(q)))
 * where x_0(q) = r1(q), x_1(q) = r2(q).  Queries [q0, q1); results are ADDED to the outputs
 * (dgamma [n_c][K], dw [K][2M], dscal [2] = {dL/dsigma, dL/dw_L}).
 */
void apsm_oracle_detect_grad(const apsm_oracle_params *p, int n_c, const double *cent, const double *gamma,
                             const double *w, int q0, int q1, const double *rx, const double *dy, double *dgamma,
                             double *dw, double *dscal)
{
    const int M = p->M, L = 2 * M, K = p->K;
    const double w_G = 1.0 - p->w_L, s = p->sigma;
    double *x[2];
    x[0] = (double *)malloc(sizeof(double) * (size_t)L);
    x[1] = (double *)malloc(sizeof(double) * (size_t)L);
    for (int q = q0; q < q1; ++q) {
        real_split(M, rx + (size_t)q * 2 * M, x[0], x[1]);
        for (int l = 0; l < 2; ++l) {
            for (int i = 0; i < n_c; ++i) {
                const double *c = cent + (size_t)i * L;
                double d2 = 0.0;
                for (int j = 0; j < L; ++j) d2 += (c[j] - x[l][j]) * (c[j] - x[l][j]);
                const double kg = exp(-d2 / (2.0 * s * s));
                for (int k = 0; k < K; ++k) {
                    const double g = dy[((size_t)q * K + k) * 2 + l];
                    dgamma[(size_t)i * K + k] += w_G * g * kg;
                    dscal[0] += w_G * g * gamma[(size_t)i * K + k] * kg * d2 / (s * s * s);
                    dscal[1] -= g * gamma[(size_t)i * K + k] * kg;
                }
            }
            for (int k = 0; k < K; ++k) {
                const double g = dy[((size_t)q * K + k) * 2 + l];
                dscal[1] += g * kappa_lin(L, w + (size_t)k * L, x[l]);
                for (int j = 0; j < L; ++j) dw[(size_t)k * L + j] += p->w_L * g * x[l][j];
            }
        }
    }
    free(x[0]);
    free(x[1]);
}
