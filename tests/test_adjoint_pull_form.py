"""The training adjoint's O(W^2 + P) formulation, checked on the CPU in FP64 against the direct
form it replaces (plain numpy models of both; neither is the oracle nor the CUDA code).

Forward (Eq. apsm with Eq. beta over the window J_n, Sec. II-D): the direct form re-evaluates every
window sample against every live centre at every step; the carried form keeps the window's
predictions and updates them with the W projections of the step, subtracting a centre's frozen
contribution when its entry leaves, and forms a sample's prediction once on arrival.
Reverse: the direct (push) form adds every step's terms to the adjoint of every live centre; the
pull form sums R_j kappa(x_i, x_j) once, when centre i enters the window from below, with the R
of centres evicted during the run corrected by the value kept at their eviction step.
Both pairs must agree to rounding, with FIFO eviction and with 2D = W + 1 (the oldest centre of a
window leaves right after its last update)."""
import numpy as np
import pytest


def _samples(M, P, seed):
    rng = np.random.default_rng(seed)
    rx = (rng.standard_normal((P, M)) + 1j * rng.standard_normal((P, M))) / np.sqrt(2 * M)
    X = np.zeros((2 * P, 2 * M))
    for t in range(P):  # real split: x_2t = [Re r; Im r], x_2t+1 = [Im r; -Re r]
        X[2 * t] = np.concatenate([rx[t].real, rx[t].imag])
        X[2 * t + 1] = np.concatenate([rx[t].imag, -rx[t].real])
    b = rng.choice([-1.0, 1.0], size=2 * P) / np.sqrt(2)
    return X, b


def _tables(X, sigma):
    L = X @ X.T
    n = np.diag(L)
    d2 = np.maximum(n[:, None] + n[None, :] - 2 * L, 0)
    return L, np.exp(-d2 / (2 * sigma ** 2)), d2


def _beta(e, eps, kap):
    if e < -eps:
        return 1.0, (-e - eps) / kap
    if e > eps:
        return -1.0, (-e + eps) / kap
    return 0.0, 0.0


def _first_centre(n, D):
    return 2 * max(0, n // 2 - D + 1)


def forward_direct(X, b, W, D, sig, mu, eps, wL, w0):
    S = X.shape[0]
    L, G, d2 = _tables(X, sig)
    gam, w, tape = np.zeros(S), w0.copy(), []
    for n in range(S):
        jlo = max(0, n - W + 1)
        lo = _first_centre(n, D)
        rec = []
        for j in range(jlo, n + 1):
            dw = w @ X[j]
            gs = gam[lo:n + 1] @ G[j, lo:n + 1]
            gd = (gam[lo:n + 1] * G[j, lo:n + 1]) @ d2[j, lo:n + 1]
            kap = wL * L[j, j] + (1 - wL)
            s, beta = _beta(wL * dw + (1 - wL) * gs - b[j], eps, kap)
            rec.append((beta, s, kap, dw, gs, gd))
        tape.append(rec)
        for o, j in enumerate(range(jlo, n + 1)):
            a = mu / len(rec) * rec[o][0]
            gam[j] += a
            w += a * X[j]
    return gam, w, tape


def forward_carried(X, b, W, D, sig, mu, eps, wL, w0):
    S = X.shape[0]
    L, G, d2 = _tables(X, sig)
    gam, w, tape = np.zeros(S), w0.copy(), []
    pred = {0: (0.0, 0.0, w @ X[0])}  # sample -> (gauss, its sigma weight, <w, x>)
    for n in range(S):
        jlo, jn = max(0, n - W + 1), n + 1
        nJ = n - jlo + 1
        if jn < S:  # the arrival's sums from the state before this step
            lo = _first_centre(jn, D)
            arr = (gam[lo:jn] @ G[jn, lo:jn], (gam[lo:jn] * G[jn, lo:jn]) @ d2[jn, lo:jn], w @ X[jn])
        rec, ca = [], []
        for j in range(jlo, n + 1):
            gs, gd, dw = pred[j]
            kap = wL * L[j, j] + (1 - wL)
            s, beta = _beta(wL * dw + (1 - wL) * gs - b[j], eps, kap)
            rec.append((beta, s, kap, dw, gs, gd))
            ca.append(mu / nJ * beta)
        tape.append(rec)
        gnew = [gam[j] + ca[o] for o, j in enumerate(range(jlo, n + 1))]
        if jn < S:
            e_lo, e_hi = _first_centre(n, D), _first_centre(jn, D)
            for j in range(max(0, n - W + 2), jn + 1):
                y, d, x = arr if j == jn else pred[j]
                for o, i in enumerate(range(jlo, n + 1)):
                    x += ca[o] * L[j, i]
                    if j == jn and i < e_hi:
                        continue  # left before the arrival
                    y += ca[o] * G[j, i]
                    d += ca[o] * G[j, i] * d2[j, i]
                if j != jn:
                    for i in range(e_lo, e_hi):
                        gi = gnew[i - jlo] if i >= jlo else gam[i]
                        y -= gi * G[j, i]
                        d -= gi * G[j, i] * d2[j, i]
                pred[j] = (y, d, x)
        for o, j in enumerate(range(jlo, n + 1)):
            gam[j] = gnew[o]
            w += ca[o] * X[j]
    return gam, w, tape


def _scalar_terms(tp, ab, q, mu, wL, sig, nrm_j):
    beta, s, kap, dw, gs, gd = tp
    out = np.array([0.0, q * beta * ab, 0.0, 0.0])  # sigma, mu, eps, w_L
    cw = cg = 0.0
    if s != 0:
        yb = -mu * q * ab / kap
        out += [yb * (1 - wL) * gd / sig ** 3, 0.0, s * yb, yb * beta * (nrm_j - 1) + yb * (dw - gs)]
        cw, cg = yb * wL, yb * (1 - wL)
    return out, cw, cg


def reverse_push(X, W, D, sig, mu, wL, tape, gfin, wfin):
    S = X.shape[0]
    L, G, _ = _tables(X, sig)
    gbar, wbar, sc = gfin.copy(), wfin.copy(), np.zeros(4)
    for n in range(S - 1, -1, -1):
        jlo = max(0, n - W + 1)
        q = 1.0 / (n - jlo + 1)
        ab = [gbar[j] + wbar @ X[j] for j in range(jlo, n + 1)]
        terms = []
        for o, j in enumerate(range(jlo, n + 1)):
            t, cw, cg = _scalar_terms(tape[n][o], ab[o], q, mu, wL, sig, L[j, j])
            sc += t
            terms.append((j, cw, cg))
        lo = _first_centre(n, D)
        for j, cw, cg in terms:
            wbar += cw * X[j]
            gbar[lo:n + 1] += cg * G[j, lo:n + 1]
    return sc, wbar


def reverse_pull(X, W, D, sig, mu, wL, tape, gfin, wfin):
    S = X.shape[0]
    L, G, _ = _tables(X, sig)
    evict = lambda i: 2 * (i // 2 + D)  # noqa: E731 -- centre i takes part in steps n < evict(i)
    R, wbar, sc, ab, snap = np.zeros(S), wfin.copy(), np.zeros(4), {}, {}
    for j in range(max(0, S - W), S):
        ab[j] = wbar @ X[j] + gfin[j]
    for n in range(S - 1, -1, -1):
        jlo, je = max(0, n - W + 1), n - W
        q = 1.0 / (n - jlo + 1)
        if (n + 1) % 2 == 0 and n + 1 <= S - 1 and (n + 1) // 2 >= D:
            snap[n + 1] = R[n + 1 - W + 1:n + 1].copy()  # R after the steps >= n + 1
        if je >= 0:  # the entrant's pull, from the steps after n in which it is alive
            e = evict(je)
            gs = 0.0
            if e > n + 1:
                s_lo = e - W + 1 if e <= S - 1 else S
                for i in range(je + 2, min(e, S)):
                    gs += (R[i] - snap[e][i - s_lo] if i >= s_lo else R[i]) * G[je, i]
            ls = wbar @ X[je]
        terms = []
        for o, j in enumerate(range(jlo, n + 1)):
            t, cw, cg = _scalar_terms(tape[n][o], ab[j], q, mu, wL, sig, L[j, j])
            sc += t
            terms.append((j, cw, cg))
        for j, cw, cg in terms:
            R[j] += cg
            wbar += cw * X[j]
        for j in range(max(0, n - W), n):  # the adjoints of J_{n-1}
            alive = True
            if j == je:
                acc = gfin[j] + gs + ls
                alive = n < evict(j)
            else:
                acc = ab[j]
            for i, cw, cg in terms:
                acc += cw * L[j, i] + (cg * G[j, i] if alive else 0.0)
            ab[j] = acc
    return sc, wbar


CASES = [  # M, P, W, D, seed
    (4, 20, 4, 20, 1),   # no eviction
    (4, 35, 6, 6, 2),    # FIFO eviction
    (3, 30, 5, 3, 3),    # 2D = W + 1
    (4, 40, 1, 2, 4),    # single-slot window
    (2, 25, 7, 4, 5),    # 2D = W + 1, longer window
    (3, 40, 9, 5, 7),    # 2D = W + 1 with eviction throughout
    (2, 3, 5, 3, 8),     # window longer than the run
]


@pytest.mark.parametrize("M,P,W,D,seed", CASES)
def test_carried_forward_and_pull_reverse_equal_direct_forms(M, P, W, D, seed):
    X, b = _samples(M, P, seed)
    sig, mu, eps, wL = 0.7, 0.6, 0.05, 0.4
    rng = np.random.default_rng(seed + 100)
    w0 = 0.2 * rng.standard_normal(2 * M)
    g1, w1, t1 = forward_direct(X, b, W, D, sig, mu, eps, wL, w0)
    g2, w2, t2 = forward_carried(X, b, W, D, sig, mu, eps, wL, w0)
    assert np.abs(g1 - g2).max() < 1e-12 and np.abs(w1 - w2).max() < 1e-12
    assert all(r1[o][1] == r2[o][1] for r1, r2 in zip(t1, t2) for o in range(len(r1)))  # same branches
    S = 2 * P
    alive = np.array([1.0 if j // 2 >= max(0, P - D) else 0.0 for j in range(S)])
    gfin, wfin = rng.standard_normal(S) * alive, rng.standard_normal(2 * M)
    s1, wb1 = reverse_push(X, W, D, sig, mu, wL, t1, gfin, wfin)
    s2, wb2 = reverse_pull(X, W, D, sig, mu, wL, t1, gfin, wfin)
    assert np.abs(s1 - s2).max() <= 1e-12 * max(1.0, np.abs(s1).max())
    assert np.abs(wb1 - wb2).max() <= 1e-12 * max(1.0, np.abs(wb1).max())


def test_dropping_the_eviction_terms_is_detected():
    """The check has teeth: a pull form that ignores eviction disagrees when entries leave."""
    M, P, W, D, seed = 4, 35, 6, 6, 2
    X, b = _samples(M, P, seed)
    sig, mu, eps, wL = 0.7, 0.6, 0.05, 0.4
    w0 = np.zeros(2 * M)
    _, _, t1 = forward_direct(X, b, W, D, sig, mu, eps, wL, w0)
    S = 2 * P
    rng = np.random.default_rng(1)
    alive = np.array([1.0 if j // 2 >= max(0, P - D) else 0.0 for j in range(S)])
    gfin, wfin = rng.standard_normal(S) * alive, rng.standard_normal(2 * M)
    s1, _ = reverse_push(X, W, D, sig, mu, wL, t1, gfin, wfin)
    s_no_evict, _ = reverse_pull(X, W, 10 ** 6, sig, mu, wL, t1, gfin, wfin)  # as if nothing left
    assert np.abs(s1 - s_no_evict).max() > 1e-6 * max(1.0, np.abs(s1).max())
