"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks a property that a plausible slip in the oracle (a dropped term, a wrong
sign or index, a swapped real-split half, a wrong weight) would break:

  * a single unit-step projection lands the sample on its hyperslab boundary (Eq. beta);
  * the hyperslab projection moves f by exactly its distance to the set (metric projection);
  * the reproducing property of the weighted sum space (Fact 1, Eq. sum_inner_product);
  * the linear dictionary equals the Euclidean span of the projected samples (Sec. II-D);
  * Fejer monotonicity of the concurrent relaxed projections on a realisable problem (Eq. apsm);
  * each projection of one concurrent step is taken from the same f_n (Eq. apsm);
  * the linear-only case reduces to textbook NLMS;
  * the real split gives g(r) = c^H r for the linear part (Sec. II-D);
  * a hand-computed detection value (tests/golden/p9_detect_hand.txt);
  * noiseless single-user training detects without error;
  * FIFO eviction keeps the last D entries and the linear part (tiny-width kernel).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2201_05024_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def split(r):
    """Test-side real split of Sec. II-D (independent of the oracle's)."""
    r = np.asarray(r, dtype=np.complex128)
    return np.concatenate([r.real, r.imag]), np.concatenate([r.imag, -r.real])


def samples(rx, sym):
    """x_n, b_n^k for n = 2t + l (Sec. II-D), built by the test."""
    xs, bs = [], []
    for t in range(rx.shape[0]):
        x1, x2 = split(rx[t])
        xs += [x1, x2]
        bs += [np.asarray(sym[t]).real.astype(np.float64), np.asarray(sym[t]).imag.astype(np.float64)]
    return np.array(xs), np.array(bs)


def kappa_state(M, K, x, beta):
    """The element beta * kappa(x, .) of H for every user: centre x with coefficient beta, linear part beta*x."""
    return oracle.State(centres=x[None, :].copy(), gamma=np.full((1, K), float(beta)),
                        w=np.tile(beta * x, (K, 1)))


def add(a, b):
    return oracle.State(centres=np.concatenate([a.centres, b.centres]),
                        gamma=np.concatenate([a.gamma, b.gamma]), w=a.w + b.w)


@pytest.mark.parametrize("w_L", [0.5, 0.2, 0.9])
def test_p1_unit_step_lands_on_slab_boundary(w_L):
    inst = synth.make_instance(3, 2, 8, 0, 5.0, instance=11)
    p = oracle.Params(M=3, K=2, W=1, D=8, sigma=0.7, mu=1.0, eps=0.05, w_L=w_L)
    xs, bs = samples(inst.rx_pilot, inst.sym_pilot)
    moved = 0
    for n in range(2 * 8):
        f_n = oracle.train(p, inst.rx_pilot, inst.sym_pilot, n_steps=n)
        f_n1 = oracle.train(p, inst.rx_pilot, inst.sym_pilot, n_steps=n + 1)
        y0 = oracle.eval_real(p, f_n, xs[n][None])[0] if f_n.centres.shape[0] else \
            w_L * (f_n.w @ xs[n])
        y1 = oracle.eval_real(p, f_n1, xs[n][None])[0]
        for k in range(2):
            e = y0[k] - bs[n][k]
            if abs(e) <= p.eps:
                assert y1[k] == pytest.approx(y0[k], abs=1e-13)
            else:
                moved += 1
                assert y1[k] == pytest.approx(bs[n][k] + math.copysign(p.eps, e), abs=1e-12)
    assert moved > 10


def test_p2_projection_moves_by_distance_to_slab():
    inst = synth.make_instance(2, 1, 6, 0, 5.0, instance=12)
    p = oracle.Params(M=2, K=1, W=1, D=6, sigma=0.6, mu=1.0, eps=0.02, w_L=0.4)
    xs, bs = samples(inst.rx_pilot, inst.sym_pilot)
    for n in range(1, 12):
        f_n = oracle.train(p, inst.rx_pilot, inst.sym_pilot, n_steps=n)
        f_n1 = oracle.train(p, inst.rx_pilot, inst.sym_pilot, n_steps=n + 1)
        e = oracle.eval_real(p, f_n, xs[n][None])[0, 0] - bs[n][0]
        kjj = p.w_L * xs[n] @ xs[n] + (1 - p.w_L)
        d = oracle.rkhs_diff(f_n1, f_n)
        dist = math.sqrt(max(oracle.rkhs_inner(p, d, d), 0.0))
        assert dist == pytest.approx(max(abs(e) - p.eps, 0.0) / math.sqrt(kjj), rel=1e-9, abs=1e-12)


def test_p3_reproducing_property():
    inst = synth.make_instance(3, 2, 10, 4, 10.0, instance=13)
    p = oracle.Params(M=3, K=2, W=4, D=10, sigma=0.8, mu=0.7, eps=0.01, w_L=0.3)
    f = oracle.train(p, inst.rx_pilot, inst.sym_pilot)
    for r in inst.rx_data:
        for u in split(r):
            ku = kappa_state(3, 2, u, 1.0)
            y = oracle.eval_real(p, f, u[None])[0]
            for k in range(2):
                assert oracle.rkhs_inner(p, f, ku, k) == pytest.approx(y[k], rel=1e-12, abs=1e-13)


def test_p4_linear_dictionary_is_span_of_projected_samples():
    inst = synth.make_instance(4, 3, 12, 0, 10.0, instance=14)
    p = oracle.Params(M=4, K=3, W=5, D=12, sigma=0.5, mu=0.5, eps=0.01, w_L=0.5)
    f = oracle.train(p, inst.rx_pilot, inst.sym_pilot)
    xs, _ = samples(inst.rx_pilot, inst.sym_pilot)
    assert f.n_entries == 12
    np.testing.assert_allclose(f.centres, xs, rtol=0, atol=1e-7)
    np.testing.assert_allclose(f.w, (xs.T @ f.gamma).T, rtol=1e-12, atol=1e-14)
    # two forms of the squared norm: gamma^T (w_L X X^T + w_G K_G) gamma == w_L |w|^2 + w_G gamma^T K_G gamma
    KG = oracle.gram_gauss(xs, xs, p.sigma)
    for k in range(3):
        g = f.gamma[:, k]
        lhs = g @ (p.w_L * xs @ xs.T + (1 - p.w_L) * KG) @ g
        assert lhs == pytest.approx(oracle.rkhs_inner(p, f, f, k), rel=1e-11)


@pytest.mark.parametrize("mu,W", [(1.0, 1), (0.5, 4), (1.9, 4), (1.0, 3)])
def test_p5_fejer_monotone_on_realisable_problem(mu, W):
    M, K, P = 2, 2, 7
    rng = np.random.default_rng(5)
    inst = synth.make_instance(M, K, P, 0, 10.0, instance=15)
    p = oracle.Params(M=M, K=K, W=W, D=P, sigma=0.6, mu=mu, eps=0.05, w_L=0.5)
    # f* with its own centres and linear part; targets within eps of f* so f* lies in every C_n.
    star = oracle.State(centres=rng.standard_normal((5, 2 * M)) * 0.5,
                        gamma=rng.standard_normal((5, K)), w=rng.standard_normal((K, 2 * M)))
    xs, _ = samples(inst.rx_pilot, inst.sym_pilot)
    fx = oracle.eval_real(p, star, xs)
    b = fx + rng.uniform(-p.eps, p.eps, size=fx.shape) * 0.999
    sym = b[0::2] + 1j * b[1::2]
    prev = None
    for n in range(2 * P + 1):
        f_n = oracle.train(p, inst.rx_pilot, sym, n_steps=n)
        d = oracle.rkhs_diff(f_n, star)
        dist = [oracle.rkhs_inner(p, d, d, k) for k in range(K)]
        if prev is not None:
            for k in range(K):
                assert dist[k] <= prev[k] * (1 + 1e-12) + 1e-14
        prev = dist
    assert prev[0] < oracle.rkhs_inner(p, star, star, 0)


def test_concurrent_projections_share_f_n():
    """Every projection of a step, applied alone to f_n, lands x_j on its slab boundary; its
    coefficient is the oracle's coefficient change / (mu q)."""
    M, K, P, W = 3, 2, 9, 5
    inst = synth.make_instance(M, K, P, 0, 3.0, instance=16)
    p = oracle.Params(M=M, K=K, W=W, D=P, sigma=0.6, mu=0.8, eps=0.03, w_L=0.6)
    xs, bs = samples(inst.rx_pilot, inst.sym_pilot)
    checked = 0
    for n in range(2, 2 * P):
        f_n = oracle.train(p, inst.rx_pilot, inst.sym_pilot, n_steps=n)
        f_n1 = oracle.train(p, inst.rx_pilot, inst.sym_pilot, n_steps=n + 1)
        J = list(range(max(0, n - W + 1), n + 1))
        q = 1.0 / len(J)
        g_n = np.zeros((2 * P, K))
        g_n[:f_n.gamma.shape[0]] = f_n.gamma
        g_n1 = np.zeros((2 * P, K))
        g_n1[:f_n1.gamma.shape[0]] = f_n1.gamma
        dg = g_n1 - g_n
        assert np.all(dg[[i for i in range(2 * P) if i not in J]] == 0)
        y = oracle.eval_real(p, f_n, xs[J])
        for a, j in enumerate(J):
            for k in range(K):
                beta = dg[j, k] / (p.mu * q)
                e = y[a, k] - bs[j][k]
                if abs(e) <= p.eps:
                    assert beta == 0.0
                    continue
                proj = add(f_n, kappa_state(M, K, xs[j], beta))
                assert oracle.eval_real(p, proj, xs[j][None])[0, k] == pytest.approx(
                    bs[j][k] + math.copysign(p.eps, e), abs=1e-11)
                checked += 1
    assert checked > 50


@pytest.mark.parametrize("mu", [1.0, 0.3])
def test_p6_linear_only_is_textbook_nlms(mu):
    inst = synth.make_instance(4, 2, 15, 0, 10.0, instance=17)
    p = oracle.Params(M=4, K=2, W=1, D=15, sigma=0.5, mu=mu, eps=0.0, w_L=1.0)
    xs, bs = samples(inst.rx_pilot, inst.sym_pilot)
    w = np.zeros((2, 8))
    for n in range(30):
        for k in range(2):
            w[k] += mu * (bs[n][k] - w[k] @ xs[n]) * xs[n] / (xs[n] @ xs[n])
        f = oracle.train(p, inst.rx_pilot, inst.sym_pilot, n_steps=n + 1)
        np.testing.assert_allclose(f.w, w, rtol=1e-11, atol=1e-13)


def test_p7_real_split_linear_part_is_complex_inner_product():
    M, K = 5, 3
    inst = synth.make_instance(M, K, 20, 50, 10.0, instance=18)
    p = oracle.Params(M=M, K=K, W=6, D=20, sigma=0.5, mu=0.5, eps=0.01, w_L=1.0)
    f = oracle.train(p, inst.rx_pilot, inst.sym_pilot)
    y = oracle.detect(p, f, inst.rx_data)
    c = oracle.clin_from_w(M, f.w)                          # [M][K]
    ref = inst.rx_data.astype(np.complex128) @ np.conj(c)  # c_k^H r
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split(None, 1)
                vals[k] = v
    return vals


def test_p9_hand_computed_detect_value():
    g = _golden("p9_detect_hand.txt")
    f = float
    p = oracle.Params(M=1, K=1, W=1, D=1, sigma=f(g["sigma"]), w_L=f(g["w_L"]))
    st = oracle.state_from_arrays(1, np.array([[f(g["entry_re"]) + 1j * f(g["entry_im"])]]),
                                  np.array([[[f(g["gamma1"])], [f(g["gamma2"])]]]),
                                  np.array([[f(g["c_re"]) + 1j * f(g["c_im"])]]))
    y = oracle.detect(p, st, np.array([[f(g["query_re"]) + 1j * f(g["query_im"])]]))[0, 0]
    env = {"exp": math.exp}
    assert y.real == pytest.approx(eval(g["y1"], env), abs=1e-15)
    assert y.imag == pytest.approx(eval(g["y2"], env), abs=1e-15)


def test_p10_noiseless_single_user_linear_training_detects_perfectly():
    inst = synth.make_instance(4, 1, 40, 500, 0.0, instance=19, noiseless=True, pa_coef=0.0)
    p = oracle.Params(M=4, K=1, W=1, D=40, sigma=0.5, mu=1.0, eps=0.0, w_L=1.0)
    f = oracle.train(p, inst.rx_pilot, inst.sym_pilot)
    y = oracle.detect(p, f, inst.rx_data)
    assert np.all(oracle.hard_qpsk(y) == inst.idx_data)
    np.testing.assert_allclose(y, inst.sym_data, atol=1e-6)


def test_fifo_eviction_keeps_last_entries_and_linear_part():
    M, K, P = 3, 2, 14
    inst = synth.make_instance(M, K, P, 0, 10.0, instance=20)
    big = oracle.Params(M=M, K=K, W=4, D=P, sigma=1e-3, mu=0.6, eps=0.01, w_L=0.5)
    small = oracle.Params(M=M, K=K, W=4, D=5, sigma=1e-3, mu=0.6, eps=0.01, w_L=0.5)
    fb = oracle.train(big, inst.rx_pilot, inst.sym_pilot)
    fs = oracle.train(small, inst.rx_pilot, inst.sym_pilot)
    assert (fs.first_entry, fs.n_entries) == (P - 5, 5)
    np.testing.assert_array_equal(fs.w, fb.w)
    np.testing.assert_array_equal(fs.gamma, fb.gamma[2 * (P - 5):])
    xs, _ = samples(inst.rx_pilot, inst.sym_pilot)
    np.testing.assert_allclose(fs.centres, xs[2 * (P - 5):], atol=1e-7)


def test_eviction_changes_predictions_at_normal_width():
    """With an overlapping kernel, dropping entries changes the trained filter (the Gaussian
    part of evicted entries is really removed)."""
    M, K, P = 3, 1, 14
    inst = synth.make_instance(M, K, P, 0, 10.0, instance=21)
    fb = oracle.train(oracle.Params(M=M, K=K, W=4, D=P, sigma=0.6), inst.rx_pilot, inst.sym_pilot)
    fs = oracle.train(oracle.Params(M=M, K=K, W=4, D=5, sigma=0.6), inst.rx_pilot, inst.sym_pilot)
    assert np.max(np.abs(fs.w - fb.w)) > 1e-6


def test_complex_gram_distances_match_direct_differences():
    """||r1(t) - r1(s)||^2 = n_t + n_s - 2 Re z, ||r1(t) - r2(s)||^2 = n_t + n_s - 2 Im z,
    ||r2(t) - r1(s)||^2 = n_t + n_s + 2 Im z with z = r_t^H r_s; J-rotation preserves distances."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        M = int(rng.integers(1, 9))
        a = rng.standard_normal(M) + 1j * rng.standard_normal(M)
        b = rng.standard_normal(M) + 1j * rng.standard_normal(M)
        a1, a2 = split(a)
        b1, b2 = split(b)
        z = np.vdot(a, b)
        nn = np.vdot(a, a).real + np.vdot(b, b).real
        assert np.sum((a1 - b1) ** 2) == pytest.approx(nn - 2 * z.real)
        assert np.sum((a2 - b2) ** 2) == pytest.approx(nn - 2 * z.real)
        assert np.sum((a1 - b2) ** 2) == pytest.approx(nn - 2 * z.imag)
        assert np.sum((a2 - b1) ** 2) == pytest.approx(nn + 2 * z.imag)
        assert a1 @ b1 == pytest.approx(z.real) and a1 @ b2 == pytest.approx(z.imag)
        assert a2 @ b1 == pytest.approx(-z.imag)


def test_case_log_and_forced_replay():
    inst = synth.make_instance(4, 2, 30, 0, 5.0, instance=22)
    p = oracle.Params(M=4, K=2, W=6, D=30, sigma=0.5)
    st, cl, ml = oracle.train(p, inst.rx_pilot, inst.sym_pilot, log_cases=True)
    assert set(np.unique(cl[cl != 127])) <= {-1, 0, 1}
    assert cl[0, :5].tolist() == [[127, 127]] * 5         # slots before sample 0 are untouched
    st2 = oracle.train(p, inst.rx_pilot, inst.sym_pilot, forced=np.where(cl == 127, 2, cl))
    np.testing.assert_array_equal(st2.gamma, st.gamma)
    # forcing one outside case to 'inside' changes the trajectory
    n, o, k = np.argwhere(cl == 1)[3]
    fo = np.full_like(cl, 2)
    fo[n, o, k] = 0
    st3 = oracle.train(p, inst.rx_pilot, inst.sym_pilot, forced=fo)
    assert np.max(np.abs(st3.gamma - st.gamma)) > 0


@pytest.mark.slow
def test_paper_default_parameters_detect_qpsk_cleanly():
    """Sec. V defaults (tests/golden/paper_defaults.txt) on a synthetic 16x6 QPSK uplink: the
    paper reports a negligible QPSK error rate over the air; here a loose sanity bound."""
    g = {k: float(v) for k, v in _golden("paper_defaults.txt").items()}
    M, K = int(g["M"]), int(g["K"])
    inst = synth.make_instance(M, K, int(g["P"]), 800, 20.0, instance=23)
    p = oracle.Params(M=M, K=K, W=int(g["W"]), D=int(g["P"]), sigma=math.sqrt(g["sigma2"]), mu=0.5,
                      eps=0.01, w_L=g["w_L"])
    f = oracle.train(p, inst.rx_pilot, inst.sym_pilot)
    y = oracle.detect(p, f, inst.rx_data)
    assert np.mean(oracle.hard_qpsk(y) != inst.idx_data) < 0.01


def _loss(p, st, rx, G):
    """L = sum Re(conj(G) soft) for the oracle's detection."""
    return float(np.sum((np.conj(G) * oracle.detect(p, st, rx)).real))


def test_detect_gradient_matches_finite_differences():
    """The oracle's detection gradient (plain partial derivatives) against FP64 finite differences
    of the oracle's own detection: exact (any step) for the coefficients, in which the output is
    linear, and central differences for sigma and w_L."""
    M, K, n = 3, 2, 5
    rng = np.random.default_rng(8)
    ent = (rng.standard_normal((n, M)) + 1j * rng.standard_normal((n, M))) * 0.4
    gam = rng.standard_normal((n, 2, K))
    clin = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    rx = (rng.standard_normal((7, M)) + 1j * rng.standard_normal((7, M))) * 0.4
    G = rng.standard_normal((7, K)) + 1j * rng.standard_normal((7, K))
    p = oracle.Params(M=M, K=K, W=1, D=n, sigma=0.6, w_L=0.35)
    st = oracle.state_from_arrays(M, ent, gam, clin)
    dg, dw, dsig, dwl = oracle.detect_grad(p, st, rx, G)
    base = _loss(p, st, rx, G)
    for i in range(2 * n):
        for k in range(K):
            s2 = oracle.State(centres=st.centres, gamma=st.gamma.copy(), w=st.w)
            s2.gamma[i, k] += 1.0
            assert _loss(p, s2, rx, G) - base == pytest.approx(dg[i, k], rel=1e-10, abs=1e-12)
    for k in range(K):
        for j in range(2 * M):
            s2 = oracle.State(centres=st.centres, gamma=st.gamma, w=st.w.copy())
            s2.w[k, j] += 1.0
            assert _loss(p, s2, rx, G) - base == pytest.approx(dw[k, j], rel=1e-10, abs=1e-12)
    h = 1e-6
    ps = [oracle.Params(M=M, K=K, W=1, D=n, sigma=0.6 + e, w_L=0.35) for e in (h, -h)]
    fd = (_loss(ps[0], st, rx, G) - _loss(ps[1], st, rx, G)) / (2 * h)
    assert dsig == pytest.approx(fd, rel=1e-6)
    ps = [oracle.Params(M=M, K=K, W=1, D=n, sigma=0.6, w_L=0.35 + e) for e in (h, -h)]
    fd = (_loss(ps[0], st, rx, G) - _loss(ps[1], st, rx, G)) / (2 * h)
    assert dwl == pytest.approx(fd, rel=1e-6)
