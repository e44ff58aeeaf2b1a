"""Pins of the oracle's extensions (no GPU): Gray square QAM decisions, the violated-slab
weighting of the concurrent projections, decision-directed targets (tracking), and the linear
(LS channel estimate + MMSE / ZF) start of the filter.

Each test checks a fact fixed by the mathematics rather than re-typing the oracle:

  * the slicer returns the nearest constellation point (brute force over all points), the
    constellations have unit mean energy, and neighbouring points differ in one label bit;
  * with the violated-slab weights (q_j = 1/|V_n| on V_n) a single violated slab in the window
    takes the whole unit step and lands on its boundary (Eq. beta), the weighting reduces to the
    uniform one for W = 1, and the relaxed steps stay Fejer monotone on a realisable problem;
  * a decision-directed run whose decisions are all correct is, bit for bit, the run on the
    true symbols; the output recorded at a vector's arrival is f_n(x_n) evaluated afresh;
  * the ZF filter from a noiseless LS channel estimate recovers the data symbols exactly, the
    MMSE filter equals the textbook (H H^H + N0 I)^-1 H form, and it tends to ZF as N0 -> 0.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2201_05024_gb300 import synth

from test_oracle_pins import add, kappa_state, samples


# ------------------------------------------------------------------------------------------
# Gray square QAM
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("bits", [2, 4, 6])
def test_qam_slicer_is_nearest_point_and_gray(bits):
    pts = synth.qam_symbols(np.arange(1 << bits), bits)
    assert np.mean(np.abs(pts) ** 2) == pytest.approx(1.0, rel=1e-12)
    rng = np.random.default_rng(bits)
    y = (rng.standard_normal(4000) + 1j * rng.standard_normal(4000)) * 0.9
    near = np.argmin(np.abs(y[:, None] - pts[None, :]), axis=1)     # brute force
    assert np.array_equal(oracle.hard_qam(y, bits), near.astype(np.uint8))
    # the C slicer of one axis returns the nearest level value
    L = 1 << (bits // 2)
    levels = np.unique(np.round(pts.real, 12))
    assert len(levels) == L
    for v in rng.standard_normal(200):
        got, lev = oracle.pam_slice(float(v), bits)
        assert got == pytest.approx(levels[np.argmin(np.abs(levels - v))], abs=1e-9)
        assert got == pytest.approx(levels[lev], abs=1e-9)
    # Gray: points one level apart on one axis differ in exactly one label bit
    a = oracle.pam_scale(bits)
    for i in range(1 << bits):
        for j in range(1 << bits):
            d = pts[i] - pts[j]
            if abs(abs(d) - 2 * a) < 1e-9 and (abs(d.real) < 1e-9 or abs(d.imag) < 1e-9):
                assert bin(i ^ j).count("1") == 1


def test_qpsk_labels_unchanged():
    """QPSK keeps its convention: bit 0 = (Re < 0), bit 1 = (Im < 0), zero counts as non-negative."""
    s = np.array([1 + 1j, -1 + 1j, 1 - 1j, -1 - 1j, 0 + 0j, -0.0 - 1e-30j])
    assert oracle.hard_qam(s, 2).tolist() == [0, 1, 2, 3, 0, 2]


# ------------------------------------------------------------------------------------------
# violated-slab weights q_j = 1/|V_n|
# ------------------------------------------------------------------------------------------

def test_violated_weights_single_violation_takes_the_full_step():
    """W = 2, mu = 1, f_0 = 0: sample 0 has target 0, so it lies strictly inside its slab and is
    never updated; at step n = 1 only sample 1 is violated, and with q = 1/|V_n| = 1 it lands
    exactly on its boundary (Eq. beta), while the uniform q = 1/2 moves it only half way."""
    M, K = 3, 2
    inst = synth.make_instance(M, K, 4, 0, 5.0, instance=21)
    sym = inst.sym_pilot.astype(np.complex128)
    sym[0] = 1j * sym[0].imag                     # b_0 = Re s(0) = 0, b_1 = Im s(0) = +-1/sqrt(2)
    xs, bs = samples(inst.rx_pilot, sym)
    for weights, lands in ((1, True), (0, False)):
        p = oracle.Params(M=M, K=K, W=2, D=4, sigma=0.7, mu=1.0, eps=0.05, w_L=0.5, weights=weights)
        f2 = oracle.train(p, inst.rx_pilot, sym, n_steps=2)
        y1 = oracle.eval_real(p, f2, xs[1][None])[0]
        for k in range(K):
            assert abs(bs[1][k]) > p.eps                                  # sample 1 violated by f_1 = 0
            target = bs[1][k] - math.copysign(p.eps, bs[1][k])            # e = -b_1: nearest edge
            if lands:
                assert y1[k] == pytest.approx(target, abs=1e-12)
            else:
                assert y1[k] == pytest.approx(0.5 * target, abs=1e-12)


def test_violated_weights_equal_uniform_for_window_one():
    inst = synth.make_instance(4, 3, 30, 0, 10.0, instance=22)
    base = dict(M=4, K=3, W=1, D=20, sigma=0.5, mu=0.7, eps=0.02, w_L=0.5)
    a = oracle.train(oracle.Params(**base, weights=0), inst.rx_pilot, inst.sym_pilot)
    b = oracle.train(oracle.Params(**base, weights=1), inst.rx_pilot, inst.sym_pilot)
    assert np.array_equal(a.gamma, b.gamma) and np.array_equal(a.w, b.w)


@pytest.mark.parametrize("mu,W", [(1.0, 4), (1.9, 3), (0.5, 5)])
def test_violated_weights_fejer_monotone(mu, W):
    """q_j = 1/|V_n| on V_n is a convex weighting of the relaxed projections onto the violated
    slabs, so the distance to any f* inside every slab never grows (APSM theory)."""
    M, K, P = 2, 2, 7
    rng = np.random.default_rng(6)
    inst = synth.make_instance(M, K, P, 0, 10.0, instance=23)
    p = oracle.Params(M=M, K=K, W=W, D=P, sigma=0.6, mu=mu, eps=0.05, w_L=0.5, weights=1)
    star = oracle.State(centres=rng.standard_normal((5, 2 * M)) * 0.5,
                        gamma=rng.standard_normal((5, K)), w=rng.standard_normal((K, 2 * M)))
    xs, _ = samples(inst.rx_pilot, inst.sym_pilot)
    fx = oracle.eval_real(p, star, xs)
    b = fx + rng.uniform(-p.eps, p.eps, size=fx.shape) * 0.999
    sym = b[0::2] + 1j * b[1::2]
    prev = None
    for n in range(2 * P + 1):
        d = oracle.rkhs_diff(oracle.train(p, inst.rx_pilot, sym, n_steps=n), star)
        dist = [oracle.rkhs_inner(p, d, d, k) for k in range(K)]
        if prev is not None:
            for k in range(K):
                assert dist[k] <= prev[k] * (1 + 1e-12) + 1e-14
        prev = dist


# ------------------------------------------------------------------------------------------
# decision-directed targets
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("bits", [2, 4])
def test_correct_decisions_reproduce_training_on_true_symbols(bits):
    """Pilots, then data vectors in decision-directed mode at high SNR: every decision is the
    transmitted symbol, so the run equals the run with the true symbols given (bit for bit;
    the symbols are passed in FP64, as the slicer's own levels)."""
    M, K, P, N = 8, 2, 120, 60
    inst = synth.make_instance(M, K, P, N, 40.0, instance=24, bits=bits)
    p = oracle.Params(M=M, K=K, W=6, D=200, sigma=0.6, mu=0.7, eps=0.01, w_L=0.5, qam_bits=bits)
    rx = np.concatenate([inst.rx_pilot, inst.rx_data])
    sym_true = synth.qam_symbols(np.concatenate([
        oracle.hard_qam(inst.sym_pilot.astype(np.complex128), bits), inst.idx_data]), bits)
    st_dd, (pred, tgt) = oracle.train(p, rx, sym_true, decide_from=2 * P, return_io=True)
    st_tr = oracle.train(p, rx, sym_true)
    assert np.array_equal(tgt[P:], sym_true[P:])            # all decisions correct
    assert np.array_equal(oracle.hard_qam(pred[P:], bits), inst.idx_data)
    assert np.array_equal(st_dd.gamma, st_tr.gamma) and np.array_equal(st_dd.w, st_tr.w)


def test_output_at_arrival_is_f_n_of_x_n():
    M, K, P = 4, 2, 12
    inst = synth.make_instance(M, K, P, 0, 6.0, instance=25)
    p = oracle.Params(M=M, K=K, W=3, D=8, sigma=0.6, mu=0.8, eps=0.02, w_L=0.4)
    _, (pred, tgt) = oracle.train(p, inst.rx_pilot, inst.sym_pilot, decide_from=9, return_io=True)
    xs, _ = samples(inst.rx_pilot, inst.sym_pilot)
    for n in range(2 * P):
        f_n = oracle.train(p, inst.rx_pilot, inst.sym_pilot, n_steps=n, decide_from=9)
        if n % 2 == 0 and n // 2 >= p.D:   # the oldest entry leaves as pilot n/2 arrives (FIFO)
            f_n = oracle.State(centres=f_n.centres[2:], gamma=f_n.gamma[2:], w=f_n.w)
        y = oracle.eval_real(p, f_n, xs[n][None])[0] if f_n.centres.shape[0] else np.zeros(K)
        comp = pred[n // 2].real if n % 2 == 0 else pred[n // 2].imag
        np.testing.assert_allclose(comp, y, rtol=0, atol=1e-13)
        tcomp = tgt[n // 2].real if n % 2 == 0 else tgt[n // 2].imag
        if n >= 9:   # decided: the nearest QPSK level of the output at arrival
            np.testing.assert_allclose(tcomp, np.where(y >= 0, 1, -1) / math.sqrt(2), rtol=0, atol=1e-15)


def test_decisions_track_a_drifting_channel():
    """Tracking through the data symbols (Sec. II-D): after the pilots the channel rotates from
    H0 towards an independent H1; continuing in decision-directed mode keeps the symbol error
    rate below that of the filter frozen after the pilots."""
    M, K, P, N = 8, 2, 200, 800
    rng = np.random.default_rng(26)
    H0 = (rng.standard_normal((K, M)) + 1j * rng.standard_normal((K, M))) / math.sqrt(2)
    H1 = (rng.standard_normal((K, M)) + 1j * rng.standard_normal((K, M))) / math.sqrt(2)
    lab = rng.integers(0, 4, size=(P + N, K))
    s = synth.qpsk_symbols(lab)
    th = np.concatenate([np.zeros(P), np.linspace(0, 0.5 * math.pi, N)])[:, None, None]
    H_t = np.cos(th) * H0[None] + np.sin(th) * H1[None]
    noise = (rng.standard_normal((P + N, M)) + 1j * rng.standard_normal((P + N, M))) * math.sqrt(0.03 / 2)
    rx = np.einsum("tk,tkm->tm", s, H_t) + noise
    rx = (rx / math.sqrt(np.mean(np.sum(np.abs(rx[:P]) ** 2, axis=1)))).astype(np.complex64)
    sym = s.astype(np.complex64)
    p = oracle.Params(M=M, K=K, W=8, D=300, sigma=0.6, mu=0.5, eps=0.01, w_L=0.5)
    frozen = oracle.train(p, rx[:P], sym[:P])
    ser_frozen = np.mean(oracle.hard_qpsk(oracle.detect(p, frozen, rx[P:])) != lab[P:])
    _, (pred, _) = oracle.train(p, rx, sym, decide_from=2 * P, return_io=True)
    ser_dd = np.mean(oracle.hard_qpsk(pred[P:]) != lab[P:])
    assert ser_frozen > 0.05 and ser_dd < 0.5 * ser_frozen


# ------------------------------------------------------------------------------------------
# linear start: LS channel estimate + MMSE / ZF
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("bits", [2, 4])
def test_zf_from_noiseless_pilots_recovers_symbols(bits):
    """Noiseless, P >= K pilots: the LS estimate is the effective channel exactly; for QPSK the
    PA is a pure gain 1.1 (unit modulus), which the estimate absorbs, so ZF returns the
    transmitted symbols (for 16-QAM the PA compresses: the ZF output is the PA output / 1.1-free
    fit, checked for QPSK only)."""
    M, K, P, N = 8, 3, 40, 50
    inst = synth.make_instance(M, K, P, N, 10.0, instance=28, noiseless=True, bits=bits)
    W = oracle.linear_filter(inst.rx_pilot, inst.sym_pilot, 0.0)
    y = inst.rx_data.astype(np.complex128) @ W.conj()
    if bits == 2:
        np.testing.assert_allclose(y, inst.sym_data, atol=2e-6)
    else:   # the cubic PA is not linear for 16-QAM: the best linear fit still decides correctly
        assert np.array_equal(oracle.hard_qam(y, bits), inst.idx_data)


def test_mmse_matches_textbook_form_and_tends_to_zf():
    M, K, P = 8, 3, 64
    inst = synth.make_instance(M, K, P, 0, 8.0, instance=29)
    Y = inst.rx_pilot.astype(np.complex128).T
    S = inst.sym_pilot.astype(np.complex128).T
    H = Y @ S.conj().T @ np.linalg.inv(S @ S.conj().T)       # LS estimate, written out
    n0 = 10 ** (-0.8)
    W = oracle.linear_filter(inst.rx_pilot, inst.sym_pilot, n0)
    textbook = np.linalg.inv(H @ H.conj().T + n0 * np.eye(M)) @ H   # M x M form
    np.testing.assert_allclose(W, textbook, rtol=1e-10, atol=1e-12)
    W0 = oracle.linear_filter(inst.rx_pilot, inst.sym_pilot, 0.0)
    np.testing.assert_allclose(W0.conj().T @ H, np.eye(K), atol=1e-10)   # ZF inverts the estimate
    Wsmall = oracle.linear_filter(inst.rx_pilot, inst.sym_pilot, 1e-9)
    np.testing.assert_allclose(Wsmall, W0, rtol=1e-6, atol=1e-8)


def test_linear_start_speeds_up_convergence():
    """Sec. I: starting the APSM from a conventional linear filter instead of zero gives a lower
    error after few pilots (here: 24 pilots, 16 x 6, SNR 12 dB)."""
    M, K, P, N = 16, 6, 24, 2000
    inst = synth.make_instance(M, K, 400, N, 12.0, instance=30)
    rp, sp = inst.rx_pilot[:P], inst.sym_pilot[:P]
    p = oracle.Params(M=M, K=K, W=16, D=P, sigma=0.5, mu=0.5, eps=0.01, w_L=0.5)
    Wm = oracle.linear_filter(inst.rx_pilot[:P], inst.sym_pilot[:P], 10 ** (-1.2))
    c0 = Wm / p.w_L
    w0 = np.concatenate([c0.real.T, c0.imag.T], axis=1)
    st0 = oracle.train(p, rp, sp)
    stl = oracle.train(p, rp, sp, w0=w0)
    mse0 = np.mean(np.abs(oracle.detect(p, st0, inst.rx_data) - inst.sym_data) ** 2)
    msel = np.mean(np.abs(oracle.detect(p, stl, inst.rx_data) - inst.sym_data) ** 2)
    assert msel < 0.5 * mse0
