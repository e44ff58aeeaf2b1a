"""GPU parity of the rows beyond the baseline path, against the FP64 oracle on identical seeded
inputs:

  * Gray square-QAM decisions (16-QAM, 64-QAM) in every detection engine, and training on 16-QAM
    pilots, where the cubic power amplifier is truly nonlinear;
  * the violated-slab weights q_j = 1/|V_n| in every form of the training recurrence (blocked
    window warp, register ring, plain per-step loop);
  * resuming training from a state (apsm_train_continue) -- the oracle is the recurrence over the
    concatenated sequence -- including FIFO eviction across calls, a first call shorter than the
    window and a state loaded by apsm_state_set;
  * decision-directed tracking through the data vectors (targets decided at each arrival), with
    the outputs at arrival and the decided labels;
  * the linear start (LS channel estimate + MMSE / ZF filter) and training from it.
Tolerances and decision rules are those of tests/parity.py."""
import numpy as np
import pytest
import torch

import oracle
from paper_2201_05024_gb300 import apsm, synth

from parity import (TOL_FP32, assert_hard_match, assert_soft_close, boundary_distance, gpu_params, load_state,
                    oracle_state_fp32, rms, to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    apsm.load_library()


def _coef_errors(op, st, fst):
    ent, gam = st.entries()
    g_ref = fst.gamma.reshape(-1, 2, op.K)
    assert gam.shape == g_ref.shape
    dg = np.abs(gam.astype(np.float64) - g_ref).max() / max(rms(g_ref), 1e-30)
    c_ref = oracle.clin_from_w(op.M, fst.w)
    dc = np.abs(st.clin.cpu().numpy().astype(np.complex128) - c_ref).max() / max(rms(np.abs(c_ref)), 1e-30)
    return ent, dg, dc


# ------------------------------------------------------------------------------------------
# Gray square QAM
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("bits", [4, 6])
@pytest.mark.parametrize("engine", ["tensor", "ffma", "bf16"])
def test_qam_decisions_in_every_engine(bits, engine):
    M, K, D, N = 16, 6, 300, 2000
    ent, gam, clin = synth.random_state(M, K, D, instance=60 + bits)
    inst = synth.make_instance(M, K, 4, N, 10.0, instance=61, bits=bits)
    op = oracle.Params(M=M, K=K, W=1, D=D, qam_bits=bits)
    gp = gpu_params(op, dtype="bf16" if engine == "bf16" else "fp32")
    if engine == "ffma":
        apsm.tune_set(M, K, "fp32", "ffma", 64, 2, 1)
    try:
        st = load_state(gp, ent, gam, clin)
        soft, hard = apsm.detect(gp, st, to_dev(inst.rx_data))
    finally:
        apsm.tune_clear()
    ref = oracle.detect(op, oracle_state_fp32(M, ent, gam, clin), inst.rx_data)
    tol = 2e-2 if engine == "bf16" else TOL_FP32
    assert_soft_close(soft.cpu().numpy(), ref, tol=tol)
    assert_hard_match(hard.cpu().numpy(), ref, tol=tol, bits=bits)
    assert int(hard.max()) > 3            # really more than QPSK labels


@pytest.mark.parametrize("bits", [4, 6])
def test_training_on_qam_pilots(bits):
    """16 x 6 (and 64-QAM) pilots through the nonlinear PA: trained coefficients, detections and
    labels against the oracle."""
    M, K, P, N = 16, 6, 400, 1500
    inst = synth.make_instance(M, K, P, N, 25.0, instance=62, bits=bits)
    op = oracle.Params(M=M, K=K, W=16, D=P, sigma=0.5, mu=0.5, eps=0.01, w_L=0.5, qam_bits=bits)
    gp = gpu_params(op)
    st = apsm.State(gp)
    apsm.train(gp, to_dev(inst.rx_pilot), to_dev(inst.sym_pilot), st)
    fst = oracle.train(op, inst.rx_pilot, inst.sym_pilot)
    _, dg, dc = _coef_errors(op, st, fst)
    assert dg <= 1e-4 and dc <= 1e-4, (dg, dc)
    soft, hard = apsm.detect(gp, st, to_dev(inst.rx_data))
    ref = oracle.detect(op, fst, inst.rx_data)
    assert_soft_close(soft.cpu().numpy(), ref)
    assert_hard_match(hard.cpu().numpy(), ref, bits=bits)


# ------------------------------------------------------------------------------------------
# violated-slab weights
# ------------------------------------------------------------------------------------------

VIOL_CASES = [
    # M, K, P, W, D   (form of the recurrence)
    (16, 6, 300, 16, 300),     # blocked window warp
    (8, 3, 200, 8, 40),        # blocked, FIFO eviction
    (8, 2, 150, 30, 150),      # register ring (padded window 32)
    (4, 2, 120, 40, 100),      # plain per-step loop (padded window 48)
    (4, 1, 77, 1, 40),         # W = 1: the same as uniform weights
]


@pytest.mark.parametrize("M,K,P,W,D", VIOL_CASES)
def test_violated_weights_training(M, K, P, W, D):
    inst = synth.make_instance(M, K, P, 300, 10.0, instance=63 + W)
    op = oracle.Params(M=M, K=K, W=W, D=D, sigma=0.5, mu=0.8, eps=0.02, w_L=0.5, weights=1)
    gp = gpu_params(op)
    st = apsm.State(gp)
    cl = torch.full((2 * P, W, K), 127, dtype=torch.int8, device="cuda")
    apsm.train(gp, to_dev(inst.rx_pilot), to_dev(inst.sym_pilot), st, case_log=cl)
    fst, cases, margins = oracle.train(op, inst.rx_pilot, inst.sym_pilot, log_cases=True)
    gcl = cl.cpu().numpy()
    diff = (gcl != cases) & (cases != 127)
    if diff.any():
        # a branch may differ only at a near-tie; then the oracle replays the GPU's branches
        assert np.all(margins[diff] < 1e-5) and diff.sum() <= 4, (margins[diff].max(), diff.sum())
        forced = np.full(cases.shape, 127, dtype=np.int8)
        forced[diff] = gcl[diff]
        fst = oracle.train(op, inst.rx_pilot, inst.sym_pilot, forced=forced)
    _, dg, dc = _coef_errors(op, st, fst)
    assert dg <= 1e-4 and dc <= 1e-4, (dg, dc)
    soft, _ = apsm.detect(gp, st, to_dev(inst.rx_data))
    assert_soft_close(soft.cpu().numpy(), oracle.detect(op, fst, inst.rx_data))
    assert apsm.read_status(st) == 0


# ------------------------------------------------------------------------------------------
# resuming training
# ------------------------------------------------------------------------------------------

RESUME_CASES = [
    # M, K, W, D, P1, P2, (P3)     second (and third) call continue the first
    (16, 6, 16, 1024, 300, 500, 0),     # no eviction, two chunks in each call
    (8, 3, 8, 100, 150, 120, 90),       # FIFO eviction across the calls
    (4, 2, 8, 40, 2, 70, 5),            # first call shorter than the window
    (8, 2, 30, 150, 60, 80, 0),         # register-ring form, window reaching back 15 pilots
    (4, 1, 1, 30, 40, 50, 0),           # W = 1: nothing carried
    (16, 6, 16, 200, 180, 400, 0),      # 16 x 6 with eviction in the second call
]


@pytest.mark.parametrize("M,K,W,D,P1,P2,P3", RESUME_CASES)
def test_resume_equals_training_on_the_concatenation(M, K, W, D, P1, P2, P3):
    P = P1 + P2 + P3
    inst = synth.make_instance(M, K, P, 400, 10.0, instance=70 + P)
    op = oracle.Params(M=M, K=K, W=W, D=D, sigma=0.5, mu=0.6, eps=0.01, w_L=0.5)
    gp = gpu_params(op)
    rp, sp = to_dev(inst.rx_pilot), to_dev(inst.sym_pilot)
    st = apsm.State(gp)
    apsm.train(gp, rp[:P1], sp[:P1], st)
    soft2, hard2 = apsm.train_continue(gp, rp[P1:P1 + P2].contiguous(), st, sp[P1:P1 + P2].contiguous())
    if P3:
        apsm.train_continue(gp, rp[P1 + P2:].contiguous(), st, sp[P1 + P2:].contiguous(), want_outputs=False)
    torch.cuda.synchronize()
    assert st.meta[:3].tolist() == [min(P, D), P % D if P >= D else 0, P]
    fst, (pred, tgt) = oracle.train(op, inst.rx_pilot, inst.sym_pilot, return_io=True)
    ent, dg, dc = _coef_errors(op, st, fst)
    np.testing.assert_array_equal(ent, inst.rx_pilot[fst.first_entry:fst.first_entry + fst.n_entries])
    assert dg <= 1e-4 and dc <= 1e-4, (dg, dc)
    # outputs at arrival of the second call and the labels of its targets (the given symbols)
    assert_soft_close(soft2.cpu().numpy(), pred[P1:P1 + P2], what="output at arrival")
    assert np.array_equal(hard2.cpu().numpy(), oracle.hard_qam(inst.sym_pilot[P1:P1 + P2].astype(np.complex128), 2))
    soft, _ = apsm.detect(gp, st, to_dev(inst.rx_data))
    assert_soft_close(soft.cpu().numpy(), oracle.detect(op, fst, inst.rx_data))
    assert apsm.read_status(st) == 0


def test_resume_from_a_loaded_state():
    """apsm_state_set with the entries' targets, then continue: the same as the oracle training on
    the loaded entries' pilots followed by the new ones."""
    M, K, W, D, P1, P2 = 8, 3, 8, 64, 50, 90
    inst = synth.make_instance(M, K, P1 + P2, 200, 10.0, instance=77)
    op = oracle.Params(M=M, K=K, W=W, D=D, sigma=0.5, mu=0.6, eps=0.01, w_L=0.5)
    gp = gpu_params(op)
    f1 = oracle.train(op, inst.rx_pilot[:P1], inst.sym_pilot[:P1])
    ent = inst.rx_pilot[:P1]
    st = apsm.State(gp)
    apsm.state_set(gp, st, to_dev(ent), to_dev(f1.gamma.reshape(-1, 2, K).astype(np.float32)),
                   to_dev(oracle.clin_from_w(M, f1.w).astype(np.complex64)), target=to_dev(inst.sym_pilot[:P1]))
    apsm.train_continue(gp, to_dev(inst.rx_pilot[P1:]), st, to_dev(inst.sym_pilot[P1:]), want_outputs=False)
    fst = oracle.train(op, inst.rx_pilot, inst.sym_pilot)
    _, dg, dc = _coef_errors(op, st, fst)
    assert dg <= 1e-4 and dc <= 1e-4, (dg, dc)


# ------------------------------------------------------------------------------------------
# decision-directed tracking
# ------------------------------------------------------------------------------------------

TRACK_CASES = [
    # M, K, P pilots, N tracked, W, D, bits, SNR, instance
    (16, 6, 300, 600, 16, 1024, 2, 12.0, 680),
    (8, 2, 120, 300, 8, 100, 2, 8.0, 380),     # eviction while tracking
    (8, 2, 120, 300, 8, 100, 2, 0.0, 381),     # 1.3 % wrong decisions fed back as targets
    (16, 4, 400, 400, 16, 1024, 4, 22.0, 480), # 16-QAM through the nonlinear PA
]


@pytest.mark.parametrize("M,K,P,N,W,D,bits,snr,seed", TRACK_CASES)
def test_decision_directed_tracking(M, K, P, N, W, D, bits, snr, seed):
    inst = synth.make_instance(M, K, P, N, snr, instance=seed, bits=bits)
    op = oracle.Params(M=M, K=K, W=W, D=D, sigma=0.5, mu=0.5, eps=0.01, w_L=0.5, qam_bits=bits)
    gp = gpu_params(op)
    rx = np.concatenate([inst.rx_pilot, inst.rx_data])
    sym = np.concatenate([inst.sym_pilot, np.zeros((N, K), np.complex64)])
    fst, (pred, tgt) = oracle.train(op, rx, sym, decide_from=2 * P, return_io=True)
    # a decision taken in FP32 and in FP64 can differ only at a boundary; the case must keep
    # every tracked output well away from one, or the two trajectories would part
    margin = min(boundary_distance(pred[P:].real, bits).min(), boundary_distance(pred[P:].imag, bits).min())
    assert margin > 1e-3 * np.sqrt(np.mean(pred[P:].real ** 2)), "choose another seed: a decision at a tie"
    st = apsm.State(gp)
    apsm.train(gp, to_dev(inst.rx_pilot), to_dev(inst.sym_pilot), st)
    soft, hard = apsm.train_continue(gp, to_dev(inst.rx_data), st, None)
    torch.cuda.synchronize()
    assert np.array_equal(hard.cpu().numpy(), oracle.hard_qam(tgt[P:], bits))   # the same decisions
    assert_soft_close(soft.cpu().numpy(), pred[P:], what="tracked outputs")
    _, dg, dc = _coef_errors(op, st, fst)
    assert dg <= 1e-4 and dc <= 1e-4, (dg, dc)
    ser = float(np.mean(hard.cpu().numpy() != inst.idx_data))
    assert ser == float(np.mean(oracle.hard_qam(tgt[P:], bits) != inst.idx_data)) and ser < 0.2
    assert apsm.read_status(st) == 0


# ------------------------------------------------------------------------------------------
# linear start
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("M,K,P,noise", [(16, 6, 64, 0.1), (64, 16, 200, 0.03), (4, 2, 10, 0.0), (8, 8, 8, 0.5)])
def test_linear_init_matches_oracle(M, K, P, noise):
    inst = synth.make_instance(M, K, P, 10, 10.0, instance=90 + M)
    gp = apsm.Params(M=M, K=K, window=8, dict_cap=64, w_L=0.5)
    c0 = apsm.linear_init(gp, to_dev(inst.rx_pilot), to_dev(inst.sym_pilot), noise).cpu().numpy()
    ref = oracle.linear_filter(inst.rx_pilot, inst.sym_pilot, noise) / gp.w_L
    assert np.abs(c0 - ref).max() <= 1e-4 * max(rms(np.abs(ref)), 1e-30) * 10, np.abs(c0 - ref).max() / rms(np.abs(ref))


def test_zf_start_detects_noiseless_symbols_and_training_from_it():
    M, K, P, N = 16, 6, 40, 500
    inst = synth.make_instance(M, K, P, N, 10.0, instance=95, noiseless=True)
    op = oracle.Params(M=M, K=K, W=16, D=P, sigma=0.5, mu=0.5, eps=0.01, w_L=0.5)
    gp = gpu_params(op)
    c0 = apsm.linear_init(gp, to_dev(inst.rx_pilot), to_dev(inst.sym_pilot), 0.0)
    st = apsm.State(gp)
    apsm.train(gp, to_dev(inst.rx_pilot[:0]), to_dev(inst.sym_pilot[:0]), st, clin0=c0)   # f_0 only
    soft, _ = apsm.detect(gp, st, to_dev(inst.rx_data))
    np.testing.assert_allclose(soft.cpu().numpy(), inst.sym_data, atol=1e-4)
    # training from the linear start against the oracle from the same start
    w0c = c0.cpu().numpy().astype(np.complex128)
    w0 = np.concatenate([w0c.real.T, w0c.imag.T], axis=1)
    noisy = synth.make_instance(M, K, P, N, 10.0, instance=96)
    st2 = apsm.State(gp)
    apsm.train(gp, to_dev(noisy.rx_pilot), to_dev(noisy.sym_pilot), st2, clin0=c0)
    fst = oracle.train(op, noisy.rx_pilot, noisy.sym_pilot, w0=w0)
    _, dg, dc = _coef_errors(op, st2, fst)
    assert dg <= 1e-4 and dc <= 1e-4, (dg, dc)
