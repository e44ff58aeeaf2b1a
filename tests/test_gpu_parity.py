"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on identical seeded
inputs.  Detection is compared element by element; training compares the trained coefficients,
the branch of Eq. beta taken at every (step, window slot, user), and the detections of the
two trained filters.  Tolerances are in tests/parity.py."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2201_05024_gb300 import apsm, synth

from parity import (TOL_FP32, assert_hard_match, assert_soft_close, gpu_params, load_state, oracle_state_fp32,
                    rms, to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    apsm.load_library()


# ------------------------------------------------------------------------------------------
# detection
# ------------------------------------------------------------------------------------------

DETECT_CASES = [
    # M, K, D entries, N queries, sigma, w_L
    (4, 2, 200, 1000, 0.5, 0.5),        # 1-pilot-config shapes
    (16, 6, 1000, 3001, 0.5, 0.5),      # several tiles, ragged entry tile and query tail
    (2, 1, 33, 65, 0.7, 0.3),
    (8, 3, 100, 257, 0.4, 0.8),
    (32, 12, 300, 513, 0.6, 0.5),
    (64, 16, 130, 300, 0.5, 0.5),
    (64, 7, 70, 131, 0.5, 0.5),         # two lanes per query, odd user count, ragged tail
    (16, 16, 64, 70, 0.3, 0.0),         # Gaussian part only
    (8, 5, 40, 129, 0.5, 1.0),          # linear part only
    (16, 6, 1, 31, 0.5, 0.5),           # a single entry
    (8, 12, 300, 513, 0.5, 0.5),        # TMA-staged form: 8 antennas, 12 users
    (4, 8, 130, 129, 0.6, 0.4),         # TMA-staged form: three tiles, two entries in the last
    (16, 4, 129, 128, 0.5, 0.5),        # one entry in the last tile, whole query tiles
    (16, 2, 640, 2049, 0.5, 0.5),       # ten whole tiles (every stage reused several times)
]


@pytest.fixture(params=["tensor", "tensor-conv", "ffma"])
def engine(request):
    """FP32 detection engine: Gram on the tensor cores (TF32 x3, the default where a kernel exists;
    operands staged by TMA where that form applies, "tensor-conv": entry rows converted in shared
    memory everywhere) or on the FP32 FMA pipe (chosen for every class through the launch-choice
    table)."""
    if request.param == "ffma":
        for M in (2, 4, 8, 16, 32, 64):
            for K in range(1, 17):
                apsm.tune_set(M, K, "fp32", "ffma", 64, 2, 1)
    if request.param == "tensor-conv":
        apsm.set_option("detect_tma", 0)
    yield request.param
    apsm.tune_clear()
    apsm.set_option("detect_tma", 1)


@pytest.mark.parametrize("M,K,D,N,sigma,wL", DETECT_CASES)
def test_detect_matches_oracle(M, K, D, N, sigma, wL, engine):
    ent, gam, clin = synth.random_state(M, K, D, instance=D + 7 * M + K)
    inst = synth.make_instance(M, K, 4, N, 10.0, instance=M * 100 + K)
    op = oracle.Params(M=M, K=K, W=1, D=D, sigma=sigma, w_L=wL)
    gp = gpu_params(op)
    st = load_state(gp, ent, gam, clin)
    soft, hard = apsm.detect(gp, st, to_dev(inst.rx_data))
    ref = oracle.detect(op, oracle_state_fp32(M, ent, gam, clin), inst.rx_data)
    assert_soft_close(soft.cpu().numpy(), ref)
    assert_hard_match(hard.cpu().numpy(), ref)
    assert apsm.read_status(st) == 0


@pytest.mark.parametrize("M,K", [(16, 6), (8, 3), (4, 2), (32, 4), (16, 16)])
def test_detect_ignores_slots_past_the_held_entries(M, K, engine):
    """A dictionary holding fewer entries than its capacity: the unused slots (NaN here) take no
    part in detection, whatever they hold."""
    D, n, N = 300, 170, 700
    ent, gam, clin = synth.random_state(M, K, n, instance=11 * M + K)
    inst = synth.make_instance(M, K, 4, N, 10.0, instance=5 * M + K)
    op = oracle.Params(M=M, K=K, W=1, D=D, sigma=0.5, w_L=0.5)
    gp = gpu_params(op)
    st = apsm.State(gp)
    st.dict.fill_(complex(float("nan"), float("nan")))
    st.dict_norm.fill_(float("nan"))
    st.gamma.fill_(float("nan"))
    apsm.state_set(gp, st, to_dev(np.asarray(ent, np.complex64)), to_dev(np.asarray(gam, np.float32)),
                   to_dev(np.asarray(clin, np.complex64)))
    soft, hard = apsm.detect(gp, st, to_dev(inst.rx_data))
    ref = oracle.detect(op, oracle_state_fp32(M, ent, gam, clin), inst.rx_data)
    assert_soft_close(soft.cpu().numpy(), ref)
    assert_hard_match(hard.cpu().numpy(), ref)
    assert apsm.read_status(st) == 0


BALANCED_CASES = [
    # M, K, D entries, N queries
    (16, 6, 1024, 8192),      # 64 query tiles x 16 entry tiles over the SMs: tiles split between CTAs
    (16, 6, 1000, 3001),      # ragged entry tile and query tail
    (8, 4, 300, 1000),        # 40 units: fewer than the CTAs (CTAs with one unit or none)
    (4, 2, 64, 129),          # one entry tile
    (16, 12, 700, 5000),      # one CTA per SM (12 users)
    (16, 2, 1, 200),          # a single entry
    (8, 16, 2000, 777),       # 32 entry tiles over 7 query tiles
]


@pytest.mark.parametrize("M,K,D,N", BALANCED_CASES)
def test_balanced_detection(M, K, D, N):
    """apsm_detect_ws: the work split evenly over the SMs, split query tiles merged through the
    workspace.  Against the FP64 oracle; bit-identical on a second call; the workspace's arrival
    counters are left at zero; the same soft outputs as the plain form up to FP32 rounding order."""
    ent, gam, clin = synth.random_state(M, K, D, instance=3 * D + M + K)
    inst = synth.make_instance(M, K, 4, N, 10.0, instance=N + M)
    op = oracle.Params(M=M, K=K, W=1, D=D, sigma=0.5, w_L=0.5)
    gp = gpu_params(op)
    st = load_state(gp, ent, gam, clin)
    ws = apsm.detect_workspace(gp, N)
    assert ws is not None and ws.numel() > 0
    rx = to_dev(inst.rx_data)
    soft, hard = apsm.detect(gp, st, rx, workspace=ws)
    ref = oracle.detect(op, oracle_state_fp32(M, ent, gam, clin), inst.rx_data)
    assert_soft_close(soft.cpu().numpy(), ref)
    assert_hard_match(hard.cpu().numpy(), ref)
    assert apsm.read_status(st) == 0
    assert torch.count_nonzero(ws[:4 * ((N + 127) // 128)]) == 0
    soft2, hard2 = apsm.detect(gp, st, rx, workspace=ws)
    assert torch.equal(soft, soft2) and torch.equal(hard, hard2)
    plain, _ = apsm.detect(gp, st, rx)
    assert_soft_close(soft.cpu().numpy(), plain.cpu().numpy().astype(np.complex128), tol=1e-5, what="plain form")


def test_balanced_detection_ignores_slots_past_the_held_entries():
    M, K, D, n, N = 16, 6, 1000, 333, 4000
    ent, gam, clin = synth.random_state(M, K, n, instance=77)
    inst = synth.make_instance(M, K, 4, N, 10.0, instance=78)
    op = oracle.Params(M=M, K=K, W=1, D=D, sigma=0.5, w_L=0.5)
    gp = gpu_params(op)
    st = apsm.State(gp)
    st.dict.fill_(complex(float("nan"), float("nan")))
    st.dict_norm.fill_(float("nan"))
    st.gamma.fill_(float("nan"))
    apsm.state_set(gp, st, to_dev(np.asarray(ent, np.complex64)), to_dev(np.asarray(gam, np.float32)),
                   to_dev(np.asarray(clin, np.complex64)))
    ws = apsm.detect_workspace(gp, N)
    soft, hard = apsm.detect(gp, st, to_dev(inst.rx_data), workspace=ws)
    ref = oracle.detect(op, oracle_state_fp32(M, ent, gam, clin), inst.rx_data)
    assert_soft_close(soft.cpu().numpy(), ref)
    assert_hard_match(hard.cpu().numpy(), ref)
    assert torch.count_nonzero(ws[:4 * ((N + 127) // 128)]) == 0


@pytest.mark.parametrize("case", ["offset", "mixed_queries"])
def test_balanced_detection_unnormalised_inputs(case):
    """Query tiles outside the factor range take the guarded form in the balanced kernel too."""
    M, K, D, N = 16, 6, 200, 1500
    rng = np.random.default_rng(12)
    ent, gam, clin = synth.random_state(M, K, D, instance=5)
    inst = synth.make_instance(M, K, 4, N, 10.0, instance=6)
    rx = inst.rx_data.copy()
    sigma = 0.5
    if case == "offset":
        base = (rng.standard_normal(M) + 1j * rng.standard_normal(M)) * 1.6
        ent = (ent + base).astype(np.complex64)
        rx = (rx * 0.5 + base).astype(np.complex64)
        sigma = 0.8
    else:
        rx[::97] *= 5.0
    op = oracle.Params(M=M, K=K, W=1, D=D, sigma=sigma, w_L=0.5)
    gp = gpu_params(op)
    st = load_state(gp, ent, gam, clin)
    soft, hard = apsm.detect(gp, st, to_dev(rx), workspace=apsm.detect_workspace(gp, N))
    ref = oracle.detect(op, oracle_state_fp32(M, ent, gam, clin), rx)
    assert_soft_close(soft.cpu().numpy(), ref)
    assert_hard_match(hard.cpu().numpy(), ref)


@pytest.mark.parametrize("M,K", [(16, 6), (64, 5)])
@pytest.mark.parametrize("case", ["offset", "mixed_entries", "mixed_queries"])
def test_detect_unnormalised_inputs(case, M, K, engine):
    """Inputs outside the range where the factored exponentials are used: a large common offset
    (||r||^2 >> ||r - r_t||^2, where a norm expansion would cancel), a dictionary whose tiles are
    partly out of range, and query blocks that are partly out of range."""
    D, N = 200, 700
    rng = np.random.default_rng(11)
    ent, gam, clin = synth.random_state(M, K, D, instance=5)
    inst = synth.make_instance(M, K, 4, N, 10.0, instance=6)
    rx = inst.rx_data.copy()
    sigma = 0.5
    if case == "offset":
        base = (rng.standard_normal(M) + 1j * rng.standard_normal(M)) * 1.6
        ent = (ent + base).astype(np.complex64)
        rx = (rx * 0.5 + base).astype(np.complex64)
        sigma = 0.8
    elif case == "mixed_entries":
        ent = ent.copy()
        ent[64:128] *= 6.0                      # tiles 2 and 3 out of range
    else:
        rx[::97] *= 5.0                          # a few queries out of range
    op = oracle.Params(M=M, K=K, W=1, D=D, sigma=sigma, w_L=0.5)
    gp = gpu_params(op)
    st = load_state(gp, ent, gam, clin)
    soft, hard = apsm.detect(gp, st, to_dev(rx))
    ref = oracle.detect(op, oracle_state_fp32(M, ent, gam, clin), rx)
    assert_soft_close(soft.cpu().numpy(), ref)
    assert_hard_match(hard.cpu().numpy(), ref)


HALF_CASES = [
    # M, K, D, N, dtype
    (64, 16, 300, 1000, "bf16"),    # the 64-antenna, 16-user precision-form shape, small
    (64, 16, 300, 1000, "fp16"),
    (16, 6, 200, 700, "bf16"),
    (8, 3, 65, 129, "fp16"),
    (2, 1, 5, 40, "bf16"),
    (4, 2, 70, 200, "bf16"),        # operands element by element (a core row spans Re and Im)
    (32, 12, 130, 300, "bf16"),     # operands by whole core rows, coefficients as float4
]
TOL_HALF = 2e-2


@pytest.fixture(params=["tc-coef", "fma-coef"])
def half_coef(request):
    """Where the reduced-precision form forms its coefficient sums: on the tensor cores (with a
    workspace, for 16, 32 and 64 antennas) or on the FP32 FMA pipe (no workspace)."""
    yield request.param


@pytest.mark.parametrize("M,K,D,N,dtype", HALF_CASES)
def test_detect_reduced_precision_matches_oracle(M, K, D, N, dtype, half_coef):
    """BF16 / FP16 Gram on the tensor cores with FP32 accumulation, exponentials and sums:
    soft outputs within 2e-2 (scaled) of the FP64 oracle, decisions identical away from a
    boundary; the error against the FP32 path is reported by the benchmark."""
    ent, gam, clin = synth.random_state(M, K, D, instance=D + M + 3)
    inst = synth.make_instance(M, K, 4, N, 10.0, instance=N + M)
    op = oracle.Params(M=M, K=K, W=1, D=D, sigma=0.5, w_L=0.5)
    gp = gpu_params(op, dtype=dtype)
    st = load_state(gp, ent, gam, clin)
    ws = apsm.detect_workspace(gp, N) if half_coef == "tc-coef" else None
    soft, hard = apsm.detect(gp, st, to_dev(inst.rx_data), workspace=ws)
    ref = oracle.detect(op, oracle_state_fp32(M, ent, gam, clin), inst.rx_data)
    err = assert_soft_close(soft.cpu().numpy(), ref, tol=TOL_HALF, what=dtype)
    assert err > 1e-6  # really the reduced-precision path
    assert_hard_match(hard.cpu().numpy(), ref, tol=TOL_HALF)



def _unnormalised(case, M, K):
    """Inputs far outside the gain-controlled range (shared by the FP32 and BF16/FP16 checks)."""
    D, N = 200, 700
    rng = np.random.default_rng(11)
    ent, gam, clin = synth.random_state(M, K, D, instance=5)
    inst = synth.make_instance(M, K, 4, N, 10.0, instance=6)
    rx = inst.rx_data.copy()
    sigma = 0.5
    if case == "offset":
        base = (rng.standard_normal(M) + 1j * rng.standard_normal(M)) * 1.6
        ent = (ent + base).astype(np.complex64)
        rx = (rx * 0.5 + base).astype(np.complex64)
        sigma = 0.8
    elif case == "mixed_entries":
        ent = ent.copy()
        ent[64:128] *= 6.0                      # tiles 2 and 3 out of range
    else:
        rx[::97] *= 5.0                          # a few queries out of range
    return ent, gam, clin, rx, sigma


def _bf16(x):
    """Round-to-nearest-even BF16 of float32 values (test-side emulation, for the regression check)."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _unguarded_bf16_detect(M, K, ent, gam, clin, rx, sigma, w_L):
    """What a BF16 Gram with the norm expansion alone would return (no direct-difference fallback):
    exponent 2 k2 Re/Im z from BF16-rounded operands, minus k2 (n_s + n_t) in FP64."""
    k2 = 1.0 / (2 * sigma * sigma)
    q = rx.astype(np.complex128)
    e = ent.astype(np.complex128)
    qa = _bf16(np.concatenate([q.real, q.imag], 1) * 2 * k2).astype(np.float64)
    ea = _bf16(np.concatenate([e.real, e.imag], 1)).astype(np.float64)
    eb = _bf16(np.concatenate([-e.imag, e.real], 1)).astype(np.float64)
    vr, vi = qa @ ea.T, qa @ eb.T                     # 2 k2 Re z, 2 k2 Im z
    h = k2 * (np.sum(np.abs(q) ** 2, 1)[:, None] + np.sum(np.abs(e) ** 2, 1)[None, :])
    EA, EB, EC = np.exp(vr - h), np.exp(vi - h), np.exp(-vi - h)
    g1, g2 = gam[:, 0, :].astype(np.float64), gam[:, 1, :].astype(np.float64)
    lin = q @ np.conj(clin.astype(np.complex128))
    y1 = w_L * lin.real + (1 - w_L) * (EA @ g1 + EC @ g2)
    y2 = w_L * lin.imag + (1 - w_L) * (EB @ g1 + EA @ g2)
    return y1 + 1j * y2


@pytest.mark.parametrize("M,K", [(16, 6), (64, 5)])
@pytest.mark.parametrize("case", ["offset", "mixed_entries", "mixed_queries"])
@pytest.mark.parametrize("dtype", ["bf16", "fp16"])
def test_detect_reduced_precision_unnormalised_inputs(case, M, K, dtype, half_coef):
    """BF16/FP16 Gram on inputs outside the gain-controlled range: the pairs where the norm
    expansion cancels (smallest distance below 2^-4 k2 (||r||^2 + ||r_t||^2)) are recomputed by
    direct differences in FP32, so the result stays within 2e-2 of the FP64 oracle."""
    ent, gam, clin, rx, sigma = _unnormalised(case, M, K)
    op = oracle.Params(M=M, K=K, W=1, D=ent.shape[0], sigma=sigma, w_L=0.5)
    gp = gpu_params(op, dtype=dtype)
    st = load_state(gp, ent, gam, clin)
    ws = apsm.detect_workspace(gp, rx.shape[0]) if half_coef == "tc-coef" else None
    soft, hard = apsm.detect(gp, st, to_dev(rx), workspace=ws)
    ref = oracle.detect(op, oracle_state_fp32(M, ent, gam, clin), rx)
    assert_soft_close(soft.cpu().numpy(), ref, tol=TOL_HALF, what=f"{dtype} {case}")
    assert_hard_match(hard.cpu().numpy(), ref, tol=TOL_HALF)
    assert apsm.read_status(st) == 0


def test_direct_difference_fallback_regression():
    """The offset case at 16 antennas: with a BF16 Gram and the norm expansion alone (emulated on
    the CPU) the error is far above the 2e-2 tolerance -- the case needs the fallback -- while
    the GPU's guarded BF16 path stays within it."""
    M, K = 16, 6
    ent, gam, clin, rx, sigma = _unnormalised("offset", M, K)
    op = oracle.Params(M=M, K=K, W=1, D=ent.shape[0], sigma=sigma, w_L=0.5)
    ref = oracle.detect(op, oracle_state_fp32(M, ent, gam, clin), rx)
    from parity import rel_errors
    unguarded, _ = rel_errors(_unguarded_bf16_detect(M, K, ent, gam, clin, rx, sigma, 0.5), ref)
    assert unguarded.max() > 5 * TOL_HALF
    gp = gpu_params(op, dtype="bf16")
    st = load_state(gp, ent, gam, clin)
    soft, _ = apsm.detect(gp, st, to_dev(rx))
    assert_soft_close(soft.cpu().numpy(), ref, tol=TOL_HALF, what="guarded bf16")


@pytest.mark.parametrize("dtype", ["fp32", "bf16"])
def test_detect_empty_dictionary_is_linear_filter(dtype):
    M, K, N = 16, 6, 200
    ent, gam, clin = synth.random_state(M, K, 0)
    inst = synth.make_instance(M, K, 4, N, 10.0, instance=3)
    op = oracle.Params(M=M, K=K, W=1, D=8)
    gp = gpu_params(op, dtype=dtype)
    st = load_state(gp, ent, gam, clin)
    soft, _ = apsm.detect(gp, st, to_dev(inst.rx_data))
    ref = 0.5 * (inst.rx_data.astype(np.complex128) @ np.conj(clin.astype(np.complex128)))
    assert_soft_close(soft.cpu().numpy(), ref)


def test_detect_zero_queries_is_a_no_op():
    op = oracle.Params(M=8, K=2, W=1, D=8)
    gp = gpu_params(op)
    ent, gam, clin = synth.random_state(8, 2, 8)
    st = load_state(gp, ent, gam, clin)
    soft, hard = apsm.detect(gp, st, torch.empty((0, 8), dtype=torch.complex64, device="cuda"))
    assert soft.shape == (0, 2) and hard.shape == (0, 2)


def test_detect_is_deterministic():
    M, K, D, N = 16, 6, 700, 5000
    ent, gam, clin = synth.random_state(M, K, D, instance=1)
    inst = synth.make_instance(M, K, 4, N, 10.0, instance=2)
    gp = gpu_params(oracle.Params(M=M, K=K, W=1, D=D))
    st = load_state(gp, ent, gam, clin)
    rx = to_dev(inst.rx_data)
    a, _ = apsm.detect(gp, st, rx)
    b, _ = apsm.detect(gp, st, rx)
    assert torch.equal(a, b)


def test_detect_rejects_a_wrong_shape():
    gp = apsm.Params(M=16, K=6, window=4, dict_cap=16)
    st = apsm.State(gp)
    with pytest.raises(ValueError):
        apsm.detect(gp, st, torch.zeros((10, 8), dtype=torch.complex64, device="cuda"))


# ------------------------------------------------------------------------------------------
# training
# ------------------------------------------------------------------------------------------

def _train_both(op, inst, *, w0=None, log=True):
    gp = gpu_params(op)
    P = inst.rx_pilot.shape[0]
    st = apsm.State(gp)
    cl = torch.full((2 * P, op.W, op.K), 127, dtype=torch.int8, device="cuda") if log else None
    clin0 = None if w0 is None else to_dev(oracle.clin_from_w(op.M, w0).astype(np.complex64))
    apsm.train(gp, to_dev(inst.rx_pilot), to_dev(inst.sym_pilot), st, clin0=clin0, case_log=cl)
    ref = oracle.train(op, inst.rx_pilot, inst.sym_pilot, w0=w0, log_cases=log)
    torch.cuda.synchronize()
    return gp, st, cl, ref


def _compare_training(op, inst, gp, st, cl, ref, *, tol_coef, tol_soft=TOL_FP32, tie=1e-5, w0=None):
    """GPU training against the oracle.  The Eq. beta branch of a (step, slot, user) may differ
    only at a near-tie of |e| with eps in the FP64 run (margin < tie * max(1, |b|)); where any
    does, the oracle is replayed with the GPU's branches forced at those slots and the
    coefficients are compared with that replay.  Returns the errors and the number of flips."""
    fst, cases, margins = ref
    P = inst.rx_pilot.shape[0]
    meta = st.meta.cpu().numpy()
    assert meta[0] == min(P, op.D) and meta[2] == P
    assert meta[1] == (P % op.D if P >= op.D else 0)
    ent, gam = st.entries()
    # dictionary entries are copies of the last pilots, bit for bit
    np.testing.assert_array_equal(ent, inst.rx_pilot[fst.first_entry:fst.first_entry + fst.n_entries])
    # branch of Eq. beta: identical except at near-ties of |e| with eps in the FP64 run
    gcl = cl.cpu().numpy()
    valid = cases != 127
    assert np.array_equal(gcl == 127, ~valid)
    diff = valid & (gcl != cases)
    n_flip = int(diff.sum())
    if n_flip:
        b_max = max(1.0, float(np.abs(inst.sym_pilot.view(np.float32)).max()))
        assert np.all(margins[diff] < tie * b_max), f"branch differs away from a tie: margins {margins[diff].max():.2e}"
        assert n_flip <= max(4, int(1e-4 * valid.sum())), f"{n_flip} branch flips"
        forced = np.full(cases.shape, 127, dtype=np.int8)
        forced[diff] = gcl[diff]
        fst = oracle.train(op, inst.rx_pilot, inst.sym_pilot, w0=w0, forced=forced)
    # coefficients, rms-normalised
    g_ref = fst.gamma.reshape(-1, 2, op.K)
    dg = np.abs(gam.astype(np.float64) - g_ref).max() / max(rms(g_ref), 1e-30)
    c_gpu = st.clin.cpu().numpy().astype(np.complex128)
    c_ref = oracle.clin_from_w(op.M, fst.w)
    dc = np.abs(c_gpu - c_ref).max() / max(rms(np.abs(c_ref)), 1e-30)
    assert dg <= tol_coef, f"gamma error {dg:.3e}"
    assert dc <= tol_coef, f"clin error {dc:.3e}"
    # the two trained filters detect the same soft symbols
    soft, hard = apsm.detect(gp, st, to_dev(inst.rx_data))
    ref_soft = oracle.detect(op, fst, inst.rx_data)
    err = assert_soft_close(soft.cpu().numpy(), ref_soft, tol=tol_soft, what="soft after training")
    assert_hard_match(hard.cpu().numpy(), ref_soft, tol=tol_soft)
    assert apsm.read_status(st) == 0
    return dg, dc, err, n_flip


TRAIN_CASES = [
    # M, K, P, W, D, sigma, mu, eps, w_L, N
    (4, 2, 200, 8, 200, 0.5, 0.5, 0.01, 0.5, 1000),     # the small APSM configuration
    (4, 2, 100, 8, 20, 0.5, 0.5, 0.01, 0.5, 300),       # FIFO eviction, chunk limited by D
    (8, 3, 150, 5, 9, 0.6, 1.0, 0.02, 0.4, 300),        # small D: one- or few-pilot chunks
    (4, 1, 77, 1, 40, 0.5, 1.0, 0.0, 0.5, 100),         # W = 1, ragged last chunk, eps = 0
    (16, 6, 5, 16, 64, 0.5, 0.5, 0.01, 0.5, 100),       # fewer pilots than one chunk
    (2, 4, 1, 3, 4, 0.5, 0.5, 0.01, 0.5, 50),           # a single pilot
    (32, 12, 90, 31, 50, 0.7, 1.9, 0.05, 0.7, 200),     # odd window, strong relaxation
    (8, 16, 70, 16, 70, 0.5, 0.5, 0.01, 1.0, 100),      # linear-only kernel
    (8, 2, 70, 16, 70, 0.5, 0.5, 0.01, 0.0, 100),       # Gaussian-only kernel
    (64, 4, 60, 10, 60, 0.5, 0.5, 0.01, 0.5, 100),
    (64, 5, 200, 8, 100, 0.5, 0.5, 0.01, 0.5, 150),     # 64 antennas over several chunks, eviction
    (16, 6, 600, 16, 200, 0.5, 0.5, 0.01, 0.5, 300),    # many full chunks, eviction, ring wrap
]


@pytest.mark.parametrize("M,K,P,W,D,sigma,mu,eps,wL,N", TRAIN_CASES)
def test_train_matches_oracle(M, K, P, W, D, sigma, mu, eps, wL, N):
    inst = synth.make_instance(M, K, P, N, 10.0, instance=P + M + K)
    op = oracle.Params(M=M, K=K, W=W, D=D, sigma=sigma, mu=mu, eps=eps, w_L=wL)
    gp, st, cl, ref = _train_both(op, inst)
    _compare_training(op, inst, gp, st, cl, ref, tol_coef=1e-4)


@pytest.mark.parametrize("M,K,P,W,D", [(16, 6, 600, 16, 200), (8, 3, 333, 8, 1000), (4, 2, 100, 8, 20)])
def test_tracked_and_sequential_training_agree(M, K, P, W, D):
    """The next-chunk tracking form (frozen-entry phase A beside phase B) and the sequential form
    (whole-dictionary phase A between chunks) compute the same recurrence; both match the oracle."""
    inst = synth.make_instance(M, K, P, 200, 10.0, instance=7 * P + D)
    op = oracle.Params(M=M, K=K, W=W, D=D)
    results = []
    try:
        for track in (1, 0):
            apsm.set_option("train_track", track)
            gp, st, cl, ref = _train_both(op, inst)
            _compare_training(op, inst, gp, st, cl, ref, tol_coef=1e-4)
            results.append((st.gamma.cpu().numpy(), st.clin.cpu().numpy()))
    finally:
        apsm.set_option("train_track", 1)
    (g1, c1), (g0, c0) = results
    assert np.abs(g1 - g0).max() <= 1e-4 * rms(g0)
    assert np.abs(c1 - c0).max() <= 1e-4 * rms(np.abs(c0))


def test_train_with_initial_linear_filter():
    M, K, P = 8, 3, 60
    inst = synth.make_instance(M, K, P, 200, 10.0, instance=41)
    op = oracle.Params(M=M, K=K, W=6, D=30)
    w0 = np.random.default_rng(4).standard_normal((K, 2 * M)) * 0.3
    gp, st, cl, ref = _train_both(op, inst, w0=w0)
    _compare_training(op, inst, gp, st, cl, ref, tol_coef=1e-4, w0=w0)


def test_train_zero_pilots_leaves_empty_filter():
    gp = apsm.Params(M=8, K=2, window=4, dict_cap=16)
    st = apsm.State(gp)
    st.meta.fill_(7)
    apsm.train(gp, torch.empty((0, 8), dtype=torch.complex64, device="cuda"),
               torch.empty((0, 2), dtype=torch.complex64, device="cuda"), st)
    assert st.meta[:3].tolist() == [0, 0, 0]
    soft, _ = apsm.detect(gp, st, torch.ones((3, 8), dtype=torch.complex64, device="cuda"))
    assert torch.count_nonzero(soft) == 0


def test_retraining_a_state_is_deterministic():
    M, K, P = 16, 6, 300
    inst = synth.make_instance(M, K, P, 10, 10.0, instance=42)
    gp = apsm.Params(M=M, K=K, window=16, dict_cap=128)
    st = apsm.State(gp)
    rp, sp = to_dev(inst.rx_pilot), to_dev(inst.sym_pilot)
    apsm.train(gp, rp, sp, st)
    a = [t.clone() for t in (st.dict, st.gamma, st.clin, st.meta)]
    apsm.train(gp, rp, sp, st)
    for x, y in zip(a, (st.dict, st.gamma, st.clin, st.meta)):
        assert torch.equal(x, y)


def test_paper_default_parameters():
    """Sec. V defaults (w_L = w_G = 0.5, W = 20, sigma^2 = 0.05, 16 antennas, 6 users, 685 pilots,
    3840 data vectors; tests/golden/paper_defaults.txt) on synthetic data."""
    M, K, P, N = 16, 6, 685, 3840
    inst = synth.make_instance(M, K, P, N, 15.0, instance=43)
    op = oracle.Params(M=M, K=K, W=20, D=P, sigma=math.sqrt(0.05), mu=0.5, eps=0.01, w_L=0.5)
    gp, st, cl, ref = _train_both(op, inst)
    _compare_training(op, inst, gp, st, cl, ref, tol_coef=1e-4)


@pytest.mark.slow
def test_full_size_16x6_train_and_sampled_detect():
    """The 16-antenna, 6-user workload at full size (1024 pilots, window 16, D = 1024, 65536 data
    vectors) in the launch configuration the benchmark times; detection checked on a sample."""
    M, K, P, N = 16, 6, 1024, 65536
    inst = synth.make_instance(M, K, P, N, 10.0, instance=0)
    op = oracle.Params(M=M, K=K, W=16, D=1024, sigma=0.5, mu=0.5, eps=0.01, w_L=0.5)
    gp, st, cl, ref = _train_both(op, inst)
    fst = ref[0]
    sample = np.random.default_rng(0).choice(N, 2048, replace=False)
    soft, hard = apsm.detect(gp, st, to_dev(inst.rx_data))
    soft = soft.cpu().numpy()[sample]
    ref_soft = oracle.detect(op, fst, inst.rx_data[sample])
    assert_soft_close(soft, ref_soft, what="soft after training")
    assert_hard_match(hard.cpu().numpy()[sample], ref_soft)
    # detection alone from the oracle's own trained filter
    ent = inst.rx_pilot[fst.first_entry:fst.first_entry + fst.n_entries]
    gam = fst.gamma.reshape(-1, 2, K)
    clin = oracle.clin_from_w(M, fst.w)
    st2 = load_state(gp, ent, gam, clin)
    soft2, _ = apsm.detect(gp, st2, to_dev(inst.rx_data))
    ref2 = oracle.detect(op, oracle_state_fp32(M, ent, gam, clin), inst.rx_data[sample])
    assert_soft_close(soft2.cpu().numpy()[sample], ref2)
    ser = float(np.mean(hard.cpu().numpy() != inst.idx_data))
    assert ser < 0.05


# ------------------------------------------------------------------------------------------
# adjoint of detection
# ------------------------------------------------------------------------------------------

BWD_CASES = [
    # M, K, D, N, sigma, w_L
    (4, 2, 60, 300, 0.5, 0.5),
    (16, 6, 200, 1100, 0.5, 0.5),       # several entry CTAs, query slices and a ragged tail
    (8, 3, 33, 70, 0.7, 0.3),
    (32, 12, 100, 257, 0.6, 0.8),
]


@pytest.mark.parametrize("M,K,D,N,sigma,wL", BWD_CASES)
def test_detect_backward_matches_oracle_gradient(M, K, D, N, sigma, wL):
    ent, gam, clin = synth.random_state(M, K, D, instance=D + M)
    inst = synth.make_instance(M, K, 4, N, 10.0, instance=N + K)
    G = (np.random.default_rng(D).standard_normal((N, K)) + 1j * np.random.default_rng(N).standard_normal((N, K)))
    G = G.astype(np.complex64)
    op = oracle.Params(M=M, K=K, W=1, D=D, sigma=sigma, w_L=wL)
    gp = gpu_params(op)
    st = load_state(gp, ent, gam, clin)
    dgamma, dclin, dscal = apsm.detect_backward(gp, st, to_dev(inst.rx_data), to_dev(G))
    ref_g, ref_w, ref_sig, ref_wl = oracle.detect_grad(op, oracle_state_fp32(M, ent, gam, clin), inst.rx_data, G)
    dg = dgamma.cpu().numpy()
    ref_g = ref_g.reshape(D, 2, K)
    assert np.abs(dg[:D] - ref_g).max() <= TOL_FP32 * max(np.abs(ref_g).max(), 1e-30)
    assert np.all(dg[D:] == 0)
    ref_c = oracle.clin_from_w(M, ref_w)
    dc = dclin.cpu().numpy()
    assert np.abs(dc - ref_c).max() <= TOL_FP32 * np.abs(ref_c).max()
    ds = dscal.cpu().numpy()
    assert ds[0] == pytest.approx(ref_sig, rel=1e-3, abs=1e-4 * abs(ref_sig) + 1e-6)
    assert ds[1] == pytest.approx(ref_wl, rel=1e-3, abs=1e-6)


def test_detect_autograd_matches_finite_differences():
    """torch.autograd through the adjoint: gradient of an MSE loss to the transmitted symbols with
    respect to sigma, w_L, the coefficients and the linear filter, against FP64 central finite
    differences of the oracle's detection."""
    M, K, D, N = 8, 3, 40, 200
    ent, gam, clin = synth.random_state(M, K, D, instance=77)
    inst = synth.make_instance(M, K, 4, N, 10.0, instance=78)
    op = oracle.Params(M=M, K=K, W=1, D=D, sigma=0.6, w_L=0.4)
    gp = gpu_params(op)
    st = load_state(gp, ent, gam, clin)
    g_t = st.gamma.clone().requires_grad_(True)
    c_t = st.clin.clone().requires_grad_(True)
    sig = torch.tensor(0.6, dtype=torch.float64, requires_grad=True)
    wl = torch.tensor(0.4, dtype=torch.float64, requires_grad=True)
    target = to_dev(inst.sym_data)
    soft = apsm.detect_autograd(gp, st, to_dev(inst.rx_data), g_t, c_t, sig, wl)
    loss = (soft - target).abs().pow(2).sum()
    loss.backward()

    gam64, clin128 = gam.astype(np.float64), clin.astype(np.complex128)   # the FP32 values, exactly

    def L(sigma=0.6, w_L=0.4, gam_=gam64, clin_=clin128):
        p = oracle.Params(M=M, K=K, W=1, D=D, sigma=sigma, w_L=w_L)
        y = oracle.detect(p, oracle.state_from_arrays(M, ent, gam_, clin_), inst.rx_data)
        return float(np.sum(np.abs(y - inst.sym_data) ** 2))

    h = 1e-5
    assert sig.grad.item() == pytest.approx((L(sigma=0.6 + h) - L(sigma=0.6 - h)) / (2 * h), rel=2e-3)
    assert wl.grad.item() == pytest.approx((L(w_L=0.4 + h) - L(w_L=0.4 - h)) / (2 * h), rel=2e-3)
    rng = np.random.default_rng(1)
    for _ in range(5):
        t, l, k = int(rng.integers(D)), int(rng.integers(2)), int(rng.integers(K))
        gp_, gm_ = gam64.copy(), gam64.copy()
        gp_[t, l, k] += h
        gm_[t, l, k] -= h
        fd = (L(gam_=gp_) - L(gam_=gm_)) / (2 * h)
        assert g_t.grad[t, l, k].item() == pytest.approx(fd, rel=2e-3, abs=1e-4)
    for _ in range(3):
        m, k = int(rng.integers(M)), int(rng.integers(K))
        for unit in (1.0, 1j):
            cp_, cm_ = clin128.copy(), clin128.copy()
            cp_[m, k] += h * unit
            cm_[m, k] -= h * unit
            fd = (L(clin_=cp_) - L(clin_=cm_)) / (2 * h)
            got = c_t.grad[m, k].item()
            assert (got.real if unit == 1.0 else got.imag) == pytest.approx(fd, rel=2e-3, abs=1e-4)


@pytest.mark.parametrize("M,K,P,D,engine", [(64, 4, 300, 300, "ffma"), (16, 6, 300, 256, "ffma"),
                                            (16, 6, 300, 256, "tensor"), (8, 3, 100, 20, "tensor")])
def test_detect_right_behind_training_on_a_fresh_state(M, K, P, D, engine):
    """Detection queued directly behind training on the same stream (no host synchronisation
    between them) on a state that held nothing equals detection after a synchronisation.  The
    FMA engine is launched early and reads the trained state through L2 (its small CTAs can run
    beside the last training CTAs; before those reads bypassed L1 it saw a stale linear filter
    and entry count here); the tensor-core forms start after training has finished."""
    x = synth.make_instance(M, K, P, 500, 10.0, instance=1700 + M + D)
    p = apsm.Params(M=M, K=K, window=16 if D > 20 else 8, dict_cap=D)
    if engine == "ffma":
        apsm.tune_set(M, K, "fp32", "ffma", 64, 2, 1)
    try:
        rp, sp, rd = to_dev(x.rx_pilot), to_dev(x.sym_pilot), to_dev(x.rx_data)
        st = apsm.State(p)
        apsm.train(p, rp, sp, st)
        torch.cuda.synchronize()
        ref, ref_h = apsm.detect(p, st, rd)
        torch.cuda.synchronize()
        for _ in range(4):
            st = apsm.State(p)
            torch.cuda.synchronize()
            apsm.train(p, rp, sp, st)
            soft, hard = apsm.detect(p, st, rd)
            torch.cuda.synchronize()
            assert torch.equal(soft, ref) and torch.equal(hard, ref_h)
    finally:
        apsm.tune_clear()


@pytest.mark.parametrize("balanced", [False, True])
def test_train_detect_host_equals_device_calls(balanced):
    """train_detect_host (host buffers in and out) gives the device path's soft and hard outputs
    bit for bit, in the plain and the balanced detection form."""
    M, K, P, W, D, N = 16, 6, 200, 16, 200, 5000
    inst = synth.make_instance(M, K, P, N, 10.0, instance=77)
    p = apsm.Params(M=M, K=K, window=W, dict_cap=D, sigma=0.5, mu=0.5, eps=0.01, w_L=0.5)
    ws = apsm.detect_workspace(p, N) if balanced else None
    st = apsm.State(p)
    apsm.train(p, to_dev(inst.rx_pilot), to_dev(inst.sym_pilot), st)
    soft_d, hard_d = apsm.detect(p, st, to_dev(inst.rx_data), workspace=ws)
    hp, hs, hd = (torch.from_numpy(a).pin_memory() for a in (inst.rx_pilot, inst.sym_pilot, inst.rx_data))
    soft_h, hard_h = apsm.train_detect_host(p, hp, hs, hd, workspace=ws)
    assert torch.equal(soft_h, soft_d.cpu()) and torch.equal(hard_h, hard_d.cpu())
