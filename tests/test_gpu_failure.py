"""Failure detection on the GPU without a fault: a device wait that nothing satisfies runs out
after the library's bounded budget, the kernel records APSM_ERR_TIMEOUT in the state's status
word and returns, the host reads (and clears) it, and the context keeps working."""
import time

import pytest

import oracle
from paper_2201_05024_gb300 import apsm, synth
from parity import assert_hard_match, assert_soft_close, gpu_params, load_state, oracle_state_fp32, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    apsm.load_library()


@pytest.mark.timeout(120)
def test_a_wait_that_runs_out_is_reported_and_the_context_stays_usable():
    M, K, D, N = 16, 6, 100, 257
    op = oracle.Params(M=M, K=K, W=1, D=D, sigma=0.5, w_L=0.5)
    gp = gpu_params(op)
    ent, gam, clin = synth.random_state(M, K, D, instance=41)
    st = load_state(gp, ent, gam, clin)
    assert apsm.read_status(st) == apsm.APSM_OK

    t0 = time.perf_counter()
    apsm.check_wait_timeout(st)
    assert apsm.read_status(st) == apsm.APSM_ERR_TIMEOUT  # synchronises the stream
    waited = time.perf_counter() - t0
    # the budget is 4e9 SM clock cycles: about 2 s at the maximum clock, longer at lower ones
    assert 0.5 < waited < 60.0
    assert apsm.read_status(st) == apsm.APSM_OK  # reading cleared it

    # the same state and context still detect correctly
    inst = synth.make_instance(M, K, 4, N, 10.0, instance=42)
    soft, hard = apsm.detect(gp, st, to_dev(inst.rx_data))
    ref = oracle.detect(op, oracle_state_fp32(M, ent, gam, clin), inst.rx_data)
    assert_soft_close(soft.cpu().numpy(), ref)
    assert_hard_match(hard.cpu().numpy(), ref)
    assert apsm.read_status(st) == apsm.APSM_OK
