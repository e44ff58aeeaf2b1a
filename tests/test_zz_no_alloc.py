"""apsm_train_noalloc: training for callers that cannot allocate device memory (a real-time
receive loop that must not allocate while running, a plug-in whose host framework owns the
device memory).  It must give the same trained filter as apsm_train with a caller-provided
workspace, on consecutive calls that reuse the library's fixed scratch array, and must refuse
training that needs more scratch than that array holds.

This file is collected last so that a run stopping at its first failure has already run every
other test; it also passes when run alone in a fresh process."""
import ctypes
import os
import re

import numpy as np
import pytest
import torch

from paper_2201_05024_gb300 import apsm, synth

from parity import TOL_FP32, assert_soft_close, rms, to_dev

pytestmark = pytest.mark.gpu

_HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "apsm.h")


def _scratch_limit():
    """APSM_NOALLOC_SCRATCH_BYTES as the header defines it."""
    m = re.search(r"#define\s+APSM_NOALLOC_SCRATCH_BYTES\s+\((\d+)u\s*<<\s*(\d+)\)", open(_HEADER).read())
    return int(m.group(1)) << int(m.group(2))


def _noalloc_fn():
    lib = apsm.load_library()
    fn = lib.apsm_train_noalloc
    vp = ctypes.c_void_p
    fn.argtypes = [ctypes.POINTER(apsm._CParams), vp, vp, ctypes.c_int32, vp, ctypes.POINTER(apsm._CState), vp, vp]
    fn.restype = ctypes.c_int
    return fn


def _train_noalloc(gp, rp, sp, st):
    fn = _noalloc_fn()
    cst = st.c()
    return fn(ctypes.byref(gp.c()), ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(sp.data_ptr()),
              int(rp.shape[0]), None, ctypes.byref(cst), None,
              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


CASES = [  # M, K, P, W, D, instance -- two different trainings in a row through the same scratch
    (16, 6, 300, 16, 256, 1),
    (8, 3, 200, 8, 40, 2),
]


def test_noalloc_training_matches_workspace_training_on_consecutive_calls():
    for M, K, P, W, D, seed in CASES:
        inst = synth.make_instance(M, K, P, 500, 10.0, instance=100 + seed)
        gp = apsm.Params(M=M, K=K, window=W, dict_cap=D)
        assert apsm.train_workspace_bytes(gp, P) <= _scratch_limit()
        rp, sp, rd = to_dev(inst.rx_pilot), to_dev(inst.sym_pilot), to_dev(inst.rx_data)
        ref = apsm.train(gp, rp, sp, apsm.State(gp))
        st = apsm.State(gp)
        assert _train_noalloc(gp, rp, sp, st) == apsm.APSM_OK
        torch.cuda.synchronize()
        assert torch.equal(st.meta[:3], ref.meta[:3])
        assert torch.equal(st.dict[:min(P, D)], ref.dict[:min(P, D)])
        g, g_ref = st.gamma.cpu().numpy(), ref.gamma.cpu().numpy()
        assert np.abs(g - g_ref).max() <= TOL_FP32 * rms(g_ref)
        c, c_ref = st.clin.cpu().numpy(), ref.clin.cpu().numpy()
        assert np.abs(c - c_ref).max() <= TOL_FP32 * rms(np.abs(c_ref))
        soft, _ = apsm.detect(gp, st, rd)
        soft_ref, _ = apsm.detect(gp, ref, rd)
        assert_soft_close(soft.cpu().numpy(), soft_ref.cpu().numpy().astype(np.complex128))
        assert apsm.read_status(st) == 0


def test_noalloc_rejects_training_larger_than_its_scratch():
    gp = apsm.Params(M=16, K=6, window=16, dict_cap=1024)
    P = 8192
    assert apsm.train_workspace_bytes(gp, P) > _scratch_limit()
    rp = torch.zeros((P, 16), dtype=torch.complex64, device="cuda")
    sp = torch.zeros((P, 6), dtype=torch.complex64, device="cuda")
    st = apsm.State(gp)
    before = apsm.launch_count()
    assert _train_noalloc(gp, rp, sp, st) == apsm.APSM_ERR_WORKSPACE
    assert apsm.launch_count() == before
