"""Host-side checks of the C ABI (no GPU work): the library builds, loads, exports every
function include/apsm.h declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "apsm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:apsm_status|const char|int64_t|void)\s*\**\s*(apsm_\w+)\s*\(", text,
                                 flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2201_05024_gb300 import build, apsm
    build.build()
    return apsm.load_library()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for f in ("apsm_train", "apsm_detect", "apsm_dict_alloc", "apsm_train_workspace_bytes", "apsm_status_string"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_library_is_built_for_sm103a_only():
    from paper_2201_05024_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert not any("sm_90" in a or "sm_100" in a for a in build.ARCH)


def params(**kw):
    from paper_2201_05024_gb300 import apsm
    base = dict(M=16, K=6, window=16, dict_cap=1024)
    base.update(kw)
    return apsm.Params(**base)


def test_dict_alloc_rounds_to_whole_tiles(lib):
    from paper_2201_05024_gb300 import apsm
    assert apsm.dict_alloc(params(dict_cap=1000)) == 1024
    assert apsm.dict_alloc(params(dict_cap=1024)) == 1024
    assert apsm.dict_alloc(params(dict_cap=9, window=16)) == 32


@pytest.mark.parametrize("bad,code", [
    (dict(sigma=0.0), 1), (dict(sigma=-1.0), 1), (dict(mu=0.0), 1), (dict(mu=2.5), 1), (dict(eps=-0.1), 1),
    (dict(w_L=1.5), 1), (dict(window=0), 1), (dict(dict_cap=8, window=16), 1), (dict(K=0), 1),
    (dict(M=3), 2), (dict(M=128), 2), (dict(K=17), 2), (dict(window=129, dict_cap=4096), 2),
    (dict(modulation=3), 1), (dict(modulation=8), 1),
])
def test_parameter_validation(lib, bad, code):
    from paper_2201_05024_gb300 import apsm
    with pytest.raises(apsm.ApsmError) as ei:
        apsm.dict_alloc(params(**bad))
    assert ei.value.code == code


def test_workspace_query(lib):
    from paper_2201_05024_gb300 import apsm
    assert apsm.train_workspace_bytes(params(), 0) == 0
    nb = apsm.train_workspace_bytes(params(), 1024)
    assert nb > 0 and nb % 256 == 0
    assert apsm.train_workspace_bytes(params(), 2048) > nb


def _cstate(ptr=256):
    from paper_2201_05024_gb300 import apsm
    return apsm._CState(ptr, ptr, ptr, ptr, ptr, ptr)


def test_null_pointers_rejected_before_device(lib):
    from paper_2201_05024_gb300 import apsm
    p = params().c()
    st = _cstate(0)
    assert lib.apsm_train(ctypes.byref(p), None, None, 0, None, ctypes.byref(st), None, 0, None, None) == 1
    assert lib.apsm_detect(ctypes.byref(p), ctypes.byref(_cstate()), None, 5, None, None, None) == 1
    assert lib.apsm_detect(ctypes.byref(p), ctypes.byref(_cstate()), None, -1, None, None, None) == 1
    assert lib.apsm_train(ctypes.byref(p), None, None, -3, None, ctypes.byref(_cstate()), None, 0, None, None) == 1
    # too-small workspace
    assert lib.apsm_train(ctypes.byref(p), ctypes.c_void_p(256), ctypes.c_void_p(256), 64, None,
                          ctypes.byref(_cstate()), ctypes.c_void_p(256), 16, None, None) == apsm.APSM_ERR_WORKSPACE
    assert lib.apsm_read_status(None, None, None) == 1
    assert lib.apsm_check_wait_timeout(None, None) == 1


def test_misaligned_arrays_rejected_before_device(lib):
    p = params().c()
    good = _cstate(256)
    from paper_2201_05024_gb300 import apsm
    bad_state = apsm._CState(256 + 8, 256, 256, 256, 256, 256)     # dict only 8-byte aligned
    rc = lib.apsm_detect(ctypes.byref(p), ctypes.byref(bad_state), ctypes.c_void_p(256), 4, ctypes.c_void_p(256),
                         None, None)
    assert rc == apsm.APSM_ERR_INVALID_ARG
    rc = lib.apsm_detect(ctypes.byref(p), ctypes.byref(good), ctypes.c_void_p(256 + 8), 4, ctypes.c_void_p(256),
                         None, None)                          # rx only 8-byte aligned
    assert rc == apsm.APSM_ERR_INVALID_ARG
    nb = apsm.train_workspace_bytes(params(), 64)
    rc = lib.apsm_train(ctypes.byref(p), ctypes.c_void_p(256 + 8), ctypes.c_void_p(256), 64, None, ctypes.byref(good),
                        ctypes.c_void_p(256), nb, None, None)
    assert rc == apsm.APSM_ERR_INVALID_ARG
    rc = lib.apsm_train(ctypes.byref(p), ctypes.c_void_p(256), ctypes.c_void_p(256), 64, None, ctypes.byref(good),
                        ctypes.c_void_p(256 + 64), nb, None, None)   # workspace not 256-byte aligned
    assert rc == apsm.APSM_ERR_INVALID_ARG


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device path")
def test_valid_call_without_a_device_fails_loudly(lib):
    from paper_2201_05024_gb300 import apsm
    p = params().c()
    rc = lib.apsm_detect(ctypes.byref(p), ctypes.byref(_cstate(256)), ctypes.c_void_p(256), 4,
                         ctypes.c_void_p(256), None, None)
    assert rc == apsm.APSM_ERR_CUDA


def test_status_strings(lib):
    from paper_2201_05024_gb300 import apsm
    for c in range(7):
        assert apsm.status_string(c) not in ("", "unknown status")
    assert lib.apsm_launch_count() >= 0


def test_tune_table_validation(lib):
    from paper_2201_05024_gb300 import apsm
    assert lib.apsm_tune_set(16, 6, 0, 1, 64, 2, 1) == 0
    assert lib.apsm_tune_set(16, 6, 0, 0, 0, 0, 0) == 0          # tensor engine ignores the shape
    assert lib.apsm_tune_set(3, 6, 0, 0, 0, 0, 0) == apsm.APSM_ERR_INVALID_ARG
    assert lib.apsm_tune_set(16, 17, 0, 0, 0, 0, 0) == apsm.APSM_ERR_INVALID_ARG
    assert lib.apsm_tune_set(16, 6, 0, 1, 48, 1, 1) == apsm.APSM_ERR_INVALID_ARG
    assert lib.apsm_tune_set(16, 6, 0, 1, 128, 4, 1) == apsm.APSM_ERR_INVALID_ARG
    assert lib.apsm_tune_set(16, 6, 0, 2, 64, 1, 1) == apsm.APSM_ERR_INVALID_ARG
    assert lib.apsm_tune_clear() == 0


def test_batch_create_validates_every_instance_first(lib):
    import ctypes as C
    from paper_2201_05024_gb300 import apsm
    p = params(dict_cap=64).c()
    st = _cstate(256)
    good = apsm._CInstance(p, 64, 10, 256, 256, 256, 256, None, st, 256, 1 << 30)
    bad_ws = apsm._CInstance(p, 64, 10, 256, 256, 256, 256, None, st, 256, 16)
    bad_rx = apsm._CInstance(p, 64, 10, 256, 256, None, 256, None, st, 256, 1 << 30)
    h = C.c_void_p()
    nb = C.c_size_t()
    for bad, code in ((bad_ws, apsm.APSM_ERR_WORKSPACE), (bad_rx, apsm.APSM_ERR_INVALID_ARG)):
        arr = (apsm._CInstance * 2)(good, bad)
        assert lib.apsm_batch_create(arr, 2, 4, C.c_void_p(256), 1 << 20, C.byref(h)) == code
        assert lib.apsm_batch_workspace_bytes(arr, 2, C.byref(nb)) == code
    arr = (apsm._CInstance * 1)(good)
    assert lib.apsm_batch_create(arr, 0, 4, C.c_void_p(256), 1 << 20, C.byref(h)) == apsm.APSM_ERR_INVALID_ARG
    assert lib.apsm_batch_create(arr, 1, 0, C.c_void_p(256), 1 << 20, C.byref(h)) == apsm.APSM_ERR_INVALID_ARG
    # the work lists of the persistent detection need a workspace, 256-byte aligned
    assert lib.apsm_batch_workspace_bytes(arr, 1, C.byref(nb)) == 0 and nb.value > 0
    assert lib.apsm_batch_create(arr, 1, 2, None, 0, C.byref(h)) == apsm.APSM_ERR_WORKSPACE
    assert lib.apsm_batch_create(arr, 1, 2, C.c_void_p(256 + 16), nb.value, C.byref(h)) == apsm.APSM_ERR_INVALID_ARG
    assert lib.apsm_batch_launch(None, None) == apsm.APSM_ERR_INVALID_ARG
    assert lib.apsm_batch_launch_detect(None, None) == apsm.APSM_ERR_INVALID_ARG


def test_parameter_validation_of_weights(lib):
    from paper_2201_05024_gb300 import apsm
    p = params().c()
    p.weights = 2
    out = ctypes.c_int32()
    assert lib.apsm_dict_alloc(ctypes.byref(p), ctypes.byref(out)) == apsm.APSM_ERR_INVALID_ARG
    for ok in (0, 1):
        p.weights = ok
        assert lib.apsm_dict_alloc(ctypes.byref(p), ctypes.byref(out)) == apsm.APSM_OK
    for m in (0, 2, 4, 6):
        assert apsm.dict_alloc(params(modulation=m)) == 1024


def test_state_without_targets_rejected(lib):
    from paper_2201_05024_gb300 import apsm
    p = params().c()
    st = apsm._CState(256, 256, 256, 256, 256, None)
    assert lib.apsm_detect(ctypes.byref(p), ctypes.byref(st), ctypes.c_void_p(256), 4, ctypes.c_void_p(256),
                           None, None) == apsm.APSM_ERR_INVALID_ARG
    st = apsm._CState(256, 256, 256, 256, 256, 256 + 4)        # targets not 8-byte aligned
    assert lib.apsm_detect(ctypes.byref(p), ctypes.byref(st), ctypes.c_void_p(256), 4, ctypes.c_void_p(256),
                           None, None) == apsm.APSM_ERR_INVALID_ARG


def test_continue_validation_before_device(lib):
    from paper_2201_05024_gb300 import apsm
    p = params().c()
    st = _cstate()
    nb = ctypes.c_size_t()
    assert lib.apsm_train_continue_workspace_bytes(ctypes.byref(p), 256, ctypes.byref(nb)) == 0
    assert nb.value >= apsm.train_workspace_bytes(params(), 256)   # room for the carried window
    ws = ctypes.c_void_p(256)
    call = lambda P, n_prev, rx, size: lib.apsm_train_continue(ctypes.byref(p), rx, None, P, n_prev,
                                                               ctypes.byref(st), ws, size, None, None, None, None)
    assert call(64, -1, ctypes.c_void_p(256), nb.value) == apsm.APSM_ERR_INVALID_ARG   # n_prev < 0
    assert call(-1, 0, ctypes.c_void_p(256), nb.value) == apsm.APSM_ERR_INVALID_ARG
    assert call(64, 0, None, nb.value) == apsm.APSM_ERR_INVALID_ARG                    # no vectors
    assert call(64, 100, ctypes.c_void_p(256), 16) == apsm.APSM_ERR_WORKSPACE
    assert call(64, 100, ctypes.c_void_p(256 + 8), nb.value) == apsm.APSM_ERR_INVALID_ARG  # misaligned rx


def test_linear_init_validation_before_device(lib):
    from paper_2201_05024_gb300 import apsm
    p = params().c()
    f = lib.apsm_linear_init
    v = ctypes.c_void_p(256)
    assert f(ctypes.byref(p), v, v, 5, ctypes.c_float(0.1), v, None) == apsm.APSM_ERR_INVALID_ARG      # P < K
    assert f(ctypes.byref(p), v, v, 64, ctypes.c_float(-0.1), v, None) == apsm.APSM_ERR_INVALID_ARG    # N0 < 0
    assert f(ctypes.byref(p), None, v, 64, ctypes.c_float(0.1), v, None) == apsm.APSM_ERR_INVALID_ARG
    q = params(w_L=0.0).c()
    assert f(ctypes.byref(q), v, v, 64, ctypes.c_float(0.1), v, None) == apsm.APSM_ERR_INVALID_ARG      # w_L = 0


def test_set_option_validation(lib):
    from paper_2201_05024_gb300 import apsm
    assert lib.apsm_set_option(0, 64) == apsm.APSM_OK
    assert lib.apsm_set_option(1, 1) == apsm.APSM_OK
    assert lib.apsm_set_option(0, 0) == apsm.APSM_ERR_INVALID_ARG
    assert lib.apsm_set_option(1, 2) == apsm.APSM_ERR_INVALID_ARG
    assert lib.apsm_set_option(7, 1) == apsm.APSM_ERR_INVALID_ARG


def test_train_backward_validation_before_device(lib):
    """apsm_train_backward and its batched and two-call forms reject bad arguments on the host."""
    from paper_2201_05024_gb300 import apsm
    p = params(window=8, dict_cap=256).c()
    vp = ctypes.c_void_p
    one, nb = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.apsm_train_backward_workspace_bytes(ctypes.byref(p), 256, ctypes.byref(one)) == apsm.APSM_OK
    assert lib.apsm_train_backward_batched_workspace_bytes(ctypes.byref(p), 256, 5, ctypes.byref(nb)) == apsm.APSM_OK
    assert one.value > 0 and one.value % 256 == 0 and nb.value == 5 * one.value
    assert lib.apsm_train_backward_batched_workspace_bytes(ctypes.byref(p), 256, 0, ctypes.byref(nb)) == 1
    assert lib.apsm_train_backward_batched_workspace_bytes(ctypes.byref(p), -1, 2, ctypes.byref(nb)) == 1
    assert lib.apsm_train_backward_batched_workspace_bytes(ctypes.byref(p), 256, 2, None) == 1
    a = vp(256)
    ws, big = vp(1 << 20), 1 << 40

    def batched(n, rx=a, sym=a, P=256, dg=a, dc=a, ds=a, d0=a, w=ws, wb=big):
        return lib.apsm_train_backward_batched(ctypes.byref(p), n, rx, sym, P, None, dg, dc, ds, d0, w, wb, None)

    assert batched(0) == apsm.APSM_ERR_INVALID_ARG
    assert batched(70000) == apsm.APSM_ERR_INVALID_ARG
    assert batched(2, rx=None) == apsm.APSM_ERR_INVALID_ARG
    assert batched(2, sym=None) == apsm.APSM_ERR_INVALID_ARG
    assert batched(2, dg=None) == apsm.APSM_ERR_INVALID_ARG
    assert batched(2, d0=None) == apsm.APSM_ERR_INVALID_ARG
    assert batched(2, P=0) == apsm.APSM_ERR_INVALID_ARG
    assert batched(2, P=9000) == apsm.APSM_ERR_UNSUPPORTED
    assert batched(2, wb=nb.value // 5) == apsm.APSM_ERR_WORKSPACE      # room for one instance only
    assert batched(2, w=vp((1 << 20) + 64)) == apsm.APSM_ERR_INVALID_ARG  # not 256-byte aligned
    # the two-call form checks only what each half uses
    assert lib.apsm_train_backward_batched_forward(ctypes.byref(p), 2, a, None, 256, None, ws, big, None) == 1
    assert lib.apsm_train_backward_batched_reverse(ctypes.byref(p), 2, a, 256, None, a, a, a, ws, big, None) == 1
    assert lib.apsm_train_backward_batched_reverse(ctypes.byref(p), 2, a, 256, a, a, a, a, ws, 16, None) == \
        apsm.APSM_ERR_WORKSPACE
    pv = params(window=8, dict_cap=256, weights="violated").c()  # the adjoint covers uniform weights only
    assert lib.apsm_train_backward(ctypes.byref(pv), a, a, 256, None, a, a, a, a, ws, big, None) == \
        apsm.APSM_ERR_UNSUPPORTED
