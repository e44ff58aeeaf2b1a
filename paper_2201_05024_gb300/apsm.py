"""Thin Python binding of the C ABI in include/apsm.h (argument marshalling only).

Every step of training and detection runs in the CUDA kernels of libapsm_gb300.so; this
module loads the library with ctypes, allocates caller-owned device memory with torch and
passes raw pointers plus torch's current stream.  There is no fallback: if the library is
missing or the device is not sm_103 the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libapsm_gb300.so")

APSM_OK, APSM_ERR_INVALID_ARG, APSM_ERR_UNSUPPORTED, APSM_ERR_CUDA, APSM_ERR_TIMEOUT, \
    APSM_ERR_NOT_SM103, APSM_ERR_WORKSPACE = range(7)
APSM_FP32, APSM_BF16, APSM_FP16 = 0, 1, 2
_DTYPES = {"fp32": APSM_FP32, "bf16": APSM_BF16, "fp16": APSM_FP16}
APSM_Q_UNIFORM, APSM_Q_VIOLATED = 0, 1
_WEIGHTS = {"uniform": APSM_Q_UNIFORM, "violated": APSM_Q_VIOLATED}
_OPTIONS = {"train_chunk": 0, "train_track": 1, "detect_tma": 2, "half_tc_coef": 3}


class ApsmError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})")


class _CParams(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("K", ctypes.c_int32), ("window", ctypes.c_int32),
                ("dict_cap", ctypes.c_int32), ("sigma", ctypes.c_float), ("mu", ctypes.c_float),
                ("eps", ctypes.c_float), ("w_L", ctypes.c_float), ("dtype", ctypes.c_int32),
                ("modulation", ctypes.c_int32), ("weights", ctypes.c_int32)]


class _CState(ctypes.Structure):
    _fields_ = [("dict", ctypes.c_void_p), ("dict_norm", ctypes.c_void_p), ("gamma", ctypes.c_void_p),
                ("clin", ctypes.c_void_p), ("meta", ctypes.c_void_p), ("target", ctypes.c_void_p)]


class _CInstance(ctypes.Structure):
    _fields_ = [("p", _CParams), ("P", ctypes.c_int32), ("N", ctypes.c_int32), ("rx_pilot", ctypes.c_void_p),
                ("sym_pilot", ctypes.c_void_p), ("rx", ctypes.c_void_p), ("soft", ctypes.c_void_p),
                ("hard", ctypes.c_void_p), ("st", _CState), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t)]


_lib = None
_lock = threading.Lock()


def load_library(path: str | None = None):
    """Load libapsm_gb300.so (built by paper_2201_05024_gb300.build); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} is missing (run paper_2201_05024_gb300.build.build())")
        lib = ctypes.CDLL(p)
        P, S, vp = ctypes.POINTER(_CParams), ctypes.POINTER(_CState), ctypes.c_void_p
        lib.apsm_dict_alloc.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
        lib.apsm_train_workspace_bytes.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]
        lib.apsm_train.argtypes = [P, vp, vp, ctypes.c_int32, vp, S, vp, ctypes.c_size_t, vp, vp]
        lib.apsm_detect.argtypes = [P, S, vp, ctypes.c_int32, vp, vp, vp]
        lib.apsm_detect_ws.argtypes = [P, S, vp, ctypes.c_int32, vp, vp, vp, ctypes.c_size_t, vp]
        lib.apsm_detect_workspace_bytes.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]
        lib.apsm_read_status.argtypes = [S, ctypes.POINTER(ctypes.c_int32), vp]
        lib.apsm_check_wait_timeout.argtypes = [S, vp]
        lib.apsm_state_set.argtypes = [P, vp, vp, vp, vp, ctypes.c_int32, S, vp]
        lib.apsm_train_continue_workspace_bytes.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]
        lib.apsm_train_continue.argtypes = [P, vp, vp, ctypes.c_int32, ctypes.c_int32, S, vp, ctypes.c_size_t, vp, vp,
                                            vp, vp]
        lib.apsm_linear_init.argtypes = [P, vp, vp, ctypes.c_int32, ctypes.c_float, vp, vp]
        lib.apsm_set_option.argtypes = [ctypes.c_int32, ctypes.c_int32]
        lib.apsm_detect_backward_workspace_bytes.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]
        lib.apsm_detect_backward.argtypes = [P, S, vp, ctypes.c_int32, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        i32 = ctypes.c_int32
        lib.apsm_train_backward_workspace_bytes.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]
        lib.apsm_train_backward.argtypes = [P, vp, vp, ctypes.c_int32, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        lib.apsm_train_backward_batched_workspace_bytes.argtypes = [P, i32, i32, ctypes.POINTER(ctypes.c_size_t)]
        lib.apsm_train_backward_batched.argtypes = [P, i32, vp, vp, i32, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        lib.apsm_train_backward_batched_forward.argtypes = [P, i32, vp, vp, i32, vp, vp, ctypes.c_size_t, vp]
        lib.apsm_train_backward_batched_reverse.argtypes = [P, i32, vp, i32, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        lib.apsm_tune_set.argtypes = [i32, i32, i32, i32, i32, i32, i32]
        lib.apsm_tune_clear.argtypes = []
        lib.apsm_batch_workspace_bytes.argtypes = [ctypes.POINTER(_CInstance), i32, ctypes.POINTER(ctypes.c_size_t)]
        lib.apsm_batch_create.argtypes = [ctypes.POINTER(_CInstance), i32, i32, vp, ctypes.c_size_t, ctypes.POINTER(vp)]
        lib.apsm_batch_launch.argtypes = [vp, vp]
        lib.apsm_batch_launch_detect.argtypes = [vp, vp]
        lib.apsm_batch_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        lib.apsm_batch_destroy.argtypes = [vp]
        lib.apsm_status_string.argtypes = [ctypes.c_int]
        lib.apsm_status_string.restype = ctypes.c_char_p
        lib.apsm_launch_count.restype = ctypes.c_int64
        for f in ("apsm_dict_alloc", "apsm_train_workspace_bytes", "apsm_train", "apsm_detect", "apsm_detect_ws",
                  "apsm_detect_workspace_bytes",
                  "apsm_read_status", "apsm_state_set", "apsm_detect_backward_workspace_bytes",
                  "apsm_detect_backward", "apsm_tune_set", "apsm_tune_clear", "apsm_batch_create",
                  "apsm_train_backward_workspace_bytes", "apsm_train_backward",
                  "apsm_train_backward_batched_workspace_bytes", "apsm_train_backward_batched",
                  "apsm_train_backward_batched_forward", "apsm_train_backward_batched_reverse",
                  "apsm_batch_launch", "apsm_batch_destroy", "apsm_check_wait_timeout",
                  "apsm_train_continue_workspace_bytes", "apsm_train_continue", "apsm_linear_init",
                  "apsm_set_option", "apsm_batch_workspace_bytes", "apsm_batch_launch_detect",
                  "apsm_batch_info"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
        return lib


def status_string(code: int) -> str:
    try:
        return load_library().apsm_status_string(code).decode()
    except RuntimeError:
        return "library not loaded"


def _check(code: int, what: str):
    if code != APSM_OK:
        raise ApsmError(code, what)


@dataclass
class Params:
    """APSM parameters (Sec. II-D / Sec. V); w_G = 1 - w_L; sigma is the kernel width."""
    M: int
    K: int
    window: int
    dict_cap: int
    sigma: float = 0.5
    mu: float = 0.5
    eps: float = 0.01
    w_L: float = 0.5
    dtype: str = "fp32"
    modulation: int = 2         # bits per Gray square-QAM symbol: 2 (QPSK), 4 (16-QAM), 6 (64-QAM)
    weights: str = "uniform"    # q_j: "uniform" (1/|J_n|) or "violated" (1/|V_n| on violated slabs)

    def c(self) -> _CParams:
        return _CParams(self.M, self.K, self.window, self.dict_cap, self.sigma, self.mu, self.eps, self.w_L,
                        _DTYPES[self.dtype], self.modulation, _WEIGHTS[self.weights])


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def dict_alloc(p: Params) -> int:
    lib = load_library()
    out = ctypes.c_int32()
    _check(lib.apsm_dict_alloc(ctypes.byref(p.c()), ctypes.byref(out)), "apsm_dict_alloc")
    return out.value


def train_workspace_bytes(p: Params, P: int) -> int:
    lib = load_library()
    out = ctypes.c_size_t()
    _check(lib.apsm_train_workspace_bytes(ctypes.byref(p.c()), int(P), ctypes.byref(out)),
           "apsm_train_workspace_bytes")
    return out.value


class State:
    """Caller-owned device state (include/apsm.h: apsm_state) held as torch tensors."""

    def __init__(self, p: Params, device="cuda"):
        A = dict_alloc(p)
        self.p = p
        self.dict = torch.zeros((A, p.M), dtype=torch.complex64, device=device)
        self.dict_norm = torch.zeros((A,), dtype=torch.float32, device=device)
        self.gamma = torch.zeros((A, 2, p.K), dtype=torch.float32, device=device)
        self.clin = torch.zeros((p.M, p.K), dtype=torch.complex64, device=device)
        self.meta = torch.zeros((4,), dtype=torch.int32, device=device)
        self.target = torch.zeros((A, p.K), dtype=torch.complex64, device=device)
        self.n_vectors = 0   # host mirror of meta[2]: vectors trained on since the state was emptied

    def c(self) -> _CState:
        return _CState(self.dict.data_ptr(), self.dict_norm.data_ptr(), self.gamma.data_ptr(),
                       self.clin.data_ptr(), self.meta.data_ptr(), self.target.data_ptr())

    def entries(self):
        """(entries [n][M], gamma [n][2][K]) in age order (oldest first), copied to the host."""
        size, head = (int(v) for v in self.meta[:2].tolist())
        D = self.p.dict_cap
        order = [(head + i) % D for i in range(size)]
        idx = torch.tensor(order, dtype=torch.long, device=self.dict.device)
        return self.dict[idx].cpu().numpy(), self.gamma[idx].cpu().numpy()


def train(p: Params, rx_pilot: torch.Tensor, sym_pilot: torch.Tensor, state: State, *,
          clin0: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
          case_log: torch.Tensor | None = None) -> State:
    """apsm_train: run the APSM recurrence over the pilots into `state`, from f_0 with linear
    part clin0 ([M][K] complex64, zero when None) and no Gaussian part."""
    lib = load_library()
    P = int(rx_pilot.shape[0])
    _dev(rx_pilot, torch.complex64, (P, p.M), "rx_pilot")
    _dev(sym_pilot, torch.complex64, (P, p.K), "sym_pilot")
    if clin0 is not None:
        _dev(clin0, torch.complex64, (p.M, p.K), "clin0")
    nb = train_workspace_bytes(p, P)
    if workspace is None and nb > 0:
        workspace = torch.empty((nb,), dtype=torch.uint8, device=rx_pilot.device)
    if case_log is not None:
        _dev(case_log, torch.int8, (2 * P, p.window, p.K), "case_log")
    st = state.c()
    _check(lib.apsm_train(ctypes.byref(p.c()), _ptr(rx_pilot), _ptr(sym_pilot), P, _ptr(clin0), ctypes.byref(st),
                          _ptr(workspace), nb if workspace is None else workspace.numel(), _ptr(case_log),
                          _stream()), "apsm_train")
    state.n_vectors = P
    return state


def train_continue_workspace_bytes(p: Params, P: int) -> int:
    lib = load_library()
    out = ctypes.c_size_t()
    _check(lib.apsm_train_continue_workspace_bytes(ctypes.byref(p.c()), int(P), ctypes.byref(out)),
           "apsm_train_continue_workspace_bytes")
    return out.value


def train_continue(p: Params, rx: torch.Tensor, state: State, sym: torch.Tensor | None = None, *,
                   soft: torch.Tensor | None = None, hard: torch.Tensor | None = None, want_outputs: bool = True,
                   workspace: torch.Tensor | None = None, case_log: torch.Tensor | None = None):
    """apsm_train_continue: go on training `state` on the vectors rx [P][M] complex64, with targets
    sym [P][K] (or decided at each vector's arrival when sym is None: decision-directed tracking).
    Returns (soft [P][K] complex64 = the filter's output at each arrival, hard [P][K] uint8 = the
    Gray-QAM labels of the targets) when want_outputs."""
    lib = load_library()
    P = int(rx.shape[0])
    _dev(rx, torch.complex64, (P, p.M), "rx")
    if sym is not None:
        _dev(sym, torch.complex64, (P, p.K), "sym")
    if want_outputs and soft is None:
        soft = torch.empty((P, p.K), dtype=torch.complex64, device=rx.device)
    if want_outputs and hard is None:
        hard = torch.empty((P, p.K), dtype=torch.uint8, device=rx.device)
    if soft is not None:
        _dev(soft, torch.complex64, (P, p.K), "soft")
    if hard is not None:
        _dev(hard, torch.uint8, (P, p.K), "hard")
    if case_log is not None:
        _dev(case_log, torch.int8, (2 * P, p.window, p.K), "case_log")
    nb = train_continue_workspace_bytes(p, P)
    if workspace is None:
        workspace = torch.empty((max(nb, 1),), dtype=torch.uint8, device=rx.device)
    st = state.c()
    _check(lib.apsm_train_continue(ctypes.byref(p.c()), _ptr(rx), _ptr(sym), P, state.n_vectors, ctypes.byref(st),
                                   _ptr(workspace), workspace.numel(), _ptr(soft), _ptr(hard), _ptr(case_log),
                                   _stream()), "apsm_train_continue")
    state.n_vectors += P
    return soft, hard


def linear_init(p: Params, rx_pilot: torch.Tensor, sym_pilot: torch.Tensor, noise_var: float) -> torch.Tensor:
    """apsm_linear_init: clin0 [M][K] complex64 = W / w_L with W the MMSE filter (ZF for noise_var
    0) of the least-squares channel estimate from the pilots; pass it to train(..., clin0=...)."""
    lib = load_library()
    P = int(rx_pilot.shape[0])
    _dev(rx_pilot, torch.complex64, (P, p.M), "rx_pilot")
    _dev(sym_pilot, torch.complex64, (P, p.K), "sym_pilot")
    clin0 = torch.empty((p.M, p.K), dtype=torch.complex64, device=rx_pilot.device)
    _check(lib.apsm_linear_init(ctypes.byref(p.c()), _ptr(rx_pilot), _ptr(sym_pilot), P, float(noise_var),
                                _ptr(clin0), _stream()), "apsm_linear_init")
    return clin0


def set_option(name: str, value: int):
    """apsm_set_option: process-wide launch options ("train_chunk", "train_track", "detect_tma",
    "half_tc_coef")."""
    _check(load_library().apsm_set_option(_OPTIONS[name], int(value)), "apsm_set_option")


def detect_workspace_bytes(p: Params, N: int) -> int:
    """apsm_detect_workspace_bytes: bytes of the balanced detection form's workspace (0: none)."""
    nb = ctypes.c_size_t()
    _check(load_library().apsm_detect_workspace_bytes(ctypes.byref(p.c()), int(N), ctypes.byref(nb)),
           "apsm_detect_workspace_bytes")
    return nb.value


def detect_workspace(p: Params, N: int, device="cuda") -> torch.Tensor | None:
    """A zero-filled workspace for apsm_detect_ws on N vectors (None where the form does not apply)."""
    nb = detect_workspace_bytes(p, N)
    return torch.zeros((nb,), dtype=torch.uint8, device=device) if nb else None


def detect(p: Params, state: State, rx: torch.Tensor, *, soft: torch.Tensor | None = None,
           hard: torch.Tensor | None = None, want_hard: bool = True, workspace: torch.Tensor | None = None):
    """apsm_detect (apsm_detect_ws with a workspace from detect_workspace): soft [N][K] complex64
    estimates and Gray decisions [N][K] uint8."""
    lib = load_library()
    N = int(rx.shape[0])
    _dev(rx, torch.complex64, (N, p.M), "rx")
    if soft is None:
        soft = torch.empty((N, p.K), dtype=torch.complex64, device=rx.device)
    _dev(soft, torch.complex64, (N, p.K), "soft")
    if hard is None and want_hard:
        hard = torch.empty((N, p.K), dtype=torch.uint8, device=rx.device)
    if hard is not None:
        _dev(hard, torch.uint8, (N, p.K), "hard")
    st = state.c()
    if workspace is not None:
        _check(lib.apsm_detect_ws(ctypes.byref(p.c()), ctypes.byref(st), _ptr(rx), N, _ptr(soft), _ptr(hard),
                                  _ptr(workspace), workspace.numel(), _stream()), "apsm_detect_ws")
    else:
        _check(lib.apsm_detect(ctypes.byref(p.c()), ctypes.byref(st), _ptr(rx), N, _ptr(soft), _ptr(hard),
                               _stream()), "apsm_detect")
    return soft, hard


def state_set(p: Params, state: State, entries: torch.Tensor, gamma: torch.Tensor, clin: torch.Tensor,
              target: torch.Tensor | None = None) -> State:
    """apsm_state_set: load entries [n][M] complex64, gamma [n][2][K] float32, clin [M][K]
    complex64 and optionally the entries' targets [n][K] complex64 (device tensors, age order)
    into `state`."""
    lib = load_library()
    n = int(entries.shape[0])
    _dev(entries, torch.complex64, (n, p.M), "entries")
    _dev(gamma, torch.float32, (n, 2, p.K), "gamma")
    _dev(clin, torch.complex64, (p.M, p.K), "clin")
    if target is not None:
        _dev(target, torch.complex64, (n, p.K), "target")
    st = state.c()
    _check(lib.apsm_state_set(ctypes.byref(p.c()), _ptr(entries), _ptr(gamma), _ptr(clin), _ptr(target), n,
                              ctypes.byref(st), _stream()), "apsm_state_set")
    state.n_vectors = n
    return state


def detect_backward(p: Params, state: State, rx: torch.Tensor, dsoft: torch.Tensor, *,
                    workspace: torch.Tensor | None = None):
    """apsm_detect_backward: gradients (dgamma [A][2][K], dclin [M][K] complex64, dsigma, dw_L as a
    [2] float32 tensor) of a loss whose gradient with respect to soft is dsoft."""
    lib = load_library()
    N = int(rx.shape[0])
    _dev(rx, torch.complex64, (N, p.M), "rx")
    _dev(dsoft, torch.complex64, (N, p.K), "dsoft")
    nb = ctypes.c_size_t()
    _check(lib.apsm_detect_backward_workspace_bytes(ctypes.byref(p.c()), N, ctypes.byref(nb)),
           "apsm_detect_backward_workspace_bytes")
    if workspace is None:
        workspace = torch.empty((max(nb.value, 1),), dtype=torch.uint8, device=rx.device)
    dgamma = torch.empty_like(state.gamma)
    dclin = torch.empty_like(state.clin)
    dscal = torch.empty((2,), dtype=torch.float32, device=rx.device)
    st = state.c()
    _check(lib.apsm_detect_backward(ctypes.byref(p.c()), ctypes.byref(st), _ptr(rx), N, _ptr(dsoft), _ptr(dgamma),
                                    _ptr(dclin), _ptr(dscal), _ptr(workspace), workspace.numel(), _stream()),
           "apsm_detect_backward")
    return dgamma, dclin, dscal


class DetectFunction(torch.autograd.Function):
    """soft = detect(gamma, clin, sigma, w_L) with the dictionary entries fixed; backward runs
    apsm_detect_backward.  sigma and w_L are 0-d tensors (their values parametrise the kernels)."""

    @staticmethod
    def forward(ctx, gamma, clin, sigma, w_L, p: Params, state: State, rx):
        q = Params(**{**p.__dict__, "sigma": float(sigma), "w_L": float(w_L)})
        st = State.__new__(State)
        st.p, st.dict, st.dict_norm, st.meta, st.target = q, state.dict, state.dict_norm, state.meta, state.target
        st.n_vectors = state.n_vectors
        st.gamma, st.clin = gamma.detach().contiguous(), clin.detach().contiguous()
        soft, _ = detect(q, st, rx, want_hard=False)
        ctx.q, ctx.st, ctx.rx = q, st, rx
        ctx.sigma_dtype, ctx.wl_dtype = sigma.dtype, w_L.dtype
        return soft

    @staticmethod
    def backward(ctx, dsoft):
        # torch's gradient for a complex output is conj(dL/dz*) convention: dL/dRe + i dL/dIm
        dgamma, dclin, dscal = detect_backward(ctx.q, ctx.st, ctx.rx, dsoft.contiguous())
        ds = dscal.cpu()
        return (dgamma, dclin, ds[0].to(ctx.sigma_dtype), ds[1].to(ctx.wl_dtype), None, None, None)


def detect_autograd(p: Params, state: State, rx: torch.Tensor, gamma: torch.Tensor, clin: torch.Tensor,
                    sigma: torch.Tensor, w_L: torch.Tensor) -> torch.Tensor:
    """Differentiable detection: gradients flow to gamma, clin, sigma and w_L."""
    return DetectFunction.apply(gamma, clin, sigma, w_L, p, state, rx)


def train_backward(p: Params, rx_pilot: torch.Tensor, sym_pilot: torch.Tensor, dgamma: torch.Tensor,
                   dclin: torch.Tensor, *, clin0: torch.Tensor | None = None, workspace: torch.Tensor | None = None):
    """apsm_train_backward: given dL/dgamma [A][2][K] and dL/dclin [M][K] of the trained state, the
    gradients through the training recurrence: ([4] float32 = d sigma, d mu, d eps, d w_L, and
    dL/dclin0 [M][K] complex64)."""
    lib = load_library()
    P = int(rx_pilot.shape[0])
    _dev(rx_pilot, torch.complex64, (P, p.M), "rx_pilot")
    _dev(sym_pilot, torch.complex64, (P, p.K), "sym_pilot")
    _dev(dgamma, torch.float32, (dict_alloc(p), 2, p.K), "dgamma")
    _dev(dclin, torch.complex64, (p.M, p.K), "dclin")
    nb = ctypes.c_size_t()
    _check(lib.apsm_train_backward_workspace_bytes(ctypes.byref(p.c()), P, ctypes.byref(nb)),
           "apsm_train_backward_workspace_bytes")
    if workspace is None:
        workspace = torch.empty((max(nb.value, 1),), dtype=torch.uint8, device=rx_pilot.device)
    dscal = torch.empty((4,), dtype=torch.float32, device=rx_pilot.device)
    dclin0 = torch.empty((p.M, p.K), dtype=torch.complex64, device=rx_pilot.device)
    _check(lib.apsm_train_backward(ctypes.byref(p.c()), _ptr(rx_pilot), _ptr(sym_pilot), P, _ptr(clin0), _ptr(dgamma),
                                   _ptr(dclin), _ptr(dscal), _ptr(dclin0), _ptr(workspace), workspace.numel(),
                                   _stream()), "apsm_train_backward")
    return dscal, dclin0


def train_backward_batched(p: Params, rx_pilot: torch.Tensor, sym_pilot: torch.Tensor, dgamma: torch.Tensor,
                           dclin: torch.Tensor, *, clin0: torch.Tensor | None = None,
                           workspace: torch.Tensor | None = None, dscalars: torch.Tensor | None = None,
                           dclin0: torch.Tensor | None = None):
    """apsm_train_backward_batched: train_backward of n instances in one launch per kernel.
    rx_pilot [n][P][M], sym_pilot [n][P][K], dgamma [n][A][2][K], dclin [n][M][K], clin0 [n][M][K] or
    None; returns (dscalars [n][4], dclin0 [n][M][K]) (written into the given tensors if passed)."""
    lib = load_library()
    n, P = int(rx_pilot.shape[0]), int(rx_pilot.shape[1])
    _dev(rx_pilot, torch.complex64, (n, P, p.M), "rx_pilot")
    _dev(sym_pilot, torch.complex64, (n, P, p.K), "sym_pilot")
    _dev(dgamma, torch.float32, (n, dict_alloc(p), 2, p.K), "dgamma")
    _dev(dclin, torch.complex64, (n, p.M, p.K), "dclin")
    if clin0 is not None:
        _dev(clin0, torch.complex64, (n, p.M, p.K), "clin0")
    nb = ctypes.c_size_t()
    _check(lib.apsm_train_backward_batched_workspace_bytes(ctypes.byref(p.c()), P, n, ctypes.byref(nb)),
           "apsm_train_backward_batched_workspace_bytes")
    if workspace is None:
        workspace = torch.empty((max(nb.value, 1),), dtype=torch.uint8, device=rx_pilot.device)
    if dscalars is None:
        dscalars = torch.empty((n, 4), dtype=torch.float32, device=rx_pilot.device)
    if dclin0 is None:
        dclin0 = torch.empty((n, p.M, p.K), dtype=torch.complex64, device=rx_pilot.device)
    _dev(dscalars, torch.float32, (n, 4), "dscalars")
    _dev(dclin0, torch.complex64, (n, p.M, p.K), "dclin0")
    _check(lib.apsm_train_backward_batched(ctypes.byref(p.c()), n, _ptr(rx_pilot), _ptr(sym_pilot), P, _ptr(clin0),
                                           _ptr(dgamma), _ptr(dclin), _ptr(dscalars), _ptr(dclin0), _ptr(workspace),
                                           workspace.numel(), _stream()), "apsm_train_backward_batched")
    return dscalars, dclin0


def train_backward_batched_forward(p: Params, rx_pilot: torch.Tensor, sym_pilot: torch.Tensor,
                                   workspace: torch.Tensor, *, clin0: torch.Tensor | None = None):
    """apsm_train_backward_batched_forward: the tables and the forward pass of the training
    adjoint of n instances, kept in `workspace` for train_backward_batched_reverse."""
    lib = load_library()
    n, P = int(rx_pilot.shape[0]), int(rx_pilot.shape[1])
    _dev(rx_pilot, torch.complex64, (n, P, p.M), "rx_pilot")
    _dev(sym_pilot, torch.complex64, (n, P, p.K), "sym_pilot")
    if clin0 is not None:
        _dev(clin0, torch.complex64, (n, p.M, p.K), "clin0")
    _check(lib.apsm_train_backward_batched_forward(ctypes.byref(p.c()), n, _ptr(rx_pilot), _ptr(sym_pilot), P,
                                                   _ptr(clin0), _ptr(workspace), workspace.numel(), _stream()),
           "apsm_train_backward_batched_forward")


def train_backward_batched_reverse(p: Params, rx_pilot: torch.Tensor, dgamma: torch.Tensor, dclin: torch.Tensor,
                                   workspace: torch.Tensor, *, dscalars: torch.Tensor | None = None,
                                   dclin0: torch.Tensor | None = None):
    """apsm_train_backward_batched_reverse: the reverse sweep over a workspace filled by
    train_backward_batched_forward; returns (dscalars [n][4], dclin0 [n][M][K])."""
    lib = load_library()
    n, P = int(rx_pilot.shape[0]), int(rx_pilot.shape[1])
    _dev(rx_pilot, torch.complex64, (n, P, p.M), "rx_pilot")
    _dev(dgamma, torch.float32, (n, dict_alloc(p), 2, p.K), "dgamma")
    _dev(dclin, torch.complex64, (n, p.M, p.K), "dclin")
    if dscalars is None:
        dscalars = torch.empty((n, 4), dtype=torch.float32, device=rx_pilot.device)
    if dclin0 is None:
        dclin0 = torch.empty((n, p.M, p.K), dtype=torch.complex64, device=rx_pilot.device)
    _dev(dscalars, torch.float32, (n, 4), "dscalars")
    _dev(dclin0, torch.complex64, (n, p.M, p.K), "dclin0")
    _check(lib.apsm_train_backward_batched_reverse(ctypes.byref(p.c()), n, _ptr(rx_pilot), P, _ptr(dgamma),
                                                   _ptr(dclin), _ptr(dscalars), _ptr(dclin0), _ptr(workspace),
                                                   workspace.numel(), _stream()),
           "apsm_train_backward_batched_reverse")
    return dscalars, dclin0


class TrainDetectFunction(torch.autograd.Function):
    """soft = detect(train(pilots; c_0, sigma, mu, eps, w_L), rx): the APSM recurrence unrolled over
    the pilots and the detection of the data vectors, differentiable with respect to the initial
    linear filter c_0 and the four scalars (0-d tensors)."""

    @staticmethod
    def forward(ctx, clin0, sigma, mu, eps, w_L, p: Params, rx_pilot, sym_pilot, rx):
        q = Params(**{**p.__dict__, "sigma": float(sigma), "mu": float(mu), "eps": float(eps), "w_L": float(w_L)})
        st = State(q, device=rx.device)
        c0 = clin0.detach().contiguous()
        train(q, rx_pilot, sym_pilot, st, clin0=c0)
        soft, _ = detect(q, st, rx, want_hard=False)
        ctx.q, ctx.st, ctx.c0, ctx.data = q, st, c0, (rx_pilot, sym_pilot, rx)
        ctx.dtypes = (sigma.dtype, mu.dtype, eps.dtype, w_L.dtype)
        return soft

    @staticmethod
    def backward(ctx, dsoft):
        rx_pilot, sym_pilot, rx = ctx.data
        dgamma, dclin, dsd = detect_backward(ctx.q, ctx.st, rx, dsoft.contiguous())
        dst, dclin0 = train_backward(ctx.q, rx_pilot, sym_pilot, dgamma, dclin, clin0=ctx.c0)
        dsd, dst = dsd.cpu().double(), dst.cpu().double()
        ds, dm, de, dw = (dsd[0] + dst[0], dst[1], dst[2], dsd[1] + dst[3])
        t = ctx.dtypes
        return (dclin0, ds.to(t[0]), dm.to(t[1]), de.to(t[2]), dw.to(t[3]), None, None, None, None)


def train_detect_autograd(p: Params, rx_pilot, sym_pilot, rx, clin0, sigma, mu, eps, w_L):
    """Differentiable train + detect; gradients flow to clin0, sigma, mu, eps and w_L."""
    return TrainDetectFunction.apply(clin0, sigma, mu, eps, w_L, p, rx_pilot, sym_pilot, rx)


class GradBatch:
    """Batched differentiation form: forward (train from c_0, detect) and backward (loss gradient
    dsoft = 2 (soft - target), apsm_detect_backward, apsm_train_backward) of many independent
    instances with the same parameters, on `lanes` CUDA streams with no host synchronisation
    between instances; with graph=True the whole pass is captured once and replayed as one CUDA
    graph.  When every instance has the same pilot count, the training adjoints run batched over
    chunks of `chunk` instances (default: all of them), each chunk on a stream of its own: the
    forward part (apsm_train_backward_batched_forward, which needs only the pilots) from the
    start, beside the per-instance work, and the reverse sweep as soon as the chunk's detection
    adjoints are done.  Every buffer is allocated here, once.  Per-instance results stay on the device:
    loss [n] (sum |soft - target|^2), dscalars [n][4] (d sigma, d mu, d eps, d w_L) and
    dclin0 [n][M][K]; grads() sums them over the instances in instance order.  Each instance's
    results equal those of the same calls made one instance at a time, bit for bit.
    backward=False: the forward pass alone (soft outputs in buf[i]["soft"])."""

    def __init__(self, p: Params, instances, clin0: torch.Tensor, *, lanes: int = 16, graph: bool = False,
                 backward: bool = True, chunk: int | None = None):
        lib = load_library()
        self.p, self.lanes, self.backward = p, max(1, int(lanes)), backward
        self.inst = [tuple(t.contiguous() for t in x) for x in instances]  # (rx_pilot, sym_pilot, rx, target)
        n = len(self.inst)
        dev = self.inst[0][0].device
        _dev(clin0, torch.complex64, (p.M, p.K), "clin0")
        self.clin0 = clin0
        self.states, self.buf = [], []
        Ps = {int(x[0].shape[0]) for x in self.inst}
        Ns = {int(x[2].shape[0]) for x in self.inst}
        self.batched = backward and len(Ps) == 1
        # equal data counts: one batched loss (soft, dsoft and targets as [n][N][K] arrays)
        self.batched_loss = self.batched and len(Ns) == 1
        if self.batched_loss:
            N0 = next(iter(Ns))
            self.soft_all = torch.empty((n, N0, p.K), dtype=torch.complex64, device=dev)
            self.dsoft_all = torch.empty_like(self.soft_all)
            self.sd_all = torch.empty_like(self.soft_all)
        A = dict_alloc(p)
        self.dgamma = torch.empty((n, A, 2, p.K), dtype=torch.float32, device=dev)
        self.dclin = torch.empty((n, p.M, p.K), dtype=torch.complex64, device=dev)
        self.dsd = torch.empty((n, 2), dtype=torch.float32, device=dev)
        if self.batched:
            P0 = Ps.pop()
            nb_bb = ctypes.c_size_t()
            _check(lib.apsm_train_backward_batched_workspace_bytes(ctypes.byref(p.c()), P0, n, ctypes.byref(nb_bb)),
                   "apsm_train_backward_batched_workspace_bytes")
            self.ws_bb = torch.empty((max(nb_bb.value, 1),), dtype=torch.uint8, device=dev)
            self.ws_per = nb_bb.value // n  # bytes per instance (a multiple of 256)
            self.rxp_all = torch.empty((n, P0, p.M), dtype=torch.complex64, device=dev)
            self.symp_all = torch.empty((n, P0, p.K), dtype=torch.complex64, device=dev)
            self.clin0_all = torch.empty((n, p.M, p.K), dtype=torch.complex64, device=dev)
        for i, (rp, sp, rd, sd) in enumerate(self.inst):
            P, N = int(rp.shape[0]), int(rd.shape[0])
            nb_t, nb_d, nb_b = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
            _check(lib.apsm_train_workspace_bytes(ctypes.byref(p.c()), P, ctypes.byref(nb_t)), "apsm_train_workspace_bytes")
            _check(lib.apsm_detect_backward_workspace_bytes(ctypes.byref(p.c()), N, ctypes.byref(nb_d)),
                   "apsm_detect_backward_workspace_bytes")
            _check(lib.apsm_train_backward_workspace_bytes(ctypes.byref(p.c()), P, ctypes.byref(nb_b)),
                   "apsm_train_backward_workspace_bytes")
            st = State(p, device=dev)
            self.states.append(st)
            self.buf.append(dict(
                ws_t=torch.empty((max(nb_t.value, 1),), dtype=torch.uint8, device=dev),
                ws_d=torch.empty((max(nb_d.value, 1),), dtype=torch.uint8, device=dev),
                ws_b=None if self.batched else torch.empty((max(nb_b.value, 1),), dtype=torch.uint8, device=dev),
                soft=self.soft_all[i] if self.batched_loss else torch.empty((N, p.K), dtype=torch.complex64, device=dev),
                dsoft=self.dsoft_all[i] if self.batched_loss else torch.empty((N, p.K), dtype=torch.complex64,
                                                                              device=dev),
                dgamma=self.dgamma[i], dclin=self.dclin[i], dsd=self.dsd[i]))
        self.loss = torch.zeros((n,), dtype=torch.float32, device=dev)
        self.dst = torch.zeros((n, 4), dtype=torch.float32, device=dev)
        self.dclin0 = torch.zeros((n, p.M, p.K), dtype=torch.complex64, device=dev)
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(self.lanes)]
        cs = max(1, int(chunk)) if chunk else n
        self.chunks = [(c, min(n, c + cs)) for c in range(0, n, cs)] if self.batched else []
        self.bstreams = [torch.cuda.Stream(device=dev) for _ in self.chunks]
        self.graph = None
        if graph:
            self._run()                                  # warm-up outside the capture
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self._run()
            self.graph = g

    def _instance(self, i, part=3):
        """part 1: train and detect; part 2: loss (unless batched), detection adjoint and (unless
        batched) training adjoint; 3: both."""
        lib = load_library()
        p, (rp, sp, rd, sd), st, b = self.p, self.inst[i], self.states[i], self.buf[i]
        P, N = int(rp.shape[0]), int(rd.shape[0])
        c, strm = st.c(), _stream()
        if part & 1:
            _check(lib.apsm_train(ctypes.byref(p.c()), _ptr(rp), _ptr(sp), P, _ptr(self.clin0), ctypes.byref(c),
                                  _ptr(b["ws_t"]), b["ws_t"].numel(), None, strm), "apsm_train")
            _check(lib.apsm_detect(ctypes.byref(p.c()), ctypes.byref(c), _ptr(rd), N, _ptr(b["soft"]), None, strm),
                   "apsm_detect")
        if not self.backward or not part & 2:
            return
        if not self.batched_loss:
            torch.sub(b["soft"], sd, out=b["dsoft"])
            self.loss[i] = b["dsoft"].abs().square().sum()
            b["dsoft"].mul_(2.0)
        _check(lib.apsm_detect_backward(ctypes.byref(p.c()), ctypes.byref(c), _ptr(rd), N, _ptr(b["dsoft"]),
                                        _ptr(b["dgamma"]), _ptr(b["dclin"]), _ptr(b["dsd"]), _ptr(b["ws_d"]),
                                        b["ws_d"].numel(), strm), "apsm_detect_backward")
        if self.batched:
            return
        _check(lib.apsm_train_backward(ctypes.byref(p.c()), _ptr(rp), _ptr(sp), P, _ptr(self.clin0),
                                       _ptr(b["dgamma"]), _ptr(b["dclin"]), _ptr(self.dst[i]), _ptr(self.dclin0[i]),
                                       _ptr(b["ws_b"]), b["ws_b"].numel(), strm), "apsm_train_backward")
        # sigma and w_L also enter through the detection
        self.dst[i, 0] += b["dsd"][0]
        self.dst[i, 3] += b["dsd"][1]

    def _chunk_forward(self, lo, hi):
        """Forward part of the training adjoints of instances lo..hi-1 (on the current stream)."""
        sl = slice(lo, hi)
        torch.stack([x[0] for x in self.inst[sl]], out=self.rxp_all[sl])
        torch.stack([x[1] for x in self.inst[sl]], out=self.symp_all[sl])
        self.clin0_all[sl].copy_(self.clin0.expand_as(self.clin0_all[sl]))
        train_backward_batched_forward(self.p, self.rxp_all[sl], self.symp_all[sl],
                                       self.ws_bb[lo * self.ws_per:hi * self.ws_per], clin0=self.clin0_all[sl])

    def _chunk_reverse(self, lo, hi):
        """Reverse sweep of the training adjoints of instances lo..hi-1 (on the current stream)."""
        sl = slice(lo, hi)
        train_backward_batched_reverse(self.p, self.rxp_all[sl], self.dgamma[sl], self.dclin[sl],
                                       self.ws_bb[lo * self.ws_per:hi * self.ws_per], dscalars=self.dst[sl],
                                       dclin0=self.dclin0[sl])
        self.dst[sl, 0] += self.dsd[sl, 0]  # sigma and w_L also enter through the detection
        self.dst[sl, 3] += self.dsd[sl, 1]

    def _run(self):
        main = torch.cuda.current_stream()
        for s in self.streams + self.bstreams:
            s.wait_stream(main)
        if self.batched:
            for (lo, hi), bs in zip(self.chunks, self.bstreams):
                with torch.cuda.stream(bs):
                    self._chunk_forward(lo, hi)
            if self.batched_loss:  # train and detect everywhere, then one loss for all instances
                torch.stack([x[3] for x in self.inst], out=self.sd_all)
                for i in range(len(self.inst)):
                    with torch.cuda.stream(self.streams[i % self.lanes]):
                        self._instance(i, 1)
                for s in self.streams:
                    main.wait_stream(s)
                torch.sub(self.soft_all, self.sd_all, out=self.dsoft_all)
                self.loss.copy_(self.dsoft_all.abs().square().sum(dim=(1, 2)))
                self.dsoft_all.mul_(2.0)
                for s in self.streams:
                    s.wait_stream(main)
            for (lo, hi), bs in zip(self.chunks, self.bstreams):
                for i in range(lo, hi):
                    with torch.cuda.stream(self.streams[i % self.lanes]):
                        self._instance(i, 2 if self.batched_loss else 3)
                for i in range(lo, hi):
                    bs.wait_stream(self.streams[i % self.lanes])
                with torch.cuda.stream(bs):
                    self._chunk_reverse(lo, hi)
        else:
            for i in range(len(self.inst)):
                with torch.cuda.stream(self.streams[i % self.lanes]):
                    self._instance(i)
        for s in self.streams + self.bstreams:
            main.wait_stream(s)

    def run(self):
        """One forward + backward pass over every instance (no host synchronisation)."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self._run()

    def grads(self):
        """(sum of losses, d sigma, d mu, d eps, d w_L, dclin0 [M][K]) summed in instance order."""
        return self.loss.sum(), self.dst.sum(0), self.dclin0.sum(0)


ENGINES = {"tensor": 0, "ffma": 1}


def tune_set(M: int, K: int, dtype: str, engine: str, threads: int = 64, split: int = 1, qpt: int = 1):
    """apsm_tune_set: the detection launch choice for class (M, K, dtype)."""
    _check(load_library().apsm_tune_set(M, K, _DTYPES[dtype], ENGINES[engine], threads, split, qpt),
           "apsm_tune_set")


def tune_clear():
    _check(load_library().apsm_tune_clear(), "apsm_tune_clear")


def load_tuning(path: str) -> int:
    """Apply a table written by paper_2201_05024_gb300.autotune; returns the number of classes."""
    import json
    with open(path) as fh:
        table = json.load(fh)
    for e in table["classes"]:
        tune_set(e["M"], e["K"], e["dtype"], e["engine"], e.get("threads", 64), e.get("split", 1), e.get("qpt", 1))
    return len(table["classes"])


class BatchInstance:
    """Device buffers of one detector instance of a batch (apsm_instance)."""

    def __init__(self, p: Params, rx_pilot: torch.Tensor, sym_pilot: torch.Tensor, rx: torch.Tensor,
                 want_hard: bool = True):
        P, N = int(rx_pilot.shape[0]), int(rx.shape[0])
        _dev(rx_pilot, torch.complex64, (P, p.M), "rx_pilot")
        _dev(sym_pilot, torch.complex64, (P, p.K), "sym_pilot")
        _dev(rx, torch.complex64, (N, p.M), "rx")
        dev = rx.device
        self.p, self.P, self.N = p, P, N
        self.rx_pilot, self.sym_pilot, self.rx = rx_pilot, sym_pilot, rx
        self.soft = torch.empty((N, p.K), dtype=torch.complex64, device=dev)
        self.hard = torch.empty((N, p.K), dtype=torch.uint8, device=dev) if want_hard else None
        self.state = State(p, device=dev)
        nb = train_workspace_bytes(p, P)
        self.workspace = torch.empty((max(nb, 1),), dtype=torch.uint8, device=dev)

    def c(self) -> _CInstance:
        return _CInstance(self.p.c(), self.P, self.N, self.rx_pilot.data_ptr(), self.sym_pilot.data_ptr(),
                          self.rx.data_ptr(), self.soft.data_ptr(),
                          self.hard.data_ptr() if self.hard is not None else None, self.state.c(),
                          self.workspace.data_ptr(), self.workspace.numel())


class Batch:
    """apsm_batch: train + detect of many uneven instances replayed as one CUDA graph (training on
    parallel branches, detection as one persistent launch per class)."""

    def __init__(self, instances, lanes: int = 16):
        lib = load_library()
        self.instances = list(instances)   # keeps every buffer alive while the graph exists
        arr = (_CInstance * len(self.instances))(*[x.c() for x in self.instances])
        nb = ctypes.c_size_t()
        _check(lib.apsm_batch_workspace_bytes(arr, len(self.instances), ctypes.byref(nb)), "apsm_batch_workspace_bytes")
        dev = self.instances[0].rx.device
        self.workspace = torch.empty((max(nb.value, 1),), dtype=torch.uint8, device=dev)
        h = ctypes.c_void_p()
        _check(lib.apsm_batch_create(arr, len(self.instances), lanes, _ptr(self.workspace), self.workspace.numel(),
                                     ctypes.byref(h)), "apsm_batch_create")
        self._h = h

    def launch(self):
        _check(load_library().apsm_batch_launch(self._h, _stream()), "apsm_batch_launch")

    def launch_detect(self):
        """Replay only the persistent detection phase."""
        _check(load_library().apsm_batch_launch_detect(self._h, _stream()), "apsm_batch_launch_detect")

    def info(self):
        """(classes with a persistent detection launch, instances detected by them)."""
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _check(load_library().apsm_batch_info(self._h, ctypes.byref(a), ctypes.byref(b)), "apsm_batch_info")
        return a.value, b.value

    def close(self):
        if self._h:
            _check(load_library().apsm_batch_destroy(self._h), "apsm_batch_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def read_status(state: State) -> int:
    lib = load_library()
    out = ctypes.c_int32()
    st = state.c()
    _check(lib.apsm_read_status(ctypes.byref(st), ctypes.byref(out), _stream()), "apsm_read_status")
    return out.value


def check_wait_timeout(state: State) -> None:
    """apsm_check_wait_timeout: enqueue the bounded-wait self-check, which leaves APSM_ERR_TIMEOUT
    in the state's status word (read it with read_status) after about two seconds."""
    lib = load_library()
    st = state.c()
    _check(lib.apsm_check_wait_timeout(ctypes.byref(st), _stream()), "apsm_check_wait_timeout")


def launch_count() -> int:
    return int(load_library().apsm_launch_count())


def train_detect_host(p: Params, rx_pilot, sym_pilot, rx_data, *, state: State | None = None,
                      device="cuda", workspace: torch.Tensor | None = None):
    """End-to-end call on HOST tensors: copy pilots, symbols and data vectors to the device,
    train, detect (balanced form with `workspace`, see detect_workspace), and copy the soft and
    hard outputs back.  Host inputs should be pinned for asynchronous copies.  Returns (soft,
    hard) as host tensors."""
    dev = torch.device(device)
    rp = rx_pilot.to(dev, non_blocking=True)
    sp = sym_pilot.to(dev, non_blocking=True)
    rd = rx_data.to(dev, non_blocking=True)
    st = state if state is not None else State(p, device=dev)
    train(p, rp, sp, st)
    soft, hard = detect(p, st, rd, workspace=workspace)
    soft_h = torch.empty(soft.shape, dtype=soft.dtype, pin_memory=True)
    hard_h = torch.empty(hard.shape, dtype=hard.dtype, pin_memory=True)
    soft_h.copy_(soft, non_blocking=True)
    hard_h.copy_(hard, non_blocking=True)
    torch.cuda.current_stream().synchronize()
    return soft_h, hard_h
