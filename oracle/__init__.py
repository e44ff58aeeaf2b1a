"""FP64 CPU oracle of the APSM detector (arXiv 2201.05024, Sec. II) -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The product path (the CUDA library and its binding) never does, and
nothing here is shared with it.

The arithmetic lives in ``apsm_oracle.c`` (plain C, FP64, literal loops); this module
compiles it with gcc, calls it through ctypes and splits independent units (users for
training, queries for detection) over host threads.  The RKHS helpers below are the
brute-force definitions used by the invariant tests.

Parity unpinned: the absolute trained coefficients and error rates at the benchmark
shapes -- the paper prints none; the oracle is pinned by the invariants in
``tests/test_oracle_pins.py`` instead.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "apsm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libapsm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C99, no target-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("K", ctypes.c_int), ("W", ctypes.c_int), ("D", ctypes.c_int),
                ("sigma", ctypes.c_double), ("mu", ctypes.c_double), ("eps", ctypes.c_double),
                ("w_L", ctypes.c_double), ("qam_bits", ctypes.c_int), ("weights", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.apsm_oracle_train.restype = ctypes.c_int
            lib.apsm_oracle_train.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, ctypes.c_int, dp, dp,
                                              dp, ctypes.c_int, ctypes.c_int, dp, dp,
                                              ctypes.POINTER(ctypes.c_int), ctypes.c_void_p, dp,
                                              ctypes.c_void_p, ctypes.c_int, dp, dp]
            lib.apsm_oracle_pam_slice.restype = ctypes.c_double
            lib.apsm_oracle_pam_slice.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            lib.apsm_oracle_eval.restype = None
            lib.apsm_oracle_eval.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, dp, dp, dp,
                                             ctypes.c_int, ctypes.c_int, dp, dp]
            lib.apsm_oracle_detect.restype = None
            lib.apsm_oracle_detect.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, dp, dp, dp,
                                               ctypes.c_int, ctypes.c_int, dp, dp]
            lib.apsm_oracle_detect_grad.restype = None
            lib.apsm_oracle_detect_grad.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, dp, dp, dp, ctypes.c_int,
                                                    ctypes.c_int, dp, dp, dp, dp, dp]
            lib.apsm_oracle_centres.restype = None
            lib.apsm_oracle_centres.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _cplx_to_f64(a):
    """complex [.., M] -> float64 [.., M, 2] (re, im interleaved)."""
    a = np.asarray(a)
    return np.ascontiguousarray(np.stack([a.real, a.imag], axis=-1).astype(np.float64))


@dataclass
class Params:
    M: int
    K: int
    W: int
    D: int
    sigma: float = 0.5
    mu: float = 0.5
    eps: float = 0.01
    w_L: float = 0.5
    qam_bits: int = 2     # Gray square QAM of decided targets: 2 (QPSK), 4 (16-QAM), 6 (64-QAM)
    weights: int = 0      # 0: q_j = 1/|J_n|; 1: q_j = 1/|V_n| on the violated slabs V_n

    def c(self) -> _Params:
        return _Params(self.M, self.K, self.W, self.D, self.sigma, self.mu, self.eps, self.w_L, self.qam_bits,
                       self.weights)


@dataclass
class State:
    """A trained filter: f^k(x) = w_L w_k^T x + w_G sum_i gamma[i][k] kappa_G(centres[i], x)."""
    centres: np.ndarray   # [2n][2M] real-split centres in age order (entry t -> rows 2t, 2t+1)
    gamma: np.ndarray     # [2n][K]
    w: np.ndarray         # [K][2M]
    first_entry: int = 0  # index of the oldest alive pilot
    n_entries: int = 0


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def train(p: Params, rx_pilot, sym_pilot, *, n_steps: int = -1, w0=None, threads: int | None = None,
          log_cases: bool = False, forced=None, decide_from: int | None = None, return_io: bool = False):
    """Run the APSM recurrence (Eq. apsm, Eq. beta) over the vectors; users run on parallel threads.

    decide_from: real-split samples n >= decide_from take the decision Q(f_n(x_n)) as their
    target instead of sym_pilot (decision-directed tracking; sym_pilot may then be None for
    decide_from = 0).  Returns State, then (pred [P][K] complex, target [P][K] complex) when
    return_io -- the filter's output at each vector's arrival and the targets trained on -- then
    (case_log [n][W][K] int8, margin_log [n][W][K]) when log_cases."""
    lib = _load()
    P = int(np.asarray(rx_pilot).shape[0])
    ns = 2 * P if n_steps < 0 else min(int(n_steps), 2 * P)
    rx = _cplx_to_f64(rx_pilot).reshape(P, p.M, 2)
    if sym_pilot is None:
        sym_pilot = np.zeros((P, p.K), np.complex128)
    sy = _cplx_to_f64(sym_pilot).reshape(P, p.K, 2)
    L = 2 * p.M
    w_out = np.zeros((p.K, L))
    g_out = np.zeros((2 * p.D, p.K))
    alive = np.zeros(2, dtype=np.int32)
    w0a = None if w0 is None else _f64(w0).reshape(p.K, L)
    cl = np.full((max(ns, 1), p.W, p.K), 127, dtype=np.int8) if log_cases else None
    ml = np.full((max(ns, 1), p.W, p.K), np.nan) if log_cases else None
    pred = np.zeros((max(P, 1), p.K, 2)) if return_io else None
    tgt = np.zeros((max(P, 1), p.K, 2)) if return_io else None
    dfrom = 2 * P if decide_from is None else int(decide_from)
    fo = None
    if forced is not None:
        fo = np.ascontiguousarray(forced, dtype=np.int8)
        assert fo.shape == (ns, p.W, p.K)
    pc = p.c()
    nt = max(1, min(threads or default_threads(), p.K))
    bounds = np.linspace(0, p.K, nt + 1).astype(int)

    def run(i):
        k0, k1 = int(bounds[i]), int(bounds[i + 1])
        rc = lib.apsm_oracle_train(ctypes.byref(pc), P, ns, _dp(rx), _dp(sy), _dp(w0a), k0, k1, _dp(w_out),
                                   _dp(g_out), alive.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                   cl.ctypes.data if cl is not None else None, _dp(ml),
                                   fo.ctypes.data if fo is not None else None, dfrom, _dp(pred), _dp(tgt))
        if rc != 0:
            raise ValueError("oracle train rejected its arguments")

    if nt == 1:
        run(0)
    else:
        with ThreadPoolExecutor(nt) as ex:
            list(ex.map(run, range(nt)))
    first, n_ent = int(alive[0]), int(alive[1])
    ent = np.asarray(rx_pilot)[first:first + n_ent]
    st = State(centres=centres_from_entries(p.M, ent), gamma=g_out[:2 * n_ent].copy(), w=w_out,
               first_entry=first, n_entries=n_ent)
    out = [st]
    if return_io:
        out.append((pred[:P, :, 0] + 1j * pred[:P, :, 1], tgt[:P, :, 0] + 1j * tgt[:P, :, 1]))
    if log_cases:
        out.extend([cl[:ns], ml[:ns]])
    return out[0] if len(out) == 1 else tuple(out)


def centres_from_entries(M: int, entries) -> np.ndarray:
    """Complex entries [n][M] -> real-split centres [2n][2M] (Sec. II-D)."""
    lib = _load()
    n = int(np.asarray(entries).shape[0])
    e = _cplx_to_f64(entries).reshape(n, M, 2)
    out = np.zeros((2 * n, 2 * M))
    if n:
        lib.apsm_oracle_centres(M, n, _dp(e), _dp(out))
    return out


def _split(n, threads):
    nt = max(1, min(threads, (n + 255) // 256))
    b = np.linspace(0, n, nt + 1).astype(int)
    return [(int(b[i]), int(b[i + 1])) for i in range(nt)]


def eval_real(p: Params, st: State, x, threads: int | None = None) -> np.ndarray:
    """f^k(x) for real-split vectors x [n][2M] -> [n][K]."""
    lib = _load()
    x = _f64(x).reshape(-1, 2 * p.M)
    y = np.zeros((x.shape[0], p.K))
    c, g, w = _f64(st.centres), _f64(st.gamma), _f64(st.w)
    pc = p.c()
    parts = _split(x.shape[0], threads or default_threads())

    def run(r):
        lib.apsm_oracle_eval(ctypes.byref(pc), c.shape[0], _dp(c), _dp(g), _dp(w), r[0], r[1], _dp(x), _dp(y))

    with ThreadPoolExecutor(len(parts)) as ex:
        list(ex.map(run, parts))
    return y


def detect(p: Params, st: State, rx, threads: int | None = None) -> np.ndarray:
    """Complex soft estimates g^k(r) = f^k(r1) + i f^k(r2) for data vectors rx [N][M] -> [N][K]."""
    lib = _load()
    N = int(np.asarray(rx).shape[0])
    r = _cplx_to_f64(rx).reshape(N, p.M, 2)
    y = np.zeros((N, p.K, 2))
    c, g, w = _f64(st.centres), _f64(st.gamma), _f64(st.w)
    pc = p.c()
    parts = _split(N, threads or default_threads())

    def run(rg):
        lib.apsm_oracle_detect(ctypes.byref(pc), c.shape[0], _dp(c), _dp(g), _dp(w), rg[0], rg[1], _dp(r),
                               _dp(y))

    if N:
        with ThreadPoolExecutor(len(parts)) as ex:
            list(ex.map(run, parts))
    return y[..., 0] + 1j * y[..., 1]


def detect_grad(p: Params, st: State, rx, dsoft, threads: int | None = None):
    """Gradient of L = sum Re(conj(dsoft) * soft) = sum dy1 f(r1) + dy2 f(r2) with respect to the
    Gaussian coefficients, the linear coefficients, sigma and w_L (plain partial derivatives,
    FP64).  Returns (dgamma [n_c][K], dw [K][2M], dsigma, dw_L); per-thread partial sums are
    combined in thread order."""
    lib = _load()
    N = int(np.asarray(rx).shape[0])
    r = _cplx_to_f64(rx).reshape(N, p.M, 2)
    dy = _cplx_to_f64(dsoft).reshape(N, p.K, 2)
    c, g, w = _f64(st.centres), _f64(st.gamma), _f64(st.w)
    pc = p.c()
    parts = _split(N, threads or default_threads())
    outs = [(np.zeros((c.shape[0], p.K)), np.zeros((p.K, 2 * p.M)), np.zeros(2)) for _ in parts]

    def run(i):
        rg = parts[i]
        dg, dw, ds = outs[i]
        lib.apsm_oracle_detect_grad(ctypes.byref(pc), c.shape[0], _dp(c), _dp(g), _dp(w), rg[0], rg[1], _dp(r),
                                    _dp(dy), _dp(dg), _dp(dw), _dp(ds))

    if N:
        with ThreadPoolExecutor(len(parts)) as ex:
            list(ex.map(run, range(len(parts))))
    dg = sum(o[0] for o in outs)
    dw = sum(o[1] for o in outs)
    ds = sum(o[2] for o in outs)
    return dg, dw, float(ds[0]), float(ds[1])


def pam_scale(bits: int) -> float:
    """Amplitude unit a of one axis of a unit-energy Gray square QAM with 2^bits points:
    levels (2i - (L-1)) a, L = 2^(bits/2), mean energy 2 a^2 (L^2 - 1)/3 = 1."""
    L = 1 << (bits // 2)
    return float(np.sqrt(3.0 / (2.0 * (L * L - 1))))


def pam_level(y, bits: int) -> np.ndarray:
    """Nearest amplitude level index of one QAM axis: the number of decision boundaries
    (2i - L) a, i = 1..L-1, at or below y (on a boundary: the upper level; exactly 0 counts as
    non-negative)."""
    L = 1 << (bits // 2)
    a = pam_scale(bits)
    y = np.asarray(y, np.float64)
    lev = np.zeros(y.shape, np.int64)
    for b in range(1, L):
        lev += (y >= (2.0 * b - L) * a)
    return lev


def gray_axis(level, bits: int) -> np.ndarray:
    """Gray label of one axis: the level counted from the top (so that a positive amplitude of
    QPSK is bit 0), Gray coded: g = u ^ (u >> 1) with u = L - 1 - level."""
    u = (1 << (bits // 2)) - 1 - np.asarray(level, np.int64)
    return u ^ (u >> 1)


def hard_qam(soft, bits: int = 2) -> np.ndarray:
    """Gray square-QAM decision: label = gray(Re axis) | gray(Im axis) << (bits/2)."""
    soft = np.asarray(soft)
    gi = gray_axis(pam_level(soft.real, bits), bits)
    gq = gray_axis(pam_level(soft.imag, bits), bits)
    return (gi | (gq << (bits // 2))).astype(np.uint8)


def hard_qpsk(soft) -> np.ndarray:
    """Gray QPSK decision: bit0 = (Re < 0), bit1 = (Im < 0); exactly 0 counts as non-negative."""
    return hard_qam(soft, 2)


def pam_slice(y: float, bits: int):
    """The C oracle's slicer (used by its decision-directed targets): (decided value, level)."""
    lev = ctypes.c_int()
    v = _load().apsm_oracle_pam_slice(float(y), int(bits), ctypes.byref(lev))
    return v, lev.value


def linear_filter(rx_pilot, sym_pilot, noise_var: float):
    """Conventional linear detector from the pilots (the linear start of Sec. I / Sec. II-D,
    f_0 = a linear filter): least-squares channel estimate H = Y S^H (S S^H)^-1 from the received
    pilots Y [M][P] and pilot symbols S [K][P], then the MMSE filter W = H (H^H H + N0 I)^-1 (ZF
    for N0 = 0), whose soft estimates are W^H r.  FP64 (numpy solves).  Returns W [M][K]."""
    Y = np.asarray(rx_pilot, np.complex128).T
    S = np.asarray(sym_pilot, np.complex128).T
    H = np.linalg.solve((S @ S.conj().T).T, (Y @ S.conj().T).T).T     # Y S^H (S S^H)^-1
    K = S.shape[0]
    return H @ np.linalg.inv(H.conj().T @ H + noise_var * np.eye(K))


def state_from_arrays(M: int, entries, gamma_entry, clin) -> State:
    """Oracle state from the complex form a detector state is stored in:
    entries [n][M] complex, gamma_entry [n][2][K] (coefficient of centre r1(t), r2(t)),
    clin [M][K] complex linear filter c_k, whose real-split form is w_k = [Re c_k; Im c_k]."""
    entries = np.asarray(entries)
    n = entries.shape[0]
    ge = np.asarray(gamma_entry, dtype=np.float64)
    K = ge.shape[-1] if ge.size else np.asarray(clin).shape[1]
    c = np.asarray(clin)
    w = np.concatenate([c.real.T, c.imag.T], axis=1).astype(np.float64)   # [K][2M]
    return State(centres=centres_from_entries(M, entries), gamma=ge.reshape(2 * n, K), w=w,
                 first_entry=0, n_entries=n)


def clin_from_w(M: int, w) -> np.ndarray:
    """Real-split linear coefficients w [K][2M] -> complex filter c [M][K] = w[:M] + i w[M:]."""
    w = np.asarray(w)
    return (w[:, :M] + 1j * w[:, M:]).T


# ---------------------------------------------------------------------------------------------
# Brute-force RKHS quantities (Sec. II-A/B: Eq. inner_product_definition, Fact 1).
# ---------------------------------------------------------------------------------------------

def gram_gauss(A, B, sigma):
    """Brute-force Gaussian Gram kappa_G(a_i, b_j) by direct differences."""
    A = _f64(A)
    B = _f64(B)
    out = np.empty((A.shape[0], B.shape[0]))
    for i in range(A.shape[0]):
        d = B - A[i]
        out[i] = np.exp(-np.sum(d * d, axis=1) / (2.0 * sigma * sigma))
    return out


def rkhs_inner(p: Params, a: State, b: State, k: int = 0) -> float:
    """<f, g>_H for f, g in the weighted sum space (Fact 1):
    w_L^{-1}<f_L, g_L> + w_G^{-1}<f_G, g_G>, with f_L = w_L <w, .>, f_G = w_G sum gamma_i kappa_G(c_i, .),
    so the sum reduces to w_L <w_f, w_g> + w_G sum_ij gamma_i gamma'_j kappa_G(c_i, c'_j)."""
    wL, wG = p.w_L, 1.0 - p.w_L
    lin = float(np.dot(a.w[k], b.w[k]))
    gs = 0.0
    if a.centres.shape[0] and b.centres.shape[0]:
        G = gram_gauss(a.centres, b.centres, p.sigma)
        gs = float(a.gamma[:, k] @ G @ b.gamma[:, k])
    return wL * lin + wG * gs


def rkhs_diff(a: State, b: State) -> State:
    """a - b as one expansion over the union of both centre lists."""
    return State(centres=np.concatenate([a.centres, b.centres], axis=0),
                 gamma=np.concatenate([a.gamma, -b.gamma], axis=0), w=a.w - b.w)
