"""Seeded synthetic uplink workloads for the APSM detector.

This module only draws inputs: received vectors and transmitted symbols of the
non-dispersive multiuser uplink of Sec. II-C (Eq. uplink_signal),

    r(t) = sum_k sqrt(p_k) b_k(t) h_k + n(t),

with i.i.d. Rayleigh signatures h_k ~ CN(0, I_M), uniform power p_k = 1,
Gray-coded square QAM symbols (QPSK, 16-QAM or 64-QAM, unit mean energy), a memoryless
cubic power-amplifier model
x -> x + a x |x|^2 applied per user to the transmitted symbol, and AWGN
n(t) ~ CN(0, 10^(-SNR/10) I_M).  One scalar gain per instance (an AGC) scales
pilots and data alike so that the pilot mean of ||r(t)||^2 is 1; the paper
leaves the signal scale open and the Gaussian kernel width only has meaning
relative to it.

It holds none of the detector's arithmetic.  Both the FP64 oracle and the CUDA
path read the complex64 arrays it returns, so the two see identical inputs.
It imports nothing from the rest of the package.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

MASTER_SEED = 20220113
INV_SQRT2 = 1.0 / np.sqrt(2.0)


def _rng(seed: int, instance: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, instance, stream])))


def qam_symbols(index: np.ndarray, bits: int = 2) -> np.ndarray:
    """Gray square QAM with 2^bits points and unit mean energy.  Label bits [0, bits/2) select
    the real axis, the rest the imaginary axis; per axis the Gray code g maps to the amplitude
    level i = L - 1 - u, u the Gray-decoded g, amplitude (2i - (L-1)) a with
    a = sqrt(3 / (2 (L^2 - 1))) (so that for QPSK bit 0 set means a negative real part)."""
    index = np.asarray(index, dtype=np.int64)
    h = bits // 2
    L = 1 << h
    a = np.sqrt(3.0 / (2.0 * (L * L - 1)))

    def axis(g):
        u = g.copy()
        shift = g >> 1
        while np.any(shift):
            u ^= shift
            shift >>= 1
        return (2 * (L - 1 - u) - (L - 1)) * a

    return axis(index & (L - 1)) + 1j * axis((index >> h) & (L - 1))


def qpsk_symbols(index: np.ndarray) -> np.ndarray:
    """Gray QPSK: bit0 selects the sign of the real part, bit1 that of the imaginary part."""
    return qam_symbols(index, 2)


@dataclass
class Instance:
    M: int
    K: int
    rx_pilot: np.ndarray    # [P][M] complex64
    sym_pilot: np.ndarray   # [P][K] complex64  transmitted (pre-PA) pilot symbols = training targets
    rx_data: np.ndarray     # [N][M] complex64
    sym_data: np.ndarray    # [N][K] complex64
    idx_data: np.ndarray    # [N][K] uint8 Gray label of the data symbols
    snr_db: float
    agc_gain: float
    bits: int = 2           # bits per symbol (2 QPSK, 4 16-QAM, 6 64-QAM)


def make_instance(M: int, K: int, P: int, N: int, snr_db: float = 10.0, *,
                  seed: int = MASTER_SEED, instance: int = 0, pa_coef: float = 0.1,
                  agc: bool = True, noiseless: bool = False, bits: int = 2) -> Instance:
    """Draw one detector instance (channel fixed over its pilots and data: block fading).
    bits: 2 (QPSK), 4 (16-QAM) or 6 (64-QAM); for QPSK the cubic PA is a pure gain (unit
    modulus), for the larger constellations it compresses the outer points."""
    if bits not in (2, 4, 6):
        raise ValueError("bits must be 2, 4 or 6")
    g = _rng(seed, instance, 0)
    h = (g.standard_normal((M, K)) + 1j * g.standard_normal((M, K))) * INV_SQRT2
    ip = g.integers(0, 1 << bits, size=(P, K))
    idd = g.integers(0, 1 << bits, size=(N, K))
    sp = qam_symbols(ip, bits)
    sd = qam_symbols(idd, bits)

    def tx(s):
        return s + pa_coef * s * np.abs(s) ** 2

    n0 = 0.0 if noiseless else 10.0 ** (-snr_db / 10.0)
    gn = _rng(seed, instance, 1)
    noise_p = (gn.standard_normal((P, M)) + 1j * gn.standard_normal((P, M))) * np.sqrt(n0 / 2.0)
    noise_d = (gn.standard_normal((N, M)) + 1j * gn.standard_normal((N, M))) * np.sqrt(n0 / 2.0)
    rp = tx(sp) @ h.T + noise_p
    rd = tx(sd) @ h.T + noise_d
    gain = 1.0
    if agc and P > 0:
        gain = 1.0 / np.sqrt(np.mean(np.sum(np.abs(rp) ** 2, axis=1)))
    rp = rp * gain
    rd = rd * gain
    return Instance(M=M, K=K,
                    rx_pilot=np.ascontiguousarray(rp.astype(np.complex64)),
                    sym_pilot=np.ascontiguousarray(sp.astype(np.complex64)),
                    rx_data=np.ascontiguousarray(rd.astype(np.complex64)),
                    sym_data=np.ascontiguousarray(sd.astype(np.complex64)),
                    idx_data=idd.astype(np.uint8), snr_db=float(snr_db), agc_gain=float(gain), bits=bits)


def random_state(M: int, K: int, n_entries: int, *, seed: int = MASTER_SEED, instance: int = 0,
                 gamma_scale: float = 0.5, clin_scale: float = 0.5):
    """A random detector state (dictionary entries, coefficients, linear filter) for detect-only
    workloads.  Entries are unit-mean-energy complex Gaussian vectors like the AGC'd pilots.

    Returns (entries [D][M] complex64, gamma [D][2][K] float32, clin [M][K] complex64)."""
    g = _rng(seed, instance, 2)
    d = (g.standard_normal((n_entries, M)) + 1j * g.standard_normal((n_entries, M))) * np.sqrt(0.5 / max(M, 1))
    gam = g.standard_normal((n_entries, 2, K)) * gamma_scale
    c = (g.standard_normal((M, K)) + 1j * g.standard_normal((M, K))) * clin_scale
    return (np.ascontiguousarray(d.astype(np.complex64)),
            np.ascontiguousarray(gam.astype(np.float32)),
            np.ascontiguousarray(c.astype(np.complex64)))


def batched_shapes(n_instances: int, *, seed: int = MASTER_SEED, M_choices=(8, 16, 32),
                   K_range=(2, 12), D_range=(128, 2048), N_range=(1024, 16384)):
    """Per-instance (M, K, D, N) for the batched workload of uneven detector instances."""
    g = _rng(seed, 0, 3)
    M = g.choice(np.asarray(M_choices), size=n_instances)
    K = g.integers(K_range[0], K_range[1] + 1, size=n_instances)
    D = g.integers(D_range[0], D_range[1] + 1, size=n_instances)
    N = g.integers(N_range[0], N_range[1] + 1, size=n_instances)
    return [dict(M=int(m), K=int(k), D=int(d), N=int(n)) for m, k, d, n in zip(M, K, D, N)]
