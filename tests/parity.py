"""Helpers shared by the GPU parity tests: move states between the oracle's form and the
library's device form, and compare results under the stated tolerances.

Tolerance (FP32 path): an output y agrees with the FP64 value y_ref when
    |y - y_ref| <= tol * max(|y_ref|, rms(y_ref)),   tol = 1e-4,
and a Gray QPSK hard decision must match except where the deciding component of y_ref lies
within tol * rms(y_ref) of zero."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2201_05024_gb300 import apsm

TOL_FP32 = 1e-4


def gpu_params(op: oracle.Params, dtype="fp32") -> apsm.Params:
    return apsm.Params(M=op.M, K=op.K, window=op.W, dict_cap=op.D, sigma=op.sigma, mu=op.mu, eps=op.eps,
                       w_L=op.w_L, dtype=dtype, modulation=op.qam_bits,
                       weights="violated" if op.weights == 1 else "uniform")


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def load_state(gp: apsm.Params, entries, gamma_entry, clin) -> apsm.State:
    st = apsm.State(gp)
    apsm.state_set(gp, st, to_dev(np.asarray(entries, np.complex64)), to_dev(np.asarray(gamma_entry, np.float32)),
                   to_dev(np.asarray(clin, np.complex64)))
    return st


def oracle_state_fp32(M, entries, gamma_entry, clin) -> oracle.State:
    """The oracle's view of exactly the FP32 values handed to the GPU."""
    return oracle.state_from_arrays(M, np.asarray(entries, np.complex64), np.asarray(gamma_entry, np.float32),
                                    np.asarray(clin, np.complex64))


def rel_errors(y, ref):
    y = np.asarray(y, np.complex128)
    ref = np.asarray(ref, np.complex128)
    comps_y = np.stack([y.real, y.imag])
    comps_r = np.stack([ref.real, ref.imag])
    rms = np.sqrt(np.mean(comps_r ** 2)) if comps_r.size else 1.0
    scale = np.maximum(np.abs(comps_r), rms)
    err = np.abs(comps_y - comps_r) / scale
    return err, rms


def assert_soft_close(y, ref, tol=TOL_FP32, what="soft"):
    err, _ = rel_errors(y, ref)
    if err.size:
        worst = float(err.max())
        assert worst <= tol, f"{what}: max scaled error {worst:.3e} > {tol:.1e}"
    return float(err.max()) if err.size else 0.0


def boundary_distance(y, bits=2):
    """Distance of real values y to the nearest decision boundary (2b - L) a of one Gray-QAM axis."""
    L = 1 << (bits // 2)
    a = oracle.pam_scale(bits)
    bnd = np.array([(2 * b - L) * a for b in range(1, L)])
    return np.min(np.abs(np.asarray(y, np.float64)[..., None] - bnd), axis=-1)


def assert_hard_match(hard, ref_soft, tol=TOL_FP32, bits=2):
    """Gray-QAM labels identical except where the FP64 value's deciding component lies within
    tol * rms of a decision boundary."""
    ref_soft = np.asarray(ref_soft)
    ref_hard = oracle.hard_qam(ref_soft, bits)
    hard = np.asarray(hard)
    _, rms = rel_errors(ref_soft, ref_soft)
    near = (boundary_distance(ref_soft.real, bits) < tol * rms) | (boundary_distance(ref_soft.imag, bits) < tol * rms)
    bad = (hard != ref_hard) & ~near
    assert not bad.any(), f"{int(bad.sum())} hard decisions differ away from a decision boundary"


def rms(a):
    a = np.asarray(a, np.float64)
    return float(np.sqrt(np.mean(a ** 2))) if a.size else 0.0
