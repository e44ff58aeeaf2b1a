"""Adjoint of the training recurrence: gradients of an MSE detection loss with respect to sigma,
mu, eps, w_L and the initial linear filter, through training (reverse sweep of the recurrence) and
detection, against FP64 central finite differences of the oracle.  A finite difference is used
only where no branch of Eq. beta flips between the two perturbed runs (the loss has kinks
there); the number of usable checks is asserted."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2201_05024_gb300 import apsm, synth

from parity import to_dev

pytestmark = pytest.mark.gpu

CASES = [
    # M, K, P, W, D, N, sigma, mu, eps, w_L
    (4, 2, 40, 4, 40, 150, 0.6, 0.5, 0.05, 0.5),     # no eviction
    (4, 2, 70, 6, 12, 150, 0.6, 0.7, 0.05, 0.4),     # FIFO eviction
    (8, 3, 33, 3, 33, 120, 0.5, 0.9, 0.02, 0.6),     # (mu = 1 lands residuals exactly on the slab edge)
    (16, 6, 256, 8, 256, 512, 0.5, 0.5, 0.01, 0.5),  # the differentiation-form shape (one warp per user)
    (4, 2, 40, 36, 40, 150, 0.6, 0.5, 0.05, 0.5),    # window above 32 slots: one CTA per user
]


def _loss(op, inst, clin0):
    w0 = np.concatenate([clin0.real.T, clin0.imag.T], axis=1)
    fst, cases, _ = oracle.train(op, inst.rx_pilot, inst.sym_pilot, w0=w0, log_cases=True)
    y = oracle.detect(op, fst, inst.rx_data)
    return float(np.sum(np.abs(y - inst.sym_data) ** 2)), cases


@pytest.mark.parametrize("M,K,P,W,D,N,sigma,mu,eps,wL", CASES)
def test_train_and_detect_gradients_match_finite_differences(M, K, P, W, D, N, sigma, mu, eps, wL):
    inst = synth.make_instance(M, K, P, N, 8.0, instance=900 + P)
    rng = np.random.default_rng(P)
    clin0 = ((rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))) * 0.2).astype(np.complex64)
    p = apsm.Params(M=M, K=K, window=W, dict_cap=D, sigma=sigma, mu=mu, eps=eps, w_L=wL)
    c_t = to_dev(clin0).requires_grad_(True)
    th = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True)
          for k, v in dict(sigma=sigma, mu=mu, eps=eps, w_L=wL).items()}
    soft = apsm.train_detect_autograd(p, to_dev(inst.rx_pilot), to_dev(inst.sym_pilot), to_dev(inst.rx_data), c_t,
                                      th["sigma"], th["mu"], th["eps"], th["w_L"])
    loss = (soft - to_dev(inst.sym_data)).abs().pow(2).sum()
    loss.backward()

    base = dict(sigma=sigma, mu=mu, eps=eps, w_L=wL)
    c64 = clin0.astype(np.complex128)
    scale = max(abs(float(loss.item())), 1.0)
    checked = 0

    def fd(name=None, comp=None):
        h = 1e-6 if name is None else 1e-6 * max(abs(base[name]), 1e-2)
        vals, logs = [], []
        for sgn in (1, -1):
            b = dict(base)
            c = c64.copy()
            if name is not None:
                b[name] += sgn * h
            else:
                c[comp[0], comp[1]] += sgn * h * comp[2]
            op = oracle.Params(M=M, K=K, W=W, D=D, sigma=b["sigma"], mu=b["mu"], eps=b["eps"], w_L=b["w_L"])
            v, cs = _loss(op, inst, c)
            vals.append(v)
            logs.append(cs)
        if not np.array_equal(logs[0], logs[1]):
            return None  # a branch of Eq. beta flips inside the stencil
        return (vals[0] - vals[1]) / (2 * h)

    for name in ("sigma", "mu", "eps", "w_L"):
        ref = fd(name)
        if ref is None:
            continue
        got = th[name].grad.item()
        assert got == pytest.approx(ref, rel=3e-3, abs=1e-5 * scale), name
        checked += 1
    for _ in range(4):
        m, k = int(rng.integers(M)), int(rng.integers(K))
        for unit in (1.0, 1j):
            ref = fd(comp=(m, k, unit))
            if ref is None:
                continue
            g = c_t.grad[m, k].item()
            got = g.real if unit == 1.0 else g.imag
            assert got == pytest.approx(ref, rel=3e-3, abs=1e-5 * scale), (m, k, unit)
            checked += 1
    assert checked >= 8


def test_grad_batch_equals_instances_one_at_a_time():
    """apsm.GradBatch (forward + backward of many instances on parallel streams, optionally one
    CUDA graph): each instance's loss and gradients equal those of the single-stream run bit for
    bit, and match the instance-at-a-time autograd path."""
    M, K, P, W, D, N = 8, 3, 70, 6, 64, 300
    xs = [synth.make_instance(M, K, P, N, 10.0, instance=900 + i) for i in range(6)]
    data = [(to_dev(x.rx_pilot), to_dev(x.sym_pilot), to_dev(x.rx_data), to_dev(x.sym_data)) for x in xs]
    p = apsm.Params(M=M, K=K, window=W, dict_cap=D, sigma=0.6, mu=0.7, eps=0.02, w_L=0.4)
    rng = np.random.default_rng(3)
    c0 = to_dev((0.05 * (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K)))).astype(np.complex64))
    one = apsm.GradBatch(p, data, c0, lanes=1)
    one.run()
    many = apsm.GradBatch(p, data, c0, lanes=4)
    many.run()
    graph = apsm.GradBatch(p, data, c0, lanes=3, graph=True)
    graph.run()
    graph.run()
    torch.cuda.synchronize()
    for b in (many, graph):
        assert torch.equal(b.loss, one.loss) and torch.equal(b.dst, one.dst) and torch.equal(b.dclin0, one.dclin0)
    for i, (rp, sp, rd, sd) in enumerate(data):
        cg = c0.clone().requires_grad_(True)
        th = [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in (p.sigma, p.mu, p.eps, p.w_L)]
        soft = apsm.train_detect_autograd(p, rp, sp, rd, cg, *th)
        (soft - sd).abs().pow(2).sum().backward()
        ref = np.array([float(t.grad) for t in th])
        got = one.dst[i].double().cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max()), (got, ref)
        dc = (one.dclin0[i] - cg.grad).abs().max().item()
        assert dc <= 1e-4 * max(1.0, cg.grad.abs().max().item())


@pytest.mark.parametrize("M,K,P,W,D", [(8, 3, 70, 6, 12), (16, 6, 64, 8, 64), (4, 2, 33, 5, 3), (4, 2, 60, 32, 30),
                                        (4, 2, 60, 40, 21)])
def test_train_backward_batched_equals_single_calls(M, K, P, W, D):
    """apsm_train_backward_batched (one launch per kernel over users x instances) gives each
    instance's gradients bit for bit as its own apsm_train_backward call, and so does the two-call
    form (forward part, then reverse sweep, on one workspace) (FIFO eviction included;
    2D = W + 1 in two cases; W = 32 is the widest window of the warp-per-user form, W = 40 runs the
    CTA-per-user form)."""
    n = 5
    p = apsm.Params(M=M, K=K, window=W, dict_cap=D, sigma=0.6, mu=0.7, eps=0.02, w_L=0.4)
    xs = [synth.make_instance(M, K, P, 16, 10.0, instance=950 + i) for i in range(n)]
    rp = torch.stack([to_dev(x.rx_pilot) for x in xs])
    sp = torch.stack([to_dev(x.sym_pilot) for x in xs])
    g = torch.Generator(device="cpu").manual_seed(5)
    A = apsm.dict_alloc(p)
    dg = (0.1 * torch.randn((n, A, 2, K), generator=g)).cuda()
    dc = (0.1 * torch.randn((n, M, K), dtype=torch.complex64, generator=g)).cuda()
    c0 = (0.05 * torch.randn((n, M, K), dtype=torch.complex64, generator=g)).cuda()
    ds, dc0 = apsm.train_backward_batched(p, rp, sp, dg, dc, clin0=c0)
    nb = ctypes.c_size_t()
    apsm.load_library().apsm_train_backward_batched_workspace_bytes(ctypes.byref(p.c()), P, n, ctypes.byref(nb))
    ws = torch.empty((nb.value,), dtype=torch.uint8, device="cuda")
    apsm.train_backward_batched_forward(p, rp, sp, ws, clin0=c0)  # the two-call form
    ds2, dc02 = apsm.train_backward_batched_reverse(p, rp, dg, dc, ws)
    assert torch.equal(ds2, ds) and torch.equal(dc02, dc0)
    for i in range(n):
        ds1, dc01 = apsm.train_backward(p, rp[i], sp[i], dg[i], dc[i], clin0=c0[i])
        assert torch.equal(ds[i], ds1) and torch.equal(dc0[i], dc01), i


@pytest.mark.parametrize("uneven", ["data", "pilots"])
def test_grad_batch_uneven_instances(uneven):
    """GradBatch with unequal data counts (batched training adjoints, a loss per instance) or
    unequal pilot counts (the per-instance training adjoint): every instance's loss and gradients
    match the instance-at-a-time autograd path."""
    M, K, W, D = 8, 3, 6, 64
    shapes = [(70, 300), (70, 200), (70, 257)] if uneven == "data" else [(70, 300), (50, 300), (33, 300)]
    xs = [synth.make_instance(M, K, P, N, 10.0, instance=960 + i) for i, (P, N) in enumerate(shapes)]
    data = [(to_dev(x.rx_pilot), to_dev(x.sym_pilot), to_dev(x.rx_data), to_dev(x.sym_data)) for x in xs]
    p = apsm.Params(M=M, K=K, window=W, dict_cap=D, sigma=0.6, mu=0.7, eps=0.02, w_L=0.4)
    c0 = torch.zeros((M, K), dtype=torch.complex64, device="cuda")
    gb = apsm.GradBatch(p, data, c0, lanes=2, graph=True)
    assert gb.batched == (uneven == "data") and not gb.batched_loss
    gb.run()
    torch.cuda.synchronize()
    for i, (rp, sp, rd, sd) in enumerate(data):
        cg = c0.clone().requires_grad_(True)
        th = [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in (p.sigma, p.mu, p.eps, p.w_L)]
        soft = apsm.train_detect_autograd(p, rp, sp, rd, cg, *th)
        loss = (soft - sd).abs().pow(2).sum()
        loss.backward()
        lv = float(loss.detach())
        assert abs(float(gb.loss[i]) - lv) <= 1e-5 * max(1.0, abs(lv))
        ref = np.array([float(t.grad) for t in th])
        got = gb.dst[i].double().cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max()), (got, ref)
        assert (gb.dclin0[i] - cg.grad).abs().max().item() <= 1e-4 * max(1.0, cg.grad.abs().max().item())
