"""Batched form: many uneven detector instances trained and detected by one CUDA graph, and the
autotuner's launch table.  Each instance must give exactly what the single-instance calls give,
and a small instance is also checked against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2201_05024_gb300 import apsm, autotune, synth

from parity import assert_hard_match, assert_soft_close, gpu_params, load_state, oracle_state_fp32, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _converter_form():
    """The persistent batched kernel forms its Gram like the converter form of single-instance
    detection; bit-for-bit comparisons run the single-instance calls in that form too (the
    TMA-staged form differs from it by FP32 rounding order only, and is checked against the
    oracle in test_gpu_parity.py)."""
    apsm.set_option("detect_tma", 0)
    yield
    apsm.set_option("detect_tma", 1)

SHAPES = [  # M, K, P, D, N  (P > D: eviction; ragged sizes)
    (8, 2, 300, 128, 1000),
    (16, 6, 200, 512, 3000),
    (32, 12, 150, 160, 2050),
    (16, 5, 700, 333, 777),
    (8, 11, 64, 900, 1500),
    (32, 3, 257, 256, 4096),
]


def _instances():
    out = []
    for i, (M, K, P, D, N) in enumerate(SHAPES):
        inst = synth.make_instance(M, K, P, N, 10.0, instance=500 + i)
        p = apsm.Params(M=M, K=K, window=16, dict_cap=D)
        out.append((p, inst))
    return out


def test_batch_graph_matches_single_instance_calls():
    data = _instances()
    bis = [apsm.BatchInstance(p, to_dev(x.rx_pilot), to_dev(x.sym_pilot), to_dev(x.rx_data)) for p, x in data]
    batch = apsm.Batch(bis, lanes=4)
    for rep in range(2):                       # replay: the same graph on the same buffers
        for b in bis:
            b.soft.zero_()
        batch.launch()
        torch.cuda.synchronize()
        for (p, x), b in zip(data, bis):
            st = apsm.State(p)
            apsm.train(p, b.rx_pilot, b.sym_pilot, st)
            soft, hard = apsm.detect(p, st, b.rx)
            assert torch.equal(soft, b.soft), (p, rep)
            assert torch.equal(hard, b.hard)
            assert torch.equal(st.gamma, b.state.gamma) and torch.equal(st.clin, b.state.clin)
            assert apsm.read_status(b.state) == 0
    batch.close()


def test_batch_small_instance_matches_oracle():
    M, K, P, D, N = 8, 3, 120, 50, 400
    x = synth.make_instance(M, K, P, N, 10.0, instance=600)
    p = apsm.Params(M=M, K=K, window=8, dict_cap=D)
    b = apsm.BatchInstance(p, to_dev(x.rx_pilot), to_dev(x.sym_pilot), to_dev(x.rx_data))
    batch = apsm.Batch([b], lanes=2)
    batch.launch()
    torch.cuda.synchronize()
    op = oracle.Params(M=M, K=K, W=8, D=D, sigma=p.sigma, mu=p.mu, eps=p.eps, w_L=p.w_L)
    ref = oracle.detect(op, oracle.train(op, x.rx_pilot, x.sym_pilot), x.rx_data)
    assert_soft_close(b.soft.cpu().numpy(), ref)
    assert_hard_match(b.hard.cpu().numpy(), ref)
    batch.close()


def test_autotuned_table_keeps_parity():
    M, K = 16, 5
    entry = autotune.tune_class(M, K, "fp32", D=256, N=2048, reps=2)
    assert entry["engine"] in ("tensor", "ffma") and entry["candidates"] > 1
    try:
        apsm.tune_set(M, K, "fp32", entry["engine"], entry.get("threads", 64), entry.get("split", 1),
                      entry.get("qpt", 1))
        ent, gam, clin = synth.random_state(M, K, 300, instance=9)
        inst = synth.make_instance(M, K, 4, 777, 10.0, instance=10)
        op = oracle.Params(M=M, K=K, W=1, D=300)
        gp = gpu_params(op)
        st = load_state(gp, ent, gam, clin)
        soft, hard = apsm.detect(gp, st, to_dev(inst.rx_data))
        ref = oracle.detect(op, oracle_state_fp32(M, ent, gam, clin), inst.rx_data)
        assert_soft_close(soft.cpu().numpy(), ref)
        # every FFMA shape the tuner may pick is itself correct
        for t, s, q in autotune.FFMA_SHAPES:
            apsm.tune_set(M, K, "fp32", "ffma", t, s, q)
            soft, _ = apsm.detect(gp, st, to_dev(inst.rx_data))
            assert_soft_close(soft.cpu().numpy(), ref, what=f"ffma {t}x{s}x{q}")
    finally:
        apsm.tune_clear()


def test_persistent_detection_phase_replays_and_mixes_with_per_instance_detection():
    """The detection phase as one persistent launch per (antennas, user bucket) class: replayed
    alone (its work counters are reset by the graph each time) it gives the same outputs again;
    instances outside the batched kernel's range (64 antennas, BF16, 16-QAM labels) are detected
    per instance on their branch.  Everything equals the single-instance calls bit for bit."""
    shapes = [  # M, K, P, D, N, dtype, bits
        (16, 6, 300, 256, 2000, "fp32", 2), (16, 5, 200, 300, 700, "fp32", 2), (8, 3, 150, 200, 1000, "fp32", 2),
        (64, 4, 100, 100, 300, "fp32", 2), (16, 6, 120, 128, 500, "bf16", 2), (16, 6, 140, 200, 640, "fp32", 4),
    ]
    data = []
    for i, (M, K, P, D, N, dt, bits) in enumerate(shapes):
        x = synth.make_instance(M, K, P, N, 10.0, instance=700 + i, bits=bits)
        p = apsm.Params(M=M, K=K, window=16, dict_cap=D, dtype=dt, modulation=bits)
        data.append((p, x))
    bis = [apsm.BatchInstance(p, to_dev(x.rx_pilot), to_dev(x.sym_pilot), to_dev(x.rx_data)) for p, x in data]
    batch = apsm.Batch(bis, lanes=3)
    n_classes, n_batched = batch.info()
    assert n_classes == 2 and n_batched == 3        # (16, 6) holds two instances, (8, 4) one
    batch.launch()
    torch.cuda.synchronize()
    first = [b.soft.clone() for b in bis]
    for rep in range(2):
        for b in bis:
            b.soft.zero_()
        batch.launch_detect() if rep == 0 else batch.launch()
        torch.cuda.synchronize()
        for (p, x), b, f in zip(data, bis, first):
            if rep == 0 and not (p.dtype == "fp32" and p.M <= 32 and p.modulation == 2):
                continue                            # detected on the training branches only
            assert torch.equal(b.soft, f), (p, rep)
    for (p, x), b in zip(data, bis):
        st = apsm.State(p)
        apsm.train(p, b.rx_pilot, b.sym_pilot, st)
        soft, hard = apsm.detect(p, st, b.rx)
        assert torch.equal(soft, b.soft), p
        assert torch.equal(hard, b.hard), p
        assert apsm.read_status(b.state) == 0
    batch.close()
