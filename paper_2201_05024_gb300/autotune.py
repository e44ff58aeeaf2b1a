"""Autotuner for the detection launch choice per class (antennas M, users K, dtype).

For each class it times the tensor-core engine and a grid of FP32-FMA launch shapes
(query lanes x entry groups x queries per lane) on the current GPU with CUDA events, keeps the
fastest, and writes a JSON table that `apsm.load_tuning` applies (apsm_tune_set).  It runs
offline, never on a timed path.

    python -m paper_2201_05024_gb300.autotune --M 8 16 32 --K 2-12 --out tuning.json
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from . import apsm, synth

FFMA_SHAPES = [(t, s, q) for q in (1, 2) for t in (32, 64, 128) for s in (1, 2, 4) if t * s <= 256]


def _time(fn, reps):
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ts.sort()
    return ts[len(ts) // 2]


def tune_class(M: int, K: int, dtype: str = "fp32", D: int = 1024, N: int = 16384, reps: int = 5):
    p = apsm.Params(M=M, K=K, window=16, dict_cap=D, dtype=dtype)
    ent, gam, clin = synth.random_state(M, K, D, instance=M * 100 + K)
    st = apsm.State(p)
    apsm.state_set(p, st, torch.from_numpy(ent).cuda(), torch.from_numpy(gam).cuda(), torch.from_numpy(clin).cuda())
    rx = torch.from_numpy(synth.make_instance(M, K, 4, N, 10.0, instance=7).rx_data).cuda()
    soft = torch.empty((N, K), dtype=torch.complex64, device="cuda")
    results = []
    apsm.tune_set(M, K, dtype, "tensor")
    try:
        results.append(({"engine": "tensor"}, _time(lambda: apsm.detect(p, st, rx, soft=soft, want_hard=False), reps)))
    except apsm.ApsmError:
        pass
    if dtype == "fp32":
        for t, s, q in FFMA_SHAPES:
            if M > 16 and q == 2:
                continue
            apsm.tune_set(M, K, dtype, "ffma", t, s, q)
            ms = _time(lambda: apsm.detect(p, st, rx, soft=soft, want_hard=False), reps)
            results.append(({"engine": "ffma", "threads": t, "split": s, "qpt": q}, ms))
    best, ms = min(results, key=lambda r: r[1])
    return {"M": M, "K": K, "dtype": dtype, **best, "ms": ms, "D": D, "N": N,
            "candidates": len(results)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--M", type=int, nargs="+", default=[8, 16, 32])
    ap.add_argument("--K", default="2-12")
    ap.add_argument("--dtype", default="fp32")
    ap.add_argument("--D", type=int, default=1024)
    ap.add_argument("--N", type=int, default=16384)
    ap.add_argument("--out", default="apsm_tuning.json")
    args = ap.parse_args()
    lo, hi = (int(v) for v in args.K.split("-")) if "-" in args.K else (int(args.K), int(args.K))
    t0 = time.time()
    classes = [tune_class(M, K, args.dtype, args.D, args.N) for M in args.M for K in range(lo, hi + 1)]
    apsm.tune_clear()
    with open(args.out, "w") as fh:
        json.dump({"gpu": torch.cuda.get_device_name(), "seconds": time.time() - t0, "classes": classes}, fh,
                  indent=1)
    for c in classes:
        print(c)


if __name__ == "__main__":
    main()
