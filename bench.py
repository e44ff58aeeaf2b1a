"""Benchmark of the APSM hot path: one step = train on P pilots + detect N data vectors.

Default workload: 16 antennas, 6 QPSK users, 1024 pilots, window 16, dictionary cap 1024,
65536 data vectors, sigma 0.5, mu 0.5, eps 0.01, w_L 0.5, SNR 10 dB (synthetic, seeded).
Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead (bounded sample).

Multi-GPU (torchrun): every rank trains and detects its own independent instance (a different
seed); no data-path collective; value = all ranks' detected vectors / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "APSM symbol-vectors/s detect + pilot updates/s train; % roofline; err vs FP64"
WORKLOAD = dict(M=16, K=6, P=1024, W=16, D=1024, N=65536, sigma=0.5, mu=0.5, eps=0.01, w_L=0.5, snr_db=10.0)
L2_FLUSH_BYTES = 256 << 20
# Peaks (per GPU) for the detection roofline, derived from unit counts and the 2070 MHz maximum
# SM clock: FP32 FMA pipe 152 SM x 128 lanes x 2 flop; MUFU ex2 152 SM x 32 per clock (both
# unit counts confirmed by an FFMA / ex2 throughput microbenchmark on this GPU); TF32 tensor =
# the measured dense BF16 peak x the nominal TF32/BF16 ratio (1.1 / 2.25).
SM_CLOCK_HZ = 2.070e9
FP32_PEAK_TFLOPS = 152 * 128 * 2 * SM_CLOCK_HZ / 1e12
MUFU_PEAK_PER_S = 152 * 32 * SM_CLOCK_HZ
ORACLE_DETECT_SAMPLE = 4096
REFERENCE_DETECT_SAMPLE = 16384

# DRAM bytes per launch of the detection kernel from one ncu capture, valid only for the kernel
# source with this digest (a changed kernel reports null until it is re-captured).
DETECT_TRAFFIC = {"digest": "1308ccdfde91ed53", "bytes_per_launch": 8.63872e6}


def workload_name(w):
    return (f"APSM 16x6 QPSK paper-scale: M={w['M']} K={w['K']} P={w['P']} W={w['W']} D={w['D']} "
            f"N={w['N']} sigma={w['sigma']} mu={w['mu']} eps={w['eps']} w_L={w['w_L']} SNR={w['snr_db']}dB")


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def detect_roofline(w, n_entries, seconds, engine="tf32x3"):
    """Roofline of one detection launch.  Algorithmic work per (query, entry) pair: the complex
    Gram (2M x 2 MACs) -- on the tensor pipe as three TF32 products for FP32 accuracy
    (engine "tf32x3") or one BF16/FP16 product ("half"), or on the FP32 pipe as 4M FMA ("ffma");
    the three exponentials on MUFU; the exponent arguments and the coefficient accumulation
    (4K + 3 FMA) on the FP32 pipe.  The bound is the resource with the largest minimum time; `frac` = that minimum time /
    measured time."""
    pairs = w["N"] * n_entries
    peaks = measured_peaks()
    bf16 = peaks.get("bf16_tflops", 1900.0)
    gram = 2 * (2 * w["M"]) * 2 * pairs
    if engine == "ffma":
        res = {"alu": (2 * (4 * w["M"] + 4 * w["K"] + 3) * pairs, FP32_PEAK_TFLOPS * 1e12, "TFLOP/s")}
    elif engine == "half-tc":
        # both contractions on the tensor pipe: the Gram (one BF16/FP16 product) and the
        # coefficient GEMM (3 exponentials x 2K outputs, G as a BF16 hi + lo pair: 2 products);
        # the FP32 pipe forms the 3 exponent arguments
        res = {"tensor": (gram + 2 * 2 * 3 * (2 * w["K"]) * pairs, bf16 * 1e12, "TFLOP/s"),
               "alu": (2 * 3 * pairs, FP32_PEAK_TFLOPS * 1e12, "TFLOP/s")}
    else:
        tensor = ((3 * gram, bf16 * (1.1 / 2.25) * 1e12, "TFLOP/s") if engine == "tf32x3" else
                  (gram, bf16 * 1e12, "TFLOP/s"))
        res = {"tensor": tensor,
               "alu": (2 * (4 * w["K"] + 3) * pairs, FP32_PEAK_TFLOPS * 1e12, "TFLOP/s")}
    res["mufu"] = (3 * pairs, MUFU_PEAK_PER_S, "Gex2/s")
    tmin = {k: v[0] / v[1] for k, v in res.items()}
    bound = max(tmin, key=tmin.get)
    work, peak, unit = res[bound]
    scale = 1e12 if unit == "TFLOP/s" else 1e9
    others = {k: round(tmin[k] / seconds, 4) for k in res}
    return {"bound": bound, "achieved": work / seconds / scale, "peak": peak / scale, "unit": unit,
            "frac": tmin[bound] / seconds, "frac_by_resource": others,
            "peak_kind": ("FP32 pipe derived (152 SM x 128 FMA x 2070 MHz)" if bound == "alu" else
                          "MUFU derived (152 SM x 32 ex2 x 2070 MHz)" if bound == "mufu" else
                          "TF32 = measured BF16 x nominal 1.1/2.25" if engine == "tf32x3" else
                          "measured BF16 (FP16 taken equal)")}


def code_digest(texts):
    """Digest of CUDA sources with // comments and blank lines removed (a comment edit does not
    change the kernel, so it keeps a traffic capture valid)."""
    h = hashlib.sha256()
    for text in texts:
        for line in text.splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def kernel_digest():
    texts = []
    for f in ("detect_tma.cuh", "detect_tc.cuh", "detect_f32.cuh", "apsm_common.cuh"):
        with open(os.path.join(ROOT, "paper_2201_05024_gb300", "csrc", f)) as fh:
            texts.append(fh.read())
    return code_digest(texts)


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().strip().splitlines() if r.strip()]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[4:8]):
                if v.strip().lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def reduce_max(dist, values, device):
    """Max over ranks of each value: the slowest rank sets the job's time (one rank: unchanged)."""
    if dist is None:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_rate(world, units_per_rank, ms_per_step):
    """Whole-job throughput: every rank processes its own units in the (max-over-ranks) step time."""
    return world * units_per_rank / (ms_per_step / 1e3)


def run_oracle(w, inst, sample, threads=None):
    """Time the FP64 oracle: full training, detection of `sample` queries."""
    import oracle
    op = oracle.Params(M=w["M"], K=w["K"], W=w["W"], D=w["D"], sigma=w["sigma"], mu=w["mu"], eps=w["eps"],
                       w_L=w["w_L"])
    t0 = time.perf_counter()
    st = oracle.train(op, inst.rx_pilot, inst.sym_pilot, threads=threads)
    t1 = time.perf_counter()
    ref = oracle.detect(op, st, inst.rx_data[sample], threads=threads)
    t2 = time.perf_counter()
    return st, ref, t1 - t0, t2 - t1


def oracle_step_rate(w, t_train, t_detect, n_sample):
    step = t_train + t_detect * (w["N"] / n_sample)
    return w["N"] / step, step


def reference_arm(args, w):
    """The FP64 oracle as the reference arm: every step is full training on the workload's pilots
    plus detection of a bounded sample of its data vectors, on all host cores.  The line reports
    what ran (its measured step time and the vectors it detected per second); the rate
    extrapolated to the full data block is given beside it."""
    from paper_2201_05024_gb300 import synth
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    inst = synth.make_instance(w["M"], w["K"], w["P"], w["N"], w["snr_db"], instance=0)
    sample = np.arange(min(REFERENCE_DETECT_SAMPLE, w["N"]))
    cores = oracle.default_threads()
    for _ in range(args.warmup):
        run_oracle(w, inst, sample[:256])
    steps, t_tr, t_de = [], [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, _, tt, td = run_oracle(w, inst, sample)
        steps.append(time.perf_counter() - t0)
        t_tr.append(tt)
        t_de.append(td)
    step = sum(steps) / len(steps)
    value = len(sample) / step
    full_rate, full_step = oracle_step_rate(w, sum(t_tr) / len(t_tr), sum(t_de) / len(t_de), len(sample))
    desc = (f"per step: full FP64 training ({w['P']} pilots, {w['K']} users on {min(cores, w['K'])} threads) + "
            f"detection of {len(sample)} of the {w['N']} data vectors on {cores} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "symbol-vectors/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(w), "parallelism": "host threads",
                   "step": f"train {w['P']} pilots + detect {len(sample)} vectors"},
        "cpu_baseline": {"value": value, "unit": "symbol-vectors/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "extrapolated_full_block": {"value": full_rate, "unit": "symbol-vectors/s", "ms_per_step": full_step * 1e3,
                                    "how": f"training time + detection time x {w['N']}/{len(sample)}"},
        "e2e": {"value": value, "unit": "symbol-vectors/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def snr_sweep(w, snrs=(0.0, 5.0, 10.0, 15.0, 20.0), sample=1024):
    """Error against the FP64 oracle and symbol error rates of both paths at each SNR of the
    16 x 6 workload (full GPU train + detect; oracle training + a detection sample)."""
    import torch
    import oracle
    from paper_2201_05024_gb300 import apsm, synth
    out = []
    gp = apsm.Params(M=w["M"], K=w["K"], window=w["W"], dict_cap=w["D"], sigma=w["sigma"], mu=w["mu"], eps=w["eps"],
                     w_L=w["w_L"])
    op = oracle.Params(M=w["M"], K=w["K"], W=w["W"], D=w["D"], sigma=w["sigma"], mu=w["mu"], eps=w["eps"],
                       w_L=w["w_L"])
    for i, snr in enumerate(snrs):
        inst = synth.make_instance(w["M"], w["K"], w["P"], w["N"], snr, instance=100 + i)
        st = apsm.State(gp)
        apsm.train(gp, torch.from_numpy(inst.rx_pilot).cuda(), torch.from_numpy(inst.sym_pilot).cuda(), st)
        soft, hard = apsm.detect(gp, st, torch.from_numpy(inst.rx_data).cuda())
        idx = np.random.default_rng(i).choice(w["N"], sample, replace=False)
        fst = oracle.train(op, inst.rx_pilot, inst.sym_pilot)
        ref = oracle.detect(op, fst, inst.rx_data[idx])
        y = soft.cpu().numpy()[idx].astype(np.complex128)
        cr, cy = np.stack([ref.real, ref.imag]), np.stack([y.real, y.imag])
        err = np.abs(cy - cr) / np.maximum(np.abs(cr), np.sqrt(np.mean(cr ** 2)))
        out.append({"snr_db": snr, "err_max_scaled": float(err.max()), "err_rms_scaled": float(np.sqrt(np.mean(err ** 2))),
                    "ser_gpu": float(np.mean(hard.cpu().numpy() != inst.idx_data)),
                    "ser_gpu_sample": float(np.mean(hard.cpu().numpy()[idx] != inst.idx_data[idx])),
                    "ser_oracle_sample": float(np.mean(oracle.hard_qpsk(ref) != inst.idx_data[idx]))})
    return out


def run_batched(args):
    """1024 independent detector instances of uneven size (M in {8,16,32}, K in 2..12, D in
    128..2048, P = D pilots, N in 1024..16384 data vectors, W = 16) trained and detected by one
    CUDA graph launch per step."""
    import torch
    from paper_2201_05024_gb300 import apsm, build, synth
    torch.cuda.set_device(0)
    build.build()
    apsm.load_library()
    if args.tuning:
        apsm.load_tuning(args.tuning)
    shapes = synth.batched_shapes(args.instances)
    insts, data = [], []
    t0 = time.perf_counter()
    for i, s in enumerate(shapes):
        x = synth.make_instance(s["M"], s["K"], s["D"], s["N"], 10.0, instance=10000 + i)
        p = apsm.Params(M=s["M"], K=s["K"], window=16, dict_cap=s["D"], sigma=0.5, mu=0.5, eps=0.01, w_L=0.5)
        insts.append(apsm.BatchInstance(p, torch.from_numpy(x.rx_pilot).cuda(), torch.from_numpy(x.sym_pilot).cuda(),
                                        torch.from_numpy(x.rx_data).cuda()))
        data.append((p, x))
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    batch = apsm.Batch(insts, lanes=args.lanes)
    t_graph = time.perf_counter() - t0
    for _ in range(max(args.warmup, 3)):
        batch.launch()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in evs:
        a.record(stream)
        batch.launch()
        b.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    # the detection phase alone (one persistent launch per class), on the trained states
    evd = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in evd:
        a.record(stream)
        batch.launch_detect()
        b.record(stream)
    torch.cuda.synchronize()
    ms_det = sum(a.elapsed_time(b) for a, b in evd) / args.steps
    n_classes, n_batched = batch.info()
    n_vec = sum(s["N"] for s in shapes)
    n_pil = sum(s["D"] * s["K"] for s in shapes)
    pairs = sum(s["N"] * s["D"] for s in shapes)
    bad = [i for i, b in enumerate(insts) if apsm.read_status(b.state) != 0]
    out = {
        "metric": METRIC, "value": n_vec / (ms / 1e3), "unit": "symbol-vectors/s", "n_gpus": 1, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched: {len(shapes)} uneven instances, M in (8,16,32), K 2..12, D 128..2048, "
                               f"P = D, N 1024..16384, W = 16, one CUDA graph per step",
                   "lanes": args.lanes, "tuning": args.tuning or "built-in defaults",
                   "l2": "inputs larger than L2 (%.1f GB of data vectors)" % (n_vec * 8 * 16 / 1e9)},
        "train": {"value": n_pil / (ms / 1e3), "unit": "pilot-updates/s (within the same step)"},
        "pairs_per_s": pairs / (ms / 1e3),
        "detect_phase": {"ms": ms_det, "pairs_per_s": pairs / (ms_det / 1e3), "classes": n_classes,
                         "instances_persistent": n_batched,
                         "roofline": batched_roofline(shapes, ms_det / 1e3)},
        "graph": {"build_s": t_graph, "inputs_s": t_gen},
        "instances_with_status": bad, "clocks": clocks,
    }
    if not args.no_oracle:
        import oracle
        sample = list(range(0, len(shapes), max(1, len(shapes) // 4)))[:4]
        t_cpu, work_s, errs = 0.0, 0.0, []
        for i in sample:
            p, x = data[i]
            op = oracle.Params(M=p.M, K=p.K, W=16, D=p.dict_cap, sigma=p.sigma, mu=p.mu, eps=p.eps, w_L=p.w_L)
            q = np.arange(min(512, x.rx_data.shape[0]))
            t1 = time.perf_counter()
            fst = oracle.train(op, x.rx_pilot, x.sym_pilot)
            ref = oracle.detect(op, fst, x.rx_data[q])
            dt = time.perf_counter() - t1
            t_cpu += dt
            y = insts[i].soft.cpu().numpy()[q].astype(np.complex128)
            cr, cy = np.stack([ref.real, ref.imag]), np.stack([y.real, y.imag])
            errs.append(float((np.abs(cy - cr) / np.maximum(np.abs(cr), np.sqrt(np.mean(cr ** 2)))).max()))
            s = shapes[i]
            work_s += (s["D"] * s["D"] * (4 * s["M"] + 3) * 2 + len(q) * s["D"] * (4 * s["M"] + 4 * s["K"] + 3)) / dt
        rate = work_s / len(sample)  # oracle work units per second
        total_work = sum(s["D"] * s["D"] * (4 * s["M"] + 3) * 2 + s["N"] * s["D"] * (4 * s["M"] + 4 * s["K"] + 3)
                         for s in shapes)
        cpu_step = total_work / rate
        out["cpu_baseline"] = {"value": n_vec / cpu_step, "unit": "symbol-vectors/s", "cores": oracle.default_threads(),
                               "kind": "oracle", "sample": f"instances {sample}: full training + 512 detected vectors "
                                                           f"each ({t_cpu:.1f} s), extrapolated by pair work"}
        out["err_vs_fp64"] = {"max_scaled": max(errs), "instances": sample}
    print(json.dumps(out))


def batched_roofline(shapes, seconds):
    """Roofline of the persistent detection phase over uneven instances: per resource the summed
    algorithmic work of every instance (as in detect_roofline, TF32 x3 Gram), against one peak."""
    peaks = measured_peaks()
    bf16 = peaks.get("bf16_tflops", 1900.0)
    tensor = alu = mufu = 0.0
    for s in shapes:
        pairs = s["N"] * s["D"]
        tensor += 3 * 2 * (2 * s["M"]) * 2 * pairs
        alu += 2 * (4 * s["K"] + 3) * pairs
        mufu += 3 * pairs
    res = {"tensor": (tensor, bf16 * (1.1 / 2.25) * 1e12, "TFLOP/s"), "alu": (alu, FP32_PEAK_TFLOPS * 1e12, "TFLOP/s"),
           "mufu": (mufu, MUFU_PEAK_PER_S, "Gex2/s")}
    tmin = {k: v[0] / v[1] for k, v in res.items()}
    bound = max(tmin, key=tmin.get)
    work, peak, unit = res[bound]
    scale = 1e12 if unit == "TFLOP/s" else 1e9
    return {"bound": bound, "achieved": work / seconds / scale, "peak": peak / scale, "unit": unit,
            "frac": tmin[bound] / seconds, "frac_by_resource": {k: round(v / seconds, 4) for k, v in tmin.items()}}


def _time_events(fn, steps, warmup):
    import torch
    for _ in range(max(warmup, 3)):
        fn()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / steps


def run_precision(args):
    """Detection only, 64 antennas, 16 users, D = 4096 entries, 1,048,576 data vectors, Gram in
    BF16 (and FP16) on the tensor cores with FP32 accumulation; coefficients trained by the FP32
    GPU trainer on 4096 pilots (W = 16).  Errors against the FP64 oracle (sampled) and the FP32
    GPU path."""
    import torch
    from paper_2201_05024_gb300 import apsm, build, synth
    import oracle
    torch.cuda.set_device(0)
    build.build()
    M, K, D, N = 64, 16, 4096, args.precision_n
    x = synth.make_instance(M, K, D, N, 15.0, instance=4)
    base = dict(M=M, K=K, window=16, dict_cap=D, sigma=0.5, mu=0.5, eps=0.01, w_L=0.5)
    p32 = apsm.Params(**base)
    st = apsm.State(p32)
    rp, sp = torch.from_numpy(x.rx_pilot).cuda(), torch.from_numpy(x.sym_pilot).cuda()
    apsm.train(p32, rp, sp, st)
    rd = torch.from_numpy(x.rx_data).cuda()
    out = {"metric": METRIC, "unit": "symbol-vectors/s", "n_gpus": 1, "steps": args.steps,
           "warmup": max(args.warmup, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "data": "synthetic", "config": {"workload": f"detect-only M={M} K={K} D={D} N={N}, state trained "
                                                       "by the FP32 GPU trainer on 4096 pilots (W=16)",
                                           "l2": "inputs larger than L2 (%d MB of data vectors)" % (N * M * 8 >> 20)}}
    soft = {}
    for dt in ("fp32", "bf16", "fp16"):
        q = apsm.Params(**base, dtype=dt)
        s_ = torch.empty((N, K), dtype=torch.complex64, device="cuda")
        h_ = torch.empty((N, K), dtype=torch.uint8, device="cuda")
        dw = apsm.detect_workspace(q, N)
        ms = _time_events(lambda: apsm.detect(q, st, rd, soft=s_, hard=h_, workspace=dw), args.steps, args.warmup)
        soft[dt] = s_
        pairs = N * D
        # FP32 has no tensor-core kernel above 32 antennas (its TF32 hi/lo operands would not fit
        # shared memory), so it runs on the FMA engine here; BF16/FP16 form the Gram and the
        # coefficient sums on the tensor cores.
        engine = "half-tc" if dt != "fp32" else ("ffma" if M > 32 else "tf32x3")
        out[dt] = {"value": N / (ms / 1e3), "ms": ms, "pairs_per_s": pairs / (ms / 1e3), "engine": engine,
                   "roofline": detect_roofline(dict(M=M, K=K, N=N), D, ms / 1e3, engine),
                   "ser": float((h_.cpu().numpy() != x.idx_data).mean())}
    out["value"], out["ms_per_step"], out["dtype"] = out["bf16"]["value"], out["bf16"]["ms"], "bf16"
    out["roofline"] = {"kernel": "detect_tcc_kernel<64,16> (BF16 Gram and coefficient GEMM)", **out["bf16"]["roofline"],
                       "traffic": None}
    sample = np.random.default_rng(0).choice(N, 512, replace=False)
    ent, gam = st.entries()
    op = oracle.Params(M=M, K=K, W=16, D=D, sigma=0.5, w_L=0.5)
    ost = oracle.state_from_arrays(M, ent, gam, st.clin.cpu().numpy())
    ref = oracle.detect(op, ost, x.rx_data[sample])
    cr = np.stack([ref.real, ref.imag])
    rms = np.sqrt(np.mean(cr ** 2))
    for dt in ("fp32", "bf16", "fp16"):
        y = soft[dt].cpu().numpy()[sample].astype(np.complex128)
        cy = np.stack([y.real, y.imag])
        out[dt]["err_vs_fp64_max_scaled"] = float((np.abs(cy - cr) / np.maximum(np.abs(cr), rms)).max())
        if dt != "fp32":
            y32 = soft["fp32"].cpu().numpy().astype(np.complex128)
            yd = soft[dt].cpu().numpy().astype(np.complex128)
            c32, cd = np.stack([y32.real, y32.imag]), np.stack([yd.real, yd.imag])
            r32 = np.sqrt(np.mean(c32 ** 2))
            out[dt]["err_vs_fp32_max_scaled"] = float((np.abs(cd - c32) / np.maximum(np.abs(c32), r32)).max())
    print(json.dumps(out))


def run_grad(args):
    """Differentiation form: 256 instances of 16 antennas, 6 users, 256 pilots (W = 8, D = 256),
    4096 data vectors each; loss = sum |soft - transmitted symbol|^2; forward (train + detect) and
    backward (loss gradient, detect adjoint, training adjoint) of all instances as one CUDA graph
    (apsm.GradBatch: per-instance work over 64 streams, the training adjoints of all instances in
    one batched launch), against the forward alone batched the same way and against the
    instance-at-a-time autograd path on a sample."""
    import torch
    from paper_2201_05024_gb300 import apsm, build, synth
    torch.cuda.set_device(0)
    build.build()
    n_inst, M, K, P, W, D, N = args.grad_instances, 16, 6, 256, 8, 256, 4096
    p = apsm.Params(M=M, K=K, window=W, dict_cap=D, sigma=0.5, mu=0.5, eps=0.01, w_L=0.5)
    data = []
    for i in range(n_inst):
        x = synth.make_instance(M, K, P, N, 10.0, instance=20000 + i)
        data.append(tuple(torch.from_numpy(a).cuda() for a in (x.rx_pilot, x.sym_pilot, x.rx_data, x.sym_data)))
    c0 = torch.zeros((M, K), dtype=torch.complex64, device="cuda")
    fb = apsm.GradBatch(p, data, c0, lanes=64, graph=True)
    fo = apsm.GradBatch(p, data, c0, lanes=64, graph=True, backward=False)
    ms = _time_events(fb.run, args.steps, args.warmup)
    fwd = _time_events(fo.run, args.steps, args.warmup)
    loss, dscal, dclin0 = fb.grads()
    # the instance-at-a-time autograd path on a sample of instances (host synchronisation each)
    n_s = min(8, n_inst)
    cg = torch.zeros((M, K), dtype=torch.complex64, device="cuda", requires_grad=True)
    th = [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in (0.5, 0.5, 0.01, 0.5)]

    def serial():
        for rp, sp, rd, sd in data[:n_s]:
            soft = apsm.train_detect_autograd(p, rp, sp, rd, cg, *th)
            (soft - sd).abs().pow(2).sum().backward()

    ms_serial = _time_events(serial, max(1, args.steps // 2), 1) * n_inst / n_s
    print(json.dumps({"metric": METRIC, "value": n_inst * N / (ms / 1e3), "unit": "symbol-vectors/s (forward+backward)",
                      "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
                      "forward_ms": fwd, "backward_over_forward": (ms - fwd) / fwd,
                      "serial_autograd_ms_extrapolated": ms_serial, "higher_is_better": True, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": f"{n_inst} instances x (M={M}, K={K}, P={P}, W={W}, D={D}, N={N}); "
                                             "gradients wrt sigma, mu, eps, w_L, c_0; "
                                             "one CUDA graph over 64 streams, batched training adjoint"},
                      "loss": float(loss), "grad_sample": [float(v) for v in dscal]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-oracle", action="store_true", help="skip the CPU baseline and FP64 error legs")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--flush-mb", type=int, default=L2_FLUSH_BYTES >> 20,
                    help="MiB written between timed steps to flush L2 (0: none, for profiler captures)")
    ap.add_argument("--workload", default="paper16x6", choices=["paper16x6", "batched", "precision", "grad"])
    ap.add_argument("--precision-n", type=int, default=1 << 20)
    ap.add_argument("--grad-instances", type=int, default=256)
    ap.add_argument("--instances", type=int, default=1024)
    ap.add_argument("--lanes", type=int, default=32)
    ap.add_argument("--tuning", default=None, help="autotuner table (JSON) for the batched workload")
    args = ap.parse_args()
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "precision":
        run_precision(args)
        return
    if args.workload == "grad":
        run_grad(args)
        return
    w = dict(WORKLOAD)
    if args.impl == "reference":
        reference_arm(args, w)
        return

    import torch
    from paper_2201_05024_gb300 import apsm, build, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0 or world == 1:
        build.build()
    if dist is not None:
        dist.barrier()
    apsm.load_library()
    dev = torch.device("cuda", torch.cuda.current_device())

    inst = synth.make_instance(w["M"], w["K"], w["P"], w["N"], w["snr_db"], instance=rank)
    gp = apsm.Params(M=w["M"], K=w["K"], window=w["W"], dict_cap=w["D"], sigma=w["sigma"], mu=w["mu"],
                     eps=w["eps"], w_L=w["w_L"])
    rp = torch.from_numpy(inst.rx_pilot).to(dev)
    sp = torch.from_numpy(inst.sym_pilot).to(dev)
    rd = torch.from_numpy(inst.rx_data).to(dev)
    st = apsm.State(gp, device=dev)
    ws = torch.empty((max(apsm.train_workspace_bytes(gp, w["P"]), 1),), dtype=torch.uint8, device=dev)
    soft = torch.empty((w["N"], w["K"]), dtype=torch.complex64, device=dev)
    hard = torch.empty((w["N"], w["K"]), dtype=torch.uint8, device=dev)
    dws = None  # plain detection form (one CTA per query tile): the faster one at this size
    flush = torch.empty((max(args.flush_mb, 1) << 18,), dtype=torch.float32, device=dev)
    do_flush = args.flush_mb > 0
    stream = torch.cuda.current_stream()

    def step():
        apsm.train(gp, rp, sp, st, workspace=ws)
        apsm.detect(gp, st, rd, soft=soft, hard=hard, workspace=dws)

    for _ in range(max(args.warmup, 3)):
        if do_flush:
            flush.fill_(1.0)
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = apsm.launch_count()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        if do_flush:
            flush.fill_(float(i))       # L2 flush between timed steps (outside the events)
        ev[i][0].record(stream)
        apsm.train(gp, rp, sp, st, workspace=ws)
        ev[i][1].record(stream)
        apsm.detect(gp, st, rd, soft=soft, hard=hard, workspace=dws)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist is not None:
        dist.barrier()
    launches = apsm.launch_count() - launches0
    clocks = sampler.stop()
    t_train = [a.elapsed_time(b) for a, b, _ in ev]
    t_detect = [b.elapsed_time(c) for _, b, c in ev]
    t_step = sum(t_train) + sum(t_detect)  # ms over K steps
    mean_train = sum(t_train) / len(t_train)
    mean_detect = sum(t_detect) / len(t_detect)
    t_step, mean_train, mean_detect = reduce_max(dist, [t_step, mean_train, mean_detect], dev)
    ms_per_step = t_step / args.steps
    value = job_rate(world, w["N"], ms_per_step)
    assert apsm.read_status(st) == 0, "device status word set during the benchmark"

    # ---- end to end through the public API on host buffers (pinned), copies inside the timing
    e2e = None
    if not args.no_e2e:
        hp = torch.from_numpy(inst.rx_pilot).pin_memory()
        hs = torch.from_numpy(inst.sym_pilot).pin_memory()
        hd = torch.from_numpy(inst.rx_data).pin_memory()
        for _ in range(2):
            apsm.train_detect_host(gp, hp, hs, hd, state=st, device=dev, workspace=dws)
        e2e_times = []
        for _ in range(max(3, min(args.steps, 10))):
            if do_flush:
                flush.fill_(0.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            soft_h, hard_h = apsm.train_detect_host(gp, hp, hs, hd, state=st, device=dev, workspace=dws)
            e2e_times.append(time.perf_counter() - t0)
        e2e_step = sum(e2e_times) / len(e2e_times)
        e2e_step = reduce_max(dist, [e2e_step], dev)[0]
        h2d = hp.numel() * 8 + hs.numel() * 8 + hd.numel() * 8
        d2h = soft_h.numel() * 8 + hard_h.numel()
        e2e = {"value": world * w["N"] / e2e_step, "unit": "symbol-vectors/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_step * 1e3}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    n_entries = int(st.meta[0].item())
    roof = detect_roofline(w, n_entries, mean_detect / 1e3)
    roof["traffic"] = DETECT_TRAFFIC["bytes_per_launch"] if DETECT_TRAFFIC["digest"] == kernel_digest() else None
    out = {
        "metric": METRIC, "value": value, "unit": "symbol-vectors/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(w),
                   "l2": f"flushed between timed steps ({args.flush_mb} MiB write)" if do_flush else "not flushed",
                   "parallelism": f"independent instance per GPU x{world}", "step": "train P pilots + detect N vectors"},
        "detect": {"value": world * w["N"] / (mean_detect / 1e3), "unit": "symbol-vectors/s",
                   "ms": mean_detect},
        "train": {"value": world * w["P"] * w["K"] / (mean_train / 1e3), "unit": "pilot-updates/s",
                  "ms": mean_train, "us_per_pilot": mean_train * 1e3 / w["P"]},
        "roofline": {"kernel": "detect_tma_kernel<16,6> (TF32 x3 Gram)", **roof},
        "gpu_launches": int(launches),
        "wall_s_timed": wall,
        "e2e": e2e,
        "clocks": clocks,
    }
    if not args.no_oracle:
        sample = np.random.default_rng(0).choice(w["N"], ORACLE_DETECT_SAMPLE, replace=False)
        import oracle
        st_ref, ref, tt, td = run_oracle(w, inst, sample)
        val_cpu, _ = oracle_step_rate(w, tt, td, len(sample))
        cores = oracle.default_threads()
        # the same on one core: training with one thread, a smaller detection sample
        _, _, tt1, td1 = run_oracle(w, inst, sample[:1024], threads=1)
        val_cpu1, _ = oracle_step_rate(w, tt1, td1, 1024)
        out["cpu_baseline"] = {
            "value": val_cpu, "unit": "symbol-vectors/s", "cores": cores, "kind": "oracle",
            "sample": (f"full FP64 training ({w['P']} pilots, users on {min(cores, w['K'])} threads, {tt:.2f} s) + "
                       f"detection of {len(sample)} sampled vectors ({td:.2f} s), extrapolated to {w['N']}"),
            "one_core": {"value": val_cpu1, "unit": "symbol-vectors/s", "cores": 1,
                         "sample": f"full training on one thread ({tt1:.2f} s) + 1024 sampled vectors ({td1:.2f} s), "
                                   f"extrapolated to {w['N']}"}}
        y = soft.cpu().numpy()[sample].astype(np.complex128)
        cr = np.stack([ref.real, ref.imag])
        cy = np.stack([y.real, y.imag])
        rms = float(np.sqrt(np.mean(cr ** 2)))
        err = np.abs(cy - cr) / np.maximum(np.abs(cr), rms)
        h_ref = oracle.hard_qpsk(ref)
        out["err_vs_fp64"] = {"max_scaled": float(err.max()), "rms_scaled": float(np.sqrt(np.mean(err ** 2))),
                              "sample": len(sample),
                              "ser_gpu": float(np.mean(hard.cpu().numpy()[sample] != inst.idx_data[sample])),
                              "ser_oracle": float(np.mean(h_ref != inst.idx_data[sample]))}
        out["snr_sweep"] = snr_sweep(w)
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
