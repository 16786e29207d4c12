#!/usr/bin/env python
"""Benchmark of the GB300 sparse FFT (R-FFAST peeling) on its headline workload.

Workload (one step): a batch of S synthetic signals shaped like the paper's general sparse
experiments (Sec. 5.1): N = 127*128*129 = 2,097,024 complex64 samples, three stages with
B_d = 16512, 16383, 16256, eight delays per stage (0, 1 and six uniform draws), K = 1000
coefficients with |xhat| ~ U[1, 10] and uniform phase, complex white Gaussian noise at
20 dB SNR.  Every step recovers all S signals through the library's batched path (gather
+ prime-factor DFTs, peeling decode, compaction).  The S inputs (8.6 GB at the default
S = 512) are resident in HBM and larger than L2, so no L2 flush is needed between steps.

Printed: one JSON line (rank 0) with signals/s, per-signal latency (p50/p99), accuracy
against the plain FP64 path, the plain FP64 path's own signals/s, the dominant kernel's
roofline, the CPU oracle's rate on the host cores, an end-to-end number through host
buffers, and the SM clocks seen during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch S] [--impl gb300|reference]
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "rffast_2097024"
CFG = synth.CONFIGS[WORKLOAD]
METRIC = ("signals/s and p50/p99 latency at stated L2 error vs plain FP64 path; "
          "gather % HBM")
N_DISTINCT = 8
# sources whose hash keys the committed ncu traffic figure of the bucketization kernel
TRAFFIC_SRC = ["paper_2011_05749_gb300/csrc/dft.cu",
               "paper_2011_05749_gb300/csrc/sfft_internal.cuh",
               "paper_2011_05749_gb300/csrc/pfa_layout.h"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=512, help="signals per step per GPU")
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--max-tile", type=int, default=0,
                    help="largest DFT tile per CTA in elements (0: shared-memory limit)")
    ap.add_argument("--serve-rate", type=float, default=20000.0,
                    help="mean Poisson arrival rate of the serving measurement (requests/s)")
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--mix-seconds", type=float, default=10.0,
                    help="length of the serving-mix Poisson stream")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large single-signal measurement (N = 511*512*513)")
    ap.add_argument("--only", choices=["large", "sweep", "oneshot", "locate", "noise", "dsfft", "mix",
                                       "serve", "dft", "ml"],
                    default=None,
                    help="run only that block (a short run for profiling) and print its JSON")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip sfft_autotune and use the default schedule")
    ap.add_argument("--timed-only", action="store_true",
                    help="run only the timed batched loop (for profiler captures)")
    return ap.parse_args()


def expected_noise_var():
    lo, hi = CFG["mag"]
    e_mag2 = (hi ** 3 - lo ** 3) / (3.0 * (hi - lo))  # E|xhat|^2 for |xhat| ~ U[lo, hi]
    return CFG["K"] * e_mag2 / 10.0 ** (CFG["snr_db"] / 10.0)


def plan_delays(seed):
    rng = np.random.default_rng(10_000 + seed)
    return synth.draw_delays(CFG["N"], len(CFG["f"]), CFG["R"], rng)


def problems(seed, delays, n):
    return [synth.make_problem(CFG["N"], CFG["f"], CFG["K"], seed * 1000 + i, R=CFG["R"],
                               delays=delays, mag=CFG["mag"], snr_db=CFG["snr_db"])
            for i in range(n)]


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), max=float(parts[2]),
                                 util=float(parts[4]) if parts[4] not in ("", "[N/A]") else 0.0,
                                 reasons=[n for n, v in zip(
                                     ("hw_slowdown", "hw_thermal_slowdown",
                                      "sw_thermal_slowdown", "sw_power_cap"), parts[5:9])
                                     if v.lower() == "active"]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        busy = [r for r in rows if r["util"] > 0] or rows
        reasons = sorted({x for r in busy for x in r["reasons"]})
        return {"sm_mhz": statistics.median(r["sm"] for r in busy),
                "sm_max_mhz": max(r["max"] for r in rows), "reasons": reasons,
                "samples": len(busy)}


# ------------------------------------------------------------------------------ oracle arm
def oracle_rate(seed, budget_s, max_signals=64):
    """Time the FP64 CPU oracle (naive bucketization + peeling decode), as it stands, on
    up to max_signals workload signals until budget_s of wall time is used."""
    import oracle
    oracle.build_oracle()
    delays = plan_delays(seed)
    nv = expected_noise_var()
    opts = oracle.OracleOpts(noise_var=nv, eta=3e-3, locate=1)
    done, t_work = 0, 0.0
    for i in range(max_signals):
        p = synth.make_problem(CFG["N"], CFG["f"], CFG["K"], 77_000 + seed * 100 + i,
                               R=CFG["R"], delays=delays, mag=CFG["mag"], snr_db=CFG["snr_db"])
        x = p.x.astype(np.complex64).astype(np.complex128)
        t0 = time.perf_counter()
        Y = oracle.bucketize(p.N, p.f, p.delays, x)
        oracle.decode(p.N, p.f, p.delays, Y, p.K, opts)
        t_work += time.perf_counter() - t0
        done += 1
        if t_work >= budget_s:
            break
    return done / t_work, done, t_work


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    import oracle
    oracle.build_oracle()
    delays = plan_delays(args.seed)
    opts = oracle.OracleOpts(noise_var=expected_noise_var(), eta=3e-3, locate=1)
    probs = problems(args.seed + 500, delays, min(args.steps + args.warmup, 4))
    xs = [p.x.astype(np.complex64).astype(np.complex128) for p in probs]
    for i in range(args.warmup):
        p = probs[i % len(probs)]
        oracle.decode(p.N, p.f, p.delays, oracle.bucketize(p.N, p.f, p.delays, xs[i % len(xs)]),
                      p.K, opts)
    t0 = time.perf_counter()
    for i in range(args.steps):
        p = probs[i % len(probs)]
        oracle.decode(p.N, p.f, p.delays, oracle.bucketize(p.N, p.f, p.delays, xs[i % len(xs)]),
                      p.K, opts)
    el = time.perf_counter() - t0
    v = args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "signals/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: one signal per step through the FP64 CPU oracle "
                               "(naive B-point DFTs + peeling decode)",
                   "N": CFG["N"], "K": CFG["K"], "R": CFG["R"], "snr_db": CFG["snr_db"]},
        "cpu_baseline": {"value": v, "unit": "signals/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} signals of the workload, one per step"},
        "e2e": {"value": v, "unit": "signals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line, default=float), flush=True)
    return 0


# ------------------------------------------------------------------------------ GPU arm
def max_over_ranks(v: float, world: int, device="cuda") -> float:
    """Largest value over the ranks (the job is as slow as its slowest replica)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1e3)


def kernel_traffic(kernel: str, src_files, per_unit_key: str):
    """Traffic per unit from the committed ncu summary, if the kernel source still
    matches the hash recorded there; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    h = hashlib.sha256()
    for f in src_files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if rec.get("src_sha256") != h.hexdigest():
        return None
    return rec.get(per_unit_key)


def measure_large(sfft, hbm_peak, reps=10):
    """Large single signal, N = 511*512*513 = 134,217,216 complex64 (1.07 GB), f = (511, 512,
    513), 10 delays per stage, K = 10,000, |xhat| ~ U[1,10], exactly sparse: one sfft_execute
    per signal (two-pass bucketization in every stage).  Reports ms per signal, the phases,
    exact recovery, and the gather's share of HBM: algorithmic bytes (samples read + bins
    written) and the DRAM bytes ncu measured for this workload (when the kernel source
    still matches) over the bucketization time."""
    import torch
    p = synth.config_problem("rffast_134217216", seed=5, snr_db=None)
    plan = sfft.Plan(p.N, p.K, p.f, p.delays, precision="fp32", locate="ml")
    x = torch.from_numpy(p.x.astype(np.complex64)).cuda()
    idx, val, info = plan.execute(x)
    idx, val, info = plan.execute(x)
    torch.cuda.synchronize()
    plan.profile(reset=True)
    plan.set_profiling(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(reps):
        idx, val, info = plan.execute(x)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    prof = plan.profile(reset=True)
    inf = info.cpu().numpy()
    n = int(inf[0])
    exact = bool(inf[1] == 0 and n == p.K and np.array_equal(idx[:n].cpu().numpy(), p.support))
    bk_ms = prof["bucketize"]["ms"] / reps
    alg = p.R * sum(p.N // L for L in p.f) * 8 * 2
    dram = kernel_traffic("bucketize_kernel<float,float>@rffast_134217216", TRAFFIC_SRC,
                          "dram_bytes_per_signal")
    # end to end from a page-locked host signal, outputs to host: the copy of the whole
    # signal to device memory, against a host_gather plan whose bucketization reads the
    # samples in place over the host link
    xh = torch.from_numpy(p.x.astype(np.complex64)).pin_memory()
    del x
    e2e = {}
    for mode in ("copy", "host_gather"):
        pl = plan if mode == "copy" else sfft.Plan(p.N, p.K, p.f, p.delays, precision="fp32",
                                                     locate="ml", host_gather=True)
        outs = pl.empty_outputs("cpu")
        pl.execute(xh, out=outs)
        t0 = time.perf_counter()
        for _ in range(max(1, reps // 2)):
            pl.execute(xh, out=outs)
        dt = (time.perf_counter() - t0) / max(1, reps // 2)
        n_h = int(outs[2][0])
        e2e[mode] = {"ms_per_signal": dt * 1e3, "signals_per_s": 1.0 / dt,
                     "exact_recovery": bool(outs[2][1] == 0 and n_h == p.K
                                            and np.array_equal(outs[0][:n_h], p.support))}
        if pl is not plan:
            pl.close()
    e2e["h2d_bytes_copy"] = int(p.N) * 8
    plan.close()
    return {"workload": "rffast_134217216: N=511*512*513 complex64 (1.07 GB), f=(511,512,513), "
                        "10 delays/stage (0,1,8 random), K=10000, |xhat|~U[1,10], exactly sparse",
            "ms_per_signal": ms, "signals_per_s": 1e3 / ms,
            "phases_ms_per_signal": {k: v["ms"] / reps for k, v in prof.items()},
            "exact_recovery": exact,
            "e2e_from_pinned_host": e2e,
            "gather": {"bucketize_ms": bk_ms, "alg_bytes": alg,
                       "alg_frac_of_hbm": alg / (bk_ms * 1e-3) / (hbm_peak * 1e9),
                       "dram_bytes": dram,
                       "dram_frac_of_hbm": (dram / (bk_ms * 1e-3) / (hbm_peak * 1e9)
                                            if dram else None),
                       "sector_efficiency": (alg / dram if dram else None),
                       "peak_gbs": hbm_peak}}


def errors_vs(idx, val, n, ref_idx, ref_val, K):
    """L0, L1 and L2 of one result against a reference result over the union of the supports
    (L1 = sum |difference| / K, L2 relative to the reference's norm)."""
    got = dict(zip(idx[:n].tolist(), val[:n].tolist()))
    ref = dict(zip(ref_idx.tolist(), ref_val.tolist()))
    keys = sorted(set(got) | set(ref))
    d = np.array([got.get(k, 0) - ref.get(k, 0) for k in keys]) if keys else np.zeros(1)
    nr = np.linalg.norm(np.array(list(ref.values()))) if ref else 1.0
    return {"l0": len(set(got) ^ set(ref)), "l1": float(np.abs(d).sum() / max(K, 1)),
            "l2": float(np.linalg.norm(d) / (nr if nr > 0 else 1.0))}


def measure_large_sweep(sfft, reps=3):
    """The large-signal configuration over its SNR sweep: N = 511*512*513 complex64, f =
    (511, 512, 513), 10 delays per stage (0, 1, 8 random), K = 10,000, |xhat| ~ U[1,10], SNR in
    {inf, 30, 10} dB (one sparse spectrum, one draw of white noise scaled per SNR).  Per SNR:
    the FP32 path (FP64 location and fit; ordered, compensated peeling) and, beside it, the
    same with unordered float atomics in the peeling subtraction, and the plain FP64 path --
    each with L0/L1/L2 against the truth, and the FP32 results against the FP64 path's.
    Then the location precision experiment on the exactly sparse signal with ARG locate
    (delays 0 and 1 of every stage): the angle in FP64 or FP32, with or without the snap to
    the bin's candidate set, on FP32 bins and on FP64 bins."""
    import torch
    base = synth.config_problem("rffast_134217216", seed=5, snr_db=None)
    N, f, K = base.N, base.f, base.K
    w = synth.awgn(N, 1.0, np.random.default_rng(555))
    truth_i, truth_v = base.support, base.values
    out = {"workload": "rffast_134217216: N=511*512*513 complex64 (1.07 GB), 10 delays/stage, "
                       "K=10000, |xhat|~U[1,10]; SNR sweep {inf, 30, 10} dB", "snr": {}}

    def run(plan, x):
        o = plan.execute(x)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            o = plan.execute(x)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) / reps * 1e3
        inf = o[2].cpu().numpy()
        n = int(inf[0])
        return ms, o[0].cpu().numpy(), o[1].cpu().numpy().astype(np.complex128), n, int(inf[1])

    for snr in (None, 30.0, 10.0):
        var = synth.noise_variance(truth_v, snr)
        x = base.x + np.sqrt(var) * w if var > 0 else base.x
        x32 = torch.from_numpy(x.astype(np.complex64)).cuda()
        rec = {"noise_var": var}
        res = {}
        for name, kw in (("fp32", {}), ("fp32_atomic_peel", {"peel_atomic": True})):
            plan = sfft.Plan(N, K, f, base.delays, precision="fp32", locate="ml", noise_var=var, **kw)
            ms, i, v, n, st = run(plan, x32)
            plan.close()
            res[name] = (i, v, n)
            rec[name] = {"ms_per_signal": ms, "status": st, "count": n,
                         "vs_truth": errors_vs(i, v, n, truth_i, truth_v, K)}
        del x32
        x64 = torch.from_numpy(x.astype(np.complex64).astype(np.complex128)).cuda()
        plan = sfft.Plan(N, K, f, base.delays, precision="fp64", dtype="c128", locate="ml",
                         noise_var=var)
        ms, i64, v64, n64, st = run(plan, x64)
        plan.close()
        del x64
        rec["fp64_plain"] = {"ms_per_signal": ms, "status": st, "count": n64,
                             "vs_truth": errors_vs(i64, v64, n64, truth_i, truth_v, K)}
        for name in ("fp32", "fp32_atomic_peel"):
            i, v, n = res[name]
            rec[name]["vs_fp64_plain"] = errors_vs(i, v, n, i64[:n64], v64[:n64], K)
        out["snr"]["inf" if snr is None else f"{snr:g}dB"] = rec
    # location precision on the exactly sparse signal, ARG locate
    loc = {}
    x32 = torch.from_numpy(base.x.astype(np.complex64)).cuda()
    for mode, name in ((0, "fp64_angle_snapped"), (1, "fp32_angle_snapped"),
                       (2, "fp64_angle_unsnapped"), (3, "fp32_angle_unsnapped")):
        plan = sfft.Plan(N, K, f, base.delays, precision="fp32", locate="arg", arg_mode=mode)
        ms, i, v, n, st = run(plan, x32)
        plan.close()
        loc[f"fp32_bins/{name}"] = {"status": st, "count": n,
                                    "l0_vs_truth": errors_vs(i, v, n, truth_i, truth_v, K)["l0"]}
    del x32
    x64 = torch.from_numpy(base.x).cuda()
    for mode, name in ((0, "fp64_angle_snapped"), (2, "fp64_angle_unsnapped")):
        plan = sfft.Plan(N, K, f, base.delays, precision="fp64", dtype="c128", locate="arg",
                         arg_mode=mode)
        ms, i, v, n, st = run(plan, x64)
        plan.close()
        loc[f"fp64_bins/{name}"] = {"status": st, "count": n,
                                    "l0_vs_truth": errors_vs(i, v, n, truth_i, truth_v, K)["l0"]}
    out["arg_locate_precision"] = loc
    return out


def measure_oneshot(sfft, batch=64, steps=20, warmup=3):
    """The one-shot (sFFT-DT) decoder, Sec. 3.1: N = 2^21 complex64, one stage of B = 8192
    = 32 K buckets (L = 256), K = 256 with |xhat| ~ U[1,10], a_m = 3, delays -3 .. 5 and 7
    random (R = 16); exactly sparse and 30 dB.  Batches of `batch` signals (8 distinct, repeated)
    through sfft_execute_batch; reports signals/s, the phases and the recovery."""
    import torch
    out = {"workload": "oneshot_2097152: N=2^21 complex64, B=8192 (L=256), K=256, "
                       "|xhat|~U[1,10], a_m=3, R=16 (9 consecutive + 7 random delays); "
                       "Step 2 by enumeration (method 2) unless the key names method 1 "
                       "(polynomial roots) or 3 (matrix pencil)"}
    for snr, method in ((None, 2), (30.0, 2), (None, 1), (30.0, 1), (None, 3), (30.0, 3)):
        probs = [synth.config_problem("oneshot_2097152", seed=60 + i, snr_db=snr) for i in range(8)]
        dl = probs[0].delays  # one plan: the same delays for every signal
        probs = [synth.make_problem(p.N, p.f, p.K, seed=60 + i, delays=dl, mag=(1.0, 10.0),
                                    snr_db=snr) for i, p in enumerate(probs)]
        nv = float(np.mean([p.noise_var for p in probs]))
        plan = sfft.Plan(probs[0].N, probs[0].K, probs[0].f, dl, decoder="oneshot", a_m=3,
                         noise_var=nv, max_batch=batch, dt_method=method)
        dev = [torch.from_numpy(p.x.astype(np.complex64)).cuda() for p in probs]
        xs = torch.stack([dev[i % len(dev)] for i in range(batch)])
        res = plan.empty_outputs("cuda", batch)
        for _ in range(warmup):
            plan.execute_many(xs, res)
        torch.cuda.synchronize()
        plan.profile(reset=True)
        plan.set_profiling(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            plan.execute_many(xs, res)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        prof = plan.profile(reset=True)
        idx, val, info = (t.cpu().numpy() for t in res)
        sup_ok, l0, l2 = 0, 0, []
        for i, p in enumerate(probs):
            n = int(info[i, 0])
            sup_ok += int(n == p.K and np.array_equal(idx[i, :n], p.support))
            e0_, e2_ = union_errors(idx[i], val[i], n, p)
            l0 += e0_
            l2.append(e2_)
        plan.close()
        key = "exact" if snr is None else f"snr_{int(snr)}db"
        out[key if method == 2 else f"method{method}_{key}"] = {
            "signals_per_s": batch * 1e3 / ms, "ms_per_step": ms, "batch": batch,
            "phases_ms_per_step": {k: v["ms"] / steps for k, v in prof.items()},
            "support_equal_truth": f"{sup_ok}/{len(probs)}",
            "l0_vs_truth_total": l0, "l0_per_signal_of_K": l0 / len(probs) / probs[0].K,
            "rel_l2_vs_truth_max": max(l2)}
    return out


def union_errors(idx, val, n, p):
    """L0 and relative L2 of one result against the truth over the union of the supports
    (a missing coefficient counts as zero)."""
    got = dict(zip(idx[:n].tolist(), val[:n].tolist()))
    ref = dict(zip(p.support.tolist(), p.values.tolist()))
    keys = sorted(set(got) | set(ref))
    d = np.array([got.get(k, 0) - ref.get(k, 0) for k in keys])
    return len(set(got) ^ set(ref)), float(np.linalg.norm(d) / np.linalg.norm(p.values))


def measure_locate_modes(sfft, batch=64, steps=20, warmup=3):
    """The R-FFAST workload's signals (N = 127*128*129, K = 1000, 20 dB) located two ways:
    ML over the candidates with 8 delays per stage (0, 1, 6 random; the benchmark's mode)
    and the paper's structured delays with the Kay estimator and binary search (Sec. 3.2,
    Eq. 21-22; C = 8 iterations of m = 2, 16 delays per stage).  Same signals for both."""
    import torch
    N, f, K = CFG["N"], CFG["f"], CFG["K"]
    modes = {"ml": dict(delays=synth.draw_delays(N, 3, 8, np.random.default_rng(71)), kw={}),
             "kay": dict(delays=synth.kay_delays(N, 3, 8, 2, np.random.default_rng(72)),
                         kw=dict(locate="kay", kay_m=2))}
    out = {"workload": f"{WORKLOAD} signals at 20 dB; ml: 8 delays (0, 1, 6 random); "
                       "kay: 16 structured delays (C = 8, m = 2)"}
    for name, md in modes.items():
        probs = [synth.make_problem(N, f, K, seed=80 + i, delays=md["delays"], mag=(1.0, 10.0),
                                    snr_db=20.0) for i in range(8)]
        nv = float(np.mean([p.noise_var for p in probs]))
        kw = dict(precision="fp32", noise_var=nv, max_batch=batch, **md["kw"])
        if name == "ml":
            kw["locate"] = "ml"
        plan = sfft.Plan(N, K, f, md["delays"], **kw)
        dev = [torch.from_numpy(p.x.astype(np.complex64)).cuda() for p in probs]
        xs = torch.stack([dev[i % len(dev)] for i in range(batch)])
        res = plan.empty_outputs("cuda", batch)
        for _ in range(warmup):
            plan.execute_many(xs, res)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            plan.execute_many(xs, res)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        idx, val, info = (t.cpu().numpy() for t in res)
        errs = [union_errors(idx[i], val[i], int(info[i, 0]), p) for i, p in enumerate(probs)]
        plan.close()
        del xs, dev
        out[name] = {"delays_per_stage": int(md["delays"].shape[1]),
                     "signals_per_s": batch * 1e3 / ms, "ms_per_step": ms, "batch": batch,
                     "l0_vs_truth_total": int(sum(e[0] for e in errs)),
                     "rel_l2_vs_truth_max": max(e[1] for e in errs),
                     "status_incomplete": int(np.sum(info[:len(probs), 1] == 2))}
    return out


def measure_noise_auto(sfft, batch=64, steps=20, warmup=3):
    """The R-FFAST workload (N = 127*128*129, K = 1000, 20 dB, ML locate, 8 delays) decoded
    without a given sigma^2: each signal's sigma^2 is estimated from its bins (the lower
    median of sum_r |Y_r|^2 / B over all bins over the median of Gamma(R, 1)) and sets T0, T1.
    Reports signals/s, L0/L2 against the truth and the estimates over the true sigma^2."""
    import torch
    N, f, K = CFG["N"], CFG["f"], CFG["K"]
    delays = plan_delays(2)
    probs = problems(2, delays, N_DISTINCT)
    plan = sfft.Plan(N, K, f, delays, precision="fp32", locate="ml", noise_auto=True,
                     max_batch=batch)
    dev = [torch.from_numpy(p.x.astype(np.complex64)).cuda() for p in probs]
    xs = torch.stack([dev[i % len(dev)] for i in range(batch)])
    res = plan.empty_outputs("cuda", batch)
    for _ in range(warmup):
        plan.execute_many(xs, res)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        plan.execute_many(xs, res)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    idx, val, info = (t.cpu().numpy() for t in res)
    errs = [union_errors(idx[i], val[i], int(info[i, 0]), p) for i, p in enumerate(probs)]
    ratio = [plan.noise_var(i) / p.noise_var for i, p in enumerate(probs)]
    plan.close()
    return {"workload": f"{WORKLOAD} at 20 dB, sigma^2 estimated per signal (noise_auto)",
            "signals_per_s": batch * 1e3 / ms, "ms_per_step": ms, "batch": batch,
            "l0_vs_truth_total": int(sum(e[0] for e in errs)),
            "rel_l2_vs_truth_max": max(e[1] for e in errs),
            "sigma2_estimate_over_true": {"min": min(ratio), "max": max(ratio)}}


def measure_plan_paths(sfft, variants, batch=256, steps=20, warmup=3):
    """The R-FFAST workload through plans that differ in one option each (`variants`: pairs
    of a name and the Plan keyword arguments), the same signals and schedule otherwise:
    signals/s, the bucketization's and the decoder's ms per step and L0/L2 against the truth
    for each."""
    import torch
    N, f, K = CFG["N"], CFG["f"], CFG["K"]
    delays = plan_delays(3)
    probs = problems(3, delays, N_DISTINCT)
    nv = float(np.mean([p.noise_var for p in probs]))
    dev = [torch.from_numpy(p.x.astype(np.complex64)).cuda() for p in probs]
    xs = torch.stack([dev[i % len(dev)] for i in range(batch)])
    out = {"workload": f"{WORKLOAD}, batches of {batch}"}
    for name, kw in variants:
        plan = sfft.Plan(N, K, f, delays, precision="fp32", locate="ml", noise_var=nv,
                         max_batch=batch, **kw)
        res = plan.empty_outputs("cuda", batch)
        for _ in range(warmup):
            plan.execute_many(xs, res)
        torch.cuda.synchronize()
        plan.profile(reset=True)
        plan.set_profiling(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            plan.execute_many(xs, res)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        prof = plan.profile(reset=True)
        idx, val, info = (t.cpu().numpy() for t in res)
        errs = [union_errors(idx[i], val[i], int(info[i, 0]), p) for i, p in enumerate(probs)]
        plan.close()
        out[name] = {"signals_per_s": batch * 1e3 / ms, "ms_per_step": ms,
                     "bucketize_ms_per_step": prof["bucketize"]["ms"] / steps,
                     "decode_ms_per_step": prof["decode"]["ms"] / steps,
                     "l0_vs_truth_total": int(sum(e[0] for e in errs)),
                     "rel_l2_vs_truth_max": max(e[1] for e in errs)}
    return out


def measure_dft_paths(sfft, batch=256, steps=20, warmup=3):
    """The R-FFAST workload's DFTs on the two paths the library has: the default (the 43- and
    127-point direct DFTs on the tensor cores as 3-term split FP16 products) and a
    dft_fma_only plan (every axis on the FMA pipes)."""
    return measure_plan_paths(sfft, [("tensor_core_odd_axes", {}),
                                     ("fma_only", {"dft_fma_only": True})], batch, steps, warmup)


def measure_ml_paths(sfft, batch=256, steps=20, warmup=3):
    """The first round's ML candidate search three ways on the same signals: on the tensor
    cores as split-FP16 m16n8k16 MMAs (the default), as split-TF32 m16n8k8 MMAs
    (ml_tc_tf32), and on the FMA pipes with two lanes per bin (classify_lanes = 2)."""
    return measure_plan_paths(sfft, [("tensor_core_fp16", {}),
                                     ("tensor_core_tf32", {"ml_tc_tf32": True}),
                                     ("fma_lanes_2", {"classify_lanes": 2})], batch, steps, warmup)


def measure_dsfft(sfft, batch=64, steps=5, warmup=1):
    """DSFFT binary tree search (Sec. 3.3 / 4.3): N = 2^20 complex64, K = 16 tones with
    |xhat| ~ U[1,10], exactly sparse, search from layer 4 (B = 16).  Batches of `batch`
    signals (8 distinct, repeated); the library runs each signal's search on its own (one
    device round trip per layer).  Reports signals/s, the stop layers and the recovery."""
    import torch
    N, K, p0 = 1 << 20, 16, 4
    probs = [synth.make_problem(N, (1,), K, seed=90 + i, delays=np.array([[0, 1]]),
                                mag=(1.0, 10.0)) for i in range(8)]
    plan = sfft.Plan(N, K, (N >> p0,), [[0, 1]], precision="fp32", decoder="dsfft",
                     max_batch=batch)
    dev = [torch.from_numpy(p.x.astype(np.complex64)).cuda() for p in probs]
    xs = torch.stack([dev[i % len(dev)] for i in range(batch)])
    res = plan.empty_outputs("cuda", batch)
    for _ in range(warmup):
        plan.execute_many(xs, res)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        plan.execute_many(xs, res)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    idx, val, info = (t.cpu().numpy() for t in res)
    errs = [union_errors(idx[i], val[i], int(info[i, 0]), p) for i, p in enumerate(probs)]
    plan.close()
    return {"workload": "dsfft_1048576: N=2^20 complex64, K=16, |xhat|~U[1,10], exactly sparse, "
                        "search from layer 4, delays {0, 1}",
            "signals_per_s": batch * 1e3 / ms, "ms_per_step": ms, "batch": batch,
            "timing": "host clock around the batch (the search synchronises per layer)",
            "stop_layer": {"min": int(info[:, 2].min()), "max": int(info[:, 2].max())},
            "l0_vs_truth_total": int(sum(e[0] for e in errs)),
            "rel_l2_vs_truth_max": max(e[1] for e in errs)}


def measure_batched_mix(sfft, n_signals=4096, steps=3, warmup=1, plain_per_size=8):
    """The batched configuration: n_signals complex64 signals in one sfft_execute_batch
    call, N drawn from {9660, 124950 = 49*50*51, 2097024 = 127*128*129} (three stages, 6
    delays: 0, 1 and 4 random), K uniform in [10, 500], SNR uniform in [10, 40] dB, |xhat|
    ~ U[1,10].  Each signal's noise variance is estimated from its own bins (noise_auto), so
    one plan per N serves every SNR.  The batch is timed in a shuffled order (the library
    groups each plan's signals wherever they sit: one launch set per plan) and, beside it,
    ordered by N.  Beside them: the plain FP64 path, one signal per sfft_execute, on
    plain_per_size signals of each N; the ratio is the batched rate over the plain rate of
    the same mix.  Inputs: 8 distinct signals per N, each stored n_signals / 24 times."""
    import torch
    sizes = [(9660, (20, 21, 23)), (124950, (49, 50, 51)), (2097024, (127, 128, 129))]
    rng = np.random.default_rng(2024)
    per = n_signals // len(sizes)
    out = {"workload": f"{n_signals} complex64 signals, N from {{9660, 124950, 2097024}}, "
                       "K ~ U{10..500}, SNR ~ U[10,40] dB, 6 delays (0, 1, 4 random), "
                       "sigma^2 estimated per signal", "sizes": {}}
    plans, xs, probs_all, plan_of = [], [], [], []
    for N, f in sizes:
        delays = synth.draw_delays(N, 3, 6, rng)
        probs = []
        for i in range(8):
            K = int(rng.integers(10, 501))
            snr = float(rng.uniform(10.0, 40.0))
            probs.append(synth.make_problem(N, f, K, seed=int(rng.integers(1 << 30)),
                                            delays=delays, mag=(1.0, 10.0), snr_db=snr))
        plan = sfft.Plan(N, 500, f, delays, precision="fp32", locate="ml", noise_auto=True,
                         max_batch=per)
        dev = [torch.from_numpy(p.x.astype(np.complex64)).cuda() for p in probs]
        for i in range(per):
            xs.append(dev[i % 8])
            probs_all.append(probs[i % 8])
            plan_of.append(plan)
        plans.append((N, f, delays, probs, plan))
    n = len(xs)
    idx = [torch.zeros(500, dtype=torch.int64, device="cuda") for _ in range(n)]
    val = [torch.zeros(500, dtype=torch.complex64, device="cuda") for _ in range(n)]
    infos = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    perm = np.random.default_rng(77).permutation(n)

    def timed(order):
        po = [plan_of[i] for i in order]
        xo = [xs[i] for i in order]
        io = [idx[i] for i in order]
        vo = [val[i] for i in order]
        inf_o = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
        for _ in range(warmup):
            sfft.execute_batch(po, xo, (io, vo, inf_o))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            sfft.execute_batch(po, xo, (io, vo, inf_o))
        e1.record()
        torch.cuda.synchronize()
        infos[torch.from_numpy(np.asarray(order)).cuda()] = inf_o
        return e0.elapsed_time(e1) / steps

    ms_sorted = timed(np.arange(n))
    ms = timed(perm)
    inf = infos.cpu().numpy()
    k = 0
    plain_s = 0.0
    for N, f, delays, probs, plan in plans:
        l0 = 0
        for i in range(per):
            if i < 8:
                c = int(inf[k + i, 0])
                l0 += union_errors(idx[k + i].cpu().numpy(), val[k + i].cpu().numpy(), c, probs[i])[0]
        k += per
        # plain FP64 path: one signal per call
        p64 = sfft.Plan(N, 500, f, delays, precision="fp64", dtype="c128", locate="ml",
                        noise_auto=True)
        x64 = [torch.from_numpy(p.x.astype(np.complex128)).cuda() for p in probs]
        o64 = p64.empty_outputs()
        p64.execute(x64[0], o64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(plain_per_size):
            p64.execute(x64[i % 8], o64)
        torch.cuda.synchronize()
        plain_s += (time.perf_counter() - t0) / plain_per_size
        p64.close()
        out["sizes"][str(N)] = {"signals": per, "l0_vs_truth_first8_total": l0,
                                "true_K_first8": [p.K for p in probs]}
    for *_, plan in plans:
        plan.close()
    batched = n * 1e3 / ms
    plain = len(sizes) / plain_s  # signals/s over the same mix, one per call
    out.update({"signals_per_s": batched, "ms_per_batch": ms, "order": "shuffled",
                "sorted_by_n": {"signals_per_s": n * 1e3 / ms_sorted, "ms_per_batch": ms_sorted},
                "plain_fp64_signals_per_s": plain, "speedup_vs_plain_fp64": batched / plain})
    return out


def measure_serving(sfft, plan, signals, rate, seconds, seed):
    """Submit requests (one workload signal each) at Poisson arrival times for `seconds`,
    then drain; latency = submit to completion, as the server measures it."""
    import torch
    rng = np.random.default_rng(seed + 99)
    n = max(1, int(rate * seconds))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
    srv = sfft.Server(hbm_budget=16 << 30, max_slots=16)
    srv.reserve(plan, 16)
    warm = [srv.submit(plan, signals[i % len(signals)], plan.empty_outputs())
            for i in range(16 * 32)]
    srv.drain()
    del warm
    ring = 4096
    outs = [plan.empty_outputs() for _ in range(min(ring, n))]
    slot_ticket = [0] * len(outs)
    tickets = []
    t0 = time.perf_counter()
    for i in range(n):
        while time.perf_counter() - t0 < arrivals[i]:
            pass
        k = i % len(outs)
        if slot_ticket[k]:
            while srv.poll(slot_ticket[k])[0] == 1:  # ring slot still in use
                pass
        t = srv.submit(plan, signals[i % len(signals)], outs[k])
        slot_ticket[k] = t
        tickets.append(t)
    srv.drain()
    t1 = time.perf_counter()
    torch.cuda.synchronize()
    lat = sorted(srv.poll(t)[1] for t in tickets)
    srv.close()
    return {"offered_rate": rate, "requests": n, "completed_rate": n / (t1 - t0),
            "p50_us": lat[len(lat) // 2], "p99_us": lat[int(len(lat) * 0.99) - 1],
            "workload": "one rffast_2097024 signal per request, continuous batching, "
                        "up to 32 requests per launch group, 16 groups in flight"}


def measure_serving_mix(sfft, rate=20000.0, seconds=1.0, seed=4):
    """The serving configuration: Poisson arrivals (mean `rate` requests/s) of one signal
    each, N uniform from {9660, 124950, 2097024, 16776960 = 255*256*257} (three stages, 6
    delays), K log-uniform in [16, 4096] clamped to min_d B_d / 2, SNR uniform in [0, 40] dB
    or exactly sparse (one in four), complex64; each signal's noise variance is estimated
    from its bins (noise_auto), so one plan per N serves every request of that size.  The
    server admits by an HBM budget of 120 GB.  8 distinct signals per N."""
    import torch
    rng = np.random.default_rng(seed)
    sizes = [(9660, (20, 21, 23)), (124950, (49, 50, 51)), (2097024, (127, 128, 129)),
             (16776960, (255, 256, 257))]
    plans, sigs, outs_all = [], [], []
    for N, f in sizes:
        Kcap = min(4096, min(N // L for L in f) // 2)
        delays = synth.draw_delays(N, 3, 6, rng)
        plan = sfft.Plan(N, Kcap, f, delays, precision="fp32", locate="ml", noise_auto=True)
        xs = []
        for i in range(8):
            K = int(min(Kcap, round(float(np.exp(rng.uniform(np.log(16), np.log(4096)))))))
            snr = None if rng.random() < 0.25 else float(rng.uniform(0.0, 40.0))
            p = synth.make_problem(N, f, K, seed=int(rng.integers(1 << 30)), delays=delays,
                                   mag=(1.0, 10.0), snr_db=snr)
            xs.append(torch.from_numpy(p.x.astype(np.complex64)).cuda())
        plans.append(plan)
        sigs.append(xs)
    n = max(1, int(rate * seconds))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
    which = rng.integers(0, len(sizes), size=n)
    srv = sfft.Server(hbm_budget=120 << 30, max_slots=16)
    for plan in plans:  # every plan's workspaces before the stream (none made mid-stream)
        srv.reserve(plan, 16)
    warm = []
    for j, plan in enumerate(plans):
        warm += [srv.submit(plan, sigs[j][i % 8], plan.empty_outputs()) for i in range(64)]
    srv.drain()
    del warm
    ring = 1024
    outs = [[plan.empty_outputs() for _ in range(ring)] for plan in plans]
    slot_ticket = [[0] * ring for _ in plans]
    tickets, kinds = [], []
    t0 = time.perf_counter()
    for i in range(n):
        while time.perf_counter() - t0 < arrivals[i]:
            pass
        j = int(which[i])
        k = i % ring
        if slot_ticket[j][k]:
            while srv.poll(slot_ticket[j][k])[0] == 1:  # ring slot still in use
                pass
        t = srv.submit(plans[j], sigs[j][i % 8], outs[j][k])
        slot_ticket[j][k] = t
        tickets.append(t)
        kinds.append(j)
    srv.drain()
    t1 = time.perf_counter()
    torch.cuda.synchronize()
    lat = np.array([srv.poll(t)[1] for t in tickets])
    srv.close()
    for plan in plans:
        plan.close()
    kinds = np.array(kinds)
    per_n = {str(sizes[j][0]): {"requests": int(np.sum(kinds == j)),
                               "p50_us": float(np.percentile(lat[kinds == j], 50)),
                               "p99_us": float(np.percentile(lat[kinds == j], 99))}
             for j in range(len(sizes)) if np.any(kinds == j)}
    return {"offered_rate": rate, "requests": n, "completed_rate": n / (t1 - t0),
            "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
            "per_N": per_n, "hbm_budget_gb": 120,
            "workload": "one request per signal, N from {9660, 124950, 2097024, 16776960}, "
                        "K log-uniform [16, 4096] (clamped), SNR U[0,40] dB or exact, "
                        "noise variance estimated per request"}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2011_05749_gb300 as sfft

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    S = args.batch
    N, K, R, f = CFG["N"], CFG["K"], CFG["R"], CFG["f"]
    nv = expected_noise_var()
    delays = plan_delays(args.seed)
    probs = problems(args.seed + rank, delays, N_DISTINCT)
    dev = torch.device("cuda", local)
    distinct = [torch.from_numpy(p.x.astype(np.complex64)).to(dev) for p in probs]
    xs = torch.empty((S, N), dtype=torch.complex64, device=dev)
    for i in range(S):
        xs[i].copy_(distinct[i % N_DISTINCT])
    plan_kw = dict(precision="fp32", locate="ml", noise_var=nv, max_batch=S,
                   max_tile=args.max_tile)
    tune_rate = None
    if not args.no_autotune and args.max_tile == 0:
        # schedule chosen by the library's autotuner on this batch (untimed)
        plan_kw, tune_rate = sfft.autotune(N, K, f, delays, list(xs), precision="fp32",
                                           locate="ml", noise_var=nv)
    plan = sfft.Plan(N, K, f, delays, **plan_kw)
    out = plan.empty_outputs("cuda", S)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        plan.execute_many(xs, out)
    barrier()
    plan.profile(reset=True)
    plan.set_profiling(True)
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        plan.execute_many(xs, out)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    plan.set_profiling(False)
    prof = plan.profile(reset=True)
    el_ms = ev0.elapsed_time(ev1)
    el_ms = max_over_ranks(el_ms, world)
    value = job_rate(S * args.steps, world, el_ms)
    infos = out[2].cpu().numpy()

    # dominant kernel: gather + prime-factor DFTs (bucketization), one launch per step
    bk = prof["bucketize"]
    bk_ms = bk["ms"] / max(bk["calls"], 1)
    sig_per_launch = S * args.steps / max(bk["calls"], 1)  # batches run as sub-batches
    esz = 8
    alg_bytes_sig = R * plan.num_bins * esz * 2  # samples read + bins written (complex64)
    achieved = sig_per_launch * alg_bytes_sig / (bk_ms / 1e3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    traffic_sig = kernel_traffic("bucketize_kernel<float,float>", TRAFFIC_SRC,
                                 "dram_bytes_per_signal")
    launches = sum(v["launches"] for v in prof.values())

    if args.timed_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "signals/s",
                              "timed_only": True, "phases": prof}, default=float), flush=True)
        return 0

    # per-signal latency of one request (sfft_execute, one signal per call)
    plan1 = sfft.Plan(N, K, f, delays, precision="fp32", locate="ml", noise_var=nv)
    o1 = plan1.empty_outputs("cuda")
    lat = []
    for i in range(10):
        plan1.execute(distinct[i % N_DISTINCT], o1)
    torch.cuda.synchronize()
    for i in range(200):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan1.execute(xs[(i * 7) % S], o1)
        b.record(stream)
        b.synchronize()
        lat.append(a.elapsed_time(b) * 1e3)
    lat.sort()

    # plain FP64 path: one signal per launch group, FP64 arithmetic throughout
    plan64 = sfft.Plan(N, K, f, delays, precision="fp64", locate="ml", noise_var=nv)
    o64 = [plan64.empty_outputs("cuda") for _ in range(N_DISTINCT)]
    for i in range(2):
        plan64.execute(distinct[i], o64[i])
    torch.cuda.synchronize()
    n64 = 16
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for i in range(n64):
        plan64.execute(distinct[i % N_DISTINCT], o64[i % N_DISTINCT])
    b.record(stream)
    torch.cuda.synchronize()
    fp64_rate = n64 / (a.elapsed_time(b) / 1e3)

    # accuracy of the batched FP32 results on the distinct signals
    idx32 = out[0].cpu().numpy()
    val32 = out[1].cpu().numpy()
    l2_vs64, sup_eq, l0_truth, l2_truth = [], 0, 0, []
    for i, p in enumerate(probs):
        n = int(infos[i, 0])
        i64, v64, f64 = (t.cpu().numpy() for t in o64[i])
        m = int(f64[0])
        same = n == m and np.array_equal(idx32[i, :n], i64[:m])
        sup_eq += int(same)
        if same:
            l2_vs64.append(np.linalg.norm(val32[i, :n] - v64[:m]) / np.linalg.norm(v64[:m]))
        l0_truth += len(set(idx32[i, :n].tolist()) ^ set(p.support.tolist()))
        if n == p.K and np.array_equal(idx32[i, :n], p.support):
            l2_truth.append(np.linalg.norm(val32[i, :n] - p.values) / np.linalg.norm(p.values))

    # end to end through host buffers: H2D of every input, D2H of every output per step
    e2e = None
    try:
        hx = [torch.empty(N, dtype=torch.complex64).pin_memory() for _ in range(S)]
        for i in range(S):
            hx[i].copy_(distinct[i % N_DISTINCT].cpu())
        hidx = [torch.zeros(K, dtype=torch.int64).pin_memory() for _ in range(S)]
        hval = [torch.zeros(K, dtype=torch.complex64).pin_memory() for _ in range(S)]
        hinf = torch.zeros((S, 4), dtype=torch.int32).pin_memory()
        sfft.execute_batch([plan] * S, hx, (hidx, hval, hinf))
        e_steps = max(3, min(args.steps, 10))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            sfft.execute_batch([plan] * S, hx, (hidx, hval, hinf))
        torch.cuda.synchronize()
        e_el = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": S * e_steps * world / e_el, "unit": "signals/s",
               "h2d_bytes_per_step": S * N * 8,
               "d2h_bytes_per_step": S * (K * 8 + K * 8) + S * 16,
               "path": "sfft_execute_batch with pinned host buffers (staged per launch group)"}
        assert np.array_equal(hidx[0].numpy()[:int(hinf[0, 0])], idx32[0, :int(infos[0, 0])])
    except Exception as exc:  # report, never fall back
        e2e = {"value": None, "unit": "signals/s", "error": repr(exc)[:200],
               "h2d_bytes_per_step": S * N * 8, "d2h_bytes_per_step": S * (K * 16 + 16)}

    # serving: Poisson arrivals into the continuous-batching server (sfft_submit/poll)
    serving = None
    try:
        serving = measure_serving(sfft, plan1, distinct, args.serve_rate, args.serve_seconds,
                                  args.seed)
    except Exception as exc:  # report, never fall back
        serving = {"error": repr(exc)[:200]}

    oneshot = None
    try:
        oneshot = measure_oneshot(sfft)
    except Exception as exc:  # report, never fall back
        oneshot = {"error": repr(exc)[:200]}
    locate_modes = None
    try:
        locate_modes = measure_locate_modes(sfft)
    except Exception as exc:  # report, never fall back
        locate_modes = {"error": repr(exc)[:200]}
    noise_auto = None
    try:
        noise_auto = measure_noise_auto(sfft)
    except Exception as exc:  # report, never fall back
        noise_auto = {"error": repr(exc)[:200]}
    dft_paths = None
    try:
        dft_paths = measure_dft_paths(sfft)
    except Exception as exc:  # report, never fall back
        dft_paths = {"error": repr(exc)[:200]}
    ml_paths = None
    try:
        ml_paths = measure_ml_paths(sfft)
    except Exception as exc:  # report, never fall back
        ml_paths = {"error": repr(exc)[:200]}
    dsfft = None
    try:
        dsfft = measure_dsfft(sfft)
    except Exception as exc:  # report, never fall back
        dsfft = {"error": repr(exc)[:200]}
    mix = None
    try:
        mix = measure_batched_mix(sfft)
    except Exception as exc:  # report, never fall back
        mix = {"error": repr(exc)[:200]}
    serving_mix = None
    try:
        serving_mix = measure_serving_mix(sfft, args.serve_rate, args.mix_seconds)
    except Exception as exc:  # report, never fall back
        serving_mix = {"error": repr(exc)[:200]}

    large = None
    large_sweep = None
    if not args.no_large:
        try:
            large = measure_large(sfft, hbm_peak)
        except Exception as exc:  # report, never fall back
            large = {"error": repr(exc)[:200]}
        try:
            large_sweep = measure_large_sweep(sfft)
        except Exception as exc:  # report, never fall back
            large_sweep = {"error": repr(exc)[:200]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, nsig, secs = oracle_rate(args.seed, args.cpu_seconds)
        cpu = {"value": rate, "unit": "signals/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{nsig} workload signals through the FP64 C oracle "
                         f"(naive DFT bucketization + peeling), {secs:.1f} s"}

    line = {
        "metric": METRIC, "value": value, "unit": "signals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: R-FFAST general sparse, N=127*128*129=2097024 "
                               "complex64, B=(16512,16383,16256), 8 delays/stage (0,1,6 random), "
                               "K=1000, |xhat|~U[1,10], SNR 20 dB; FP32 bulk, FP64 locate/fit",
                   "global_batch": S * world, "signals_per_step_per_gpu": S,
                   "distinct_signals": N_DISTINCT, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (S x 16.8 MB resident), no flush",
                   "schedule": {"decode_ctas": plan_kw.get("decode_ctas", 0),
                                "max_tile": plan_kw.get("max_tile", 0),
                                "autotuned": tune_rate is not None}},
        "latency_us": {"p50": lat[len(lat) // 2], "p99": lat[int(len(lat) * 0.99) - 1],
                       "path": "sfft_execute, one signal per call, device buffers"},
        "accuracy": {"support_equal_fp64_plain": f"{sup_eq}/{len(probs)}",
                     "rel_l2_vs_fp64_plain_max": max(l2_vs64) if l2_vs64 else None,
                     "l0_vs_truth_total": l0_truth,
                     "rel_l2_vs_truth_max": max(l2_truth) if l2_truth else None,
                     "status_incomplete": int(np.sum(infos[:, 1] == 2)),
                     "rounds_max": int(infos[:, 2].max())},
        "fp64_plain": {"value": fp64_rate, "unit": "signals/s",
                       "path": "FP64 arithmetic, one signal per sfft_execute"},
        "speedup_vs_fp64_plain": value / world / fp64_rate,
        "roofline": {"bound": "hbm", "kernel": "bucketize_kernel<float,float>",
                     "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "peak_source": peak_src,
                     "traffic": (traffic_sig * sig_per_launch if traffic_sig else None),
                     "alg_bytes_per_launch": sig_per_launch * alg_bytes_sig,
                     "signals_per_launch": sig_per_launch,
                     "avg_launch_ms": bk_ms,
                     # against the ~7.9 TB/s nominal HBM3e rate as well as the measured copy
                     "frac_of_nominal_7900": achieved / 7900.0,
                     # DRAM bytes the kernel moves (ncu traffic) over its time, and the share
                     # of them that are algorithmic (sector efficiency)
                     "dram_frac": ((traffic_sig * sig_per_launch) / (bk_ms / 1e3) / 1e9 / hbm_peak
                                   if traffic_sig else None),
                     "sector_efficiency": (alg_bytes_sig / traffic_sig if traffic_sig else None),
                     # the B-point DFTs in the FFTW convention, 5 B log2 B flops each
                     "dft_fftw_gflops": (sig_per_launch * R * sum(5.0 * (N // L) * np.log2(N // L)
                                                                  for L in f)
                                         / (bk_ms / 1e3) / 1e9)},
        "phases_ms_per_step": {k: v["ms"] / args.steps for k, v in prof.items()},
        "gpu_launches": launches,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "serving": serving,
        "large_signal": large,
        "large_signal_snr_sweep": large_sweep,
        "oneshot": oneshot,
        "locate_ml_vs_kay": locate_modes,
        "noise_auto": noise_auto,
        "dft_paths": dft_paths,
        "ml_paths": ml_paths,
        "dsfft": dsfft,
        "batched_mix": mix,
        "serving_mix": serving_mix,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line, default=float), flush=True)
    plan.close()
    plan1.close()
    plan64.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_only(args):
    """One block on its own, with few repetitions: the commands the ncu summaries use."""
    import paper_2011_05749_gb300 as sfft
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        peak = 6800.0
    if args.only == "large":
        out = measure_large(sfft, peak, reps=max(1, args.steps))
    elif args.only == "sweep":
        out = measure_large_sweep(sfft, reps=max(1, args.steps))
    elif args.only == "locate":
        out = measure_locate_modes(sfft, steps=max(1, args.steps), warmup=max(1, args.warmup))
    elif args.only == "noise":
        out = measure_noise_auto(sfft, steps=max(1, args.steps), warmup=max(1, args.warmup))
    elif args.only == "dsfft":
        out = measure_dsfft(sfft, steps=max(1, args.steps), warmup=max(1, args.warmup))
    elif args.only == "mix":
        out = measure_batched_mix(sfft, steps=max(1, args.steps), warmup=max(1, args.warmup))
    elif args.only == "serve":
        out = measure_serving_mix(sfft, args.serve_rate, args.mix_seconds)
    elif args.only == "dft":
        out = measure_dft_paths(sfft, steps=max(1, args.steps), warmup=max(1, args.warmup))
    elif args.only == "ml":
        out = measure_ml_paths(sfft, steps=max(1, args.steps), warmup=max(1, args.warmup))
    else:
        out = measure_oneshot(sfft, steps=max(1, args.steps), warmup=max(1, args.warmup))
    print(json.dumps(out, default=float), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
