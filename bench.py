#!/usr/bin/env python3
"""Throughput of the randomly shifted rank-1 lattice rule on one GB300.

Workload (the metric's single-sector configuration): d = 6 sector integrand
U^-2 F^-1 with U = c0 + 6 degree-1 and F = c0 + 12 degree-2 monomials
(coefficients U(0.1, 2), seed 0x5EED0002), baker transform, prime
n = 16777213, m = 32 shifts, FP32 evaluation with FP64 sums; the generating
vector comes from the library's CBC search (untimed).

One step = one full rule (all kernels of qmc_plan_execute: lattice kernel +
final pass, Eq. 2 and Eq. 3) with inputs resident on the device.  `value` is
lattice-point evaluations (n * m per step, all ranks) per second.  `e2e` is
the same metric through qmc_integrate with host inputs and a host result.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "lattice-point evals/sec & % FP pipe peak; time to 1e-8 rel err vs plain QMC"
UNIT = "evals/s"
WORKLOAD = "sector U^-2 F^-1, d=6, T_U=6, T_F=12, baker, n=16777213, m=32, FP32 eval / FP64 sums"

# Algorithmic FP32 flops per evaluation of this workload (FMA = 2): baker
# 2 per coordinate (12), U 2 per term (12), F 3 per degree-2 term (36),
# U^2 F 2, accumulate 1 -> 63, plus one reciprocal on the MUFU unit.
FLOPS_PER_EVAL = 63
# FP32 FMA peak: SMs x FP32 lanes per SM x 2 flops x maximum SM clock.  The
# SM count comes from the device and the maximum clock from nvidia-smi; 128
# FP32 lanes per SM is the sm_100-class figure.  The fallbacks are a GB300's
# 152 SMs and 2070 MHz.
LANES = 128
SMS_FALLBACK, SM_MAX_MHZ_FALLBACK = 152, 2070.0


def fp32_peak_tflops(sms: int, sm_max_mhz: float) -> float:
    return sms * LANES * 2 * sm_max_mhz * 1e6 / 1e12


def device_sms(torch, index: int) -> int:
    try:
        return int(torch.cuda.get_device_properties(index).multi_processor_count)
    except Exception:
        return SMS_FALLBACK


def device_max_sm_mhz(index: int) -> float:
    try:
        out = subprocess.run(["nvidia-smi", f"--id={index}", "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=30)
        return float(out.stdout.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        return SM_MAX_MHZ_FALLBACK

# DRAM traffic of the lattice kernel from one ncu capture of this workload;
# valid only while the kernel sources hash to KERNEL_SHA (else reported null).
NCU_TRAFFIC = {"kernel_sha": "b8f8063626ae2314", "bytes_per_launch": 89856}


# the sources the benchmark's lattice kernel is compiled from
KERNEL_SOURCES = ("device_common.cuh", "jit.cu", "qmc_internal.h", "rule_kernels.cuh")


def kernel_sha() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1811_11722_gb300", "csrc")
    for name in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks() -> dict:
    """The machine's measured peaks (HBM copy, cuBLAS bf16), else the fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return {"bf16_tflops": float(d["bf16_tflops"]), "hbm_gbs": float(d["hbm_gbs"]), "source": "of measured"}
    except (OSError, ValueError, KeyError):
        return {"bf16_tflops": 1900.0, "hbm_gbs": 6800.0, "source": "of fallback"}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def workload(rank: int, n=None):
    from paper_1811_11722_gb300 import inputs as I
    p = I.config2() if n is None else I.config2(n=n)
    if rank > 0:  # weak scaling: every rank integrates its own independent shifts
        p = I.with_shifts(p, p.m, I.SEED_BASE + 0x100 + rank)
    return p


def config_dict(world: int, n: int = 16777213):
    return {"workload": WORKLOAD if n == 16777213 else WORKLOAD.replace("16777213", str(n)) + " (profiling size)",
            "d": 6, "n": n, "m": 32, "transform": "baker",
            "integrand": "U^-2 F^-1 (T_U=6 deg-1, T_F=12 deg-2, + constants)", "precision": "FP32 eval, FP64 sums",
            "evals_per_step_per_gpu": n * 32, "parallelism": f"replicas x{world} (independent shifts)",
            "l2": "flushed between timed steps (256 MiB write); inputs are KB-sized descriptors in kernel "
                  "parameters, no HBM reads on the hot path"}


def cpu_baseline(p, g, budget_s: float = 12.0):
    """The oracle as it stands on all host cores over a leading run of lattice points."""
    import oracle
    threads = host_cores()
    S = 1 << 16
    t = time.perf_counter()
    oracle.rule_sums(p, g, 0, S, nthreads=threads)
    dt = time.perf_counter() - t
    S2 = int(min(p.n, max(S, S * budget_s / max(dt, 1e-3))))
    t = time.perf_counter()
    oracle.rule_sums(p, g, 0, S2, nthreads=threads)
    dt = time.perf_counter() - t
    return {"value": S2 * p.m / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"j in [0, {S2}) of n={p.n}, all m={p.m} shifts ({S2 * p.m} evals, FP64, {dt:.1f} s)"}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle (plain FP64 definition) on the same workload."""
    if rank != 0:
        return 0
    import oracle
    from oracle.cbc import cbc_fast
    from paper_1811_11722_gb300 import inputs as I
    p = workload(0)
    lat = os.path.join(ROOT, "tests", "golden", "lattices.json")
    table = json.load(open(lat))["g"] if os.path.exists(lat) else {}
    g = table.get(str(p.n), None)
    g = (g[: p.d] if g else list(cbc_fast(p.d, p.n, p.gamma)))
    threads = host_cores()
    S = 1 << 20
    for _ in range(args.warmup):
        oracle.rule_sums(p, g, 0, 1 << 14, nthreads=threads)
    times = []
    for s in range(args.steps):
        j0 = (s * S) % (p.n - S)
        t = time.perf_counter()
        oracle.rule_sums(p, g, j0, j0 + S, nthreads=threads)
        times.append(time.perf_counter() - t)
    tot = sum(times)
    val = S * p.m * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(world),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"each step: {S} consecutive lattice points x {p.m} shifts of the workload"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def device_time(fn, stream, reps=5):
    """Best device time (s) of fn() bracketed by CUDA events on `stream`."""
    import torch
    best = 1e30
    fn()
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b) / 1e3)
    return best


def extras(qmc, I, torch):
    """Measured peaks and the other configurations' throughput (one GPU)."""
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    out = {"peaks_measured": qmc.qmc_measure_peaks(sh)}
    dev_res = torch.zeros(qmc.RESULT_BYTES * 256, dtype=torch.uint8, device="cuda")
    # configuration 1 at the throughput size (FP64, separable exp, Korobov 3)
    p = I.config1(n=I.N_C1_THROUGHPUT)
    g = I.random_generating_vector(I.SplitMix64(1), p.d, p.n)
    plan = qmc.Plan(p.d, p.n, p.m, g, p.shifts, qmc.transform(p.transform, p.alpha), qmc.integrand_from_problem(p))
    t = device_time(lambda: plan.execute(out=dev_res, stream=sh), stream)
    out["c1_fp64_separable_d3_n16777213_m10"] = {"evals_per_s": p.n * p.m / t, "ms": 1e3 * t}
    plan.destroy()
    # configuration 4 (complex deformed, d=5, Korobov 3, n=4194301, m=20), FP64 and FP32
    p = I.config4()
    g = I.random_generating_vector(I.SplitMix64(4), p.d, p.n)
    for prec in ("fp64", "fp32"):
        plan = qmc.Plan(p.d, p.n, p.m, g, p.shifts, qmc.transform(p.transform, p.alpha),
                        qmc.integrand_from_problem(p, prec))
        t = device_time(lambda: plan.execute(out=dev_res, stream=sh), stream, reps=3)
        r = plan.execute()
        out[f"c4_deformed_d5_{prec}"] = {"evals_per_s": p.n * p.m / t, "ms": 1e3 * t,
                                         "mean": [r.mean[0], r.mean[1]], "err": [r.err[0], r.err[1]]}
        plan.destroy()
    c32, c64 = out["c4_deformed_d5_fp32"], out["c4_deformed_d5_fp64"]
    mag = abs(complex(*c64["mean"]))
    out["c4_fp32_vs_fp64"] = {"rel_diff": abs(complex(*c32["mean"]) - complex(*c64["mean"])) / mag,
                              "rel_err_estimate_fp64": abs(complex(*c64["err"])) / mag,
                              "rel_err_estimate_fp32": abs(complex(*c32["err"])) / mag}
    # precision of the FP32 evaluation on the benchmark's workload: |Q_FP32 - Q_FP64| / |Qbar|
    # against the Eq. (3) error estimate, same lattice and shifts
    p = I.config2()
    g = I.random_generating_vector(I.SplitMix64(2), p.d, p.n)
    t_ = qmc.transform(p.transform, p.alpha)
    r32, _ = qmc.qmc_integrate(p.d, p.n, p.m, g, p.shifts, t_, qmc.integrand_from_problem(p, "fp32"))
    r64, _ = qmc.qmc_integrate(p.d, p.n, p.m, g, p.shifts, t_, qmc.integrand_from_problem(p, "fp64"))
    out["c2_fp32_vs_fp64"] = {"rel_diff": abs(r32.mean[0] - r64.mean[0]) / abs(r64.mean[0]),
                              "rel_err_estimate_fp64": r64.err[0] / abs(r64.mean[0]),
                              "rel_err_estimate_fp32": r32.err[0] / abs(r32.mean[0])}
    # the same workload on the FP64 path (the paper's arithmetic): throughput and
    # the fraction of the measured FP64 FMA peak at the same 63 algorithmic flops
    # per evaluation
    plan = qmc.Plan(p.d, p.n, p.m, g, p.shifts, t_, qmc.integrand_from_problem(p, "fp64"))
    plan.tune(sh)
    t = device_time(lambda: plan.execute(out=dev_res, stream=sh), stream, reps=3)
    fp64_tf = FLOPS_PER_EVAL * p.n * p.m / t / 1e12
    pk64 = out["peaks_measured"]["fp64_tflops"]
    out["c2_fp64_path"] = {"evals_per_s": p.n * p.m / t, "ms": 1e3 * t, "plan": plan.describe(),
                           "algorithmic_tflops": fp64_tf, "fp64_peak_measured_tflops": pk64,
                           "frac_of_measured_fp64_peak": fp64_tf / pk64,
                           "note": "63 algorithmic flops per evaluation as on the FP32 path; whole step "
                                   "(lattice kernels and final pass) timed with CUDA events"}
    plan.destroy()
    # epsilon expansion of the configuration-2 integrand, U^(-2+eps) F^(-1-eps):
    # orders 0..2 and 0..5 from one pass (FP32 eval), against the plain rule
    p = I.config2()
    g = I.random_generating_vector(I.SplitMix64(2), p.d, p.n)
    t_ = qmc.transform(p.transform, p.alpha)
    f_ = qmc.integrand_from_problem(p, "fp32")
    for orders in (3, 6):
        plan = qmc.Plan(p.d, p.n, p.m, g, p.shifts, t_, f_, qmc.eps_spec(orders, 1.0, -1.0))
        t = device_time(lambda: plan.execute(out=dev_res, stream=sh), stream, reps=3)
        out[f"c2_eps_orders{orders}_fp32"] = {"evals_per_s": p.n * p.m / t, "ms": 1e3 * t,
                                              "order_evals_per_s": orders * p.n * p.m / t,
                                              "plan": plan.describe()}
        plan.destroy()
    # shared-lattice variant of configuration 3: 32 sectors of d = 6 on the
    # configuration-2 lattice, one fused sweep vs one tuned plan per sector
    probs = I.config3_shared()
    g = I.random_generating_vector(I.SplitMix64(2), 6, probs[0].n)
    fs = [qmc.integrand_from_problem(q) for q in probs]
    tb = qmc.transform("baker")
    t0 = time.perf_counter()
    mp = qmc.MultiPlan(6, probs[0].n, probs[0].m, g, probs[0].shifts, tb, fs)
    build_s = time.perf_counter() - t0
    t = device_time(lambda: mp.execute(out=dev_res, stream=sh), stream, reps=3)
    singles = [qmc.Plan(6, q.n, q.m, g, q.shifts, tb, f) for q, f in zip(probs, fs)]
    for pl in singles:
        pl.tune(sh)
    t1 = device_time(lambda: [pl.execute(out=dev_res, stream=sh) for pl in singles], stream, reps=2)
    evals = sum(q.n * q.m for q in probs)
    out["c3_shared_lattice_32_sectors_d6"] = {
        "evals": evals, "evals_per_s_fused": evals / t, "ms_fused": 1e3 * t, "ms_one_plan_per_sector": 1e3 * t1,
        "speedup_vs_one_plan_per_sector": t1 / t, "plan_build_s": build_s, "launches": mp.launches(),
        "workload": "32 sectors, d=6, T_U~U{4..10}, T_F~U{6..20}, baker, n=16777213, m=16, FP32 eval"}
    mp.destroy()
    for pl in singles:
        pl.destroy()
    # configuration 3: 256 sectors in one graph replay vs the same plans one after another,
    # each sector on the CBC vector of its table prime (d = 8, restricted to its d)
    sect = I.config3()
    cbc = cbc8(qmc, I, {q.n for q in sect})
    gs = [cbc[q.n][:q.d].copy() for q in sect]
    tuples = [(q.d, q.n, q.m, gg, q.shifts, qmc.transform(q.transform, q.alpha), qmc.integrand_from_problem(q))
              for q, gg in zip(sect, gs)]
    evals = sum(q.n * q.m for q in sect)
    t0 = time.perf_counter()
    bp = qmc.BatchPlan(tuples)
    build_s = time.perf_counter() - t0
    w = bp.tune(sh)
    t = device_time(lambda: bp.execute(out=dev_res, stream=sh), stream, reps=3)
    plans = [qmc.Plan(*tt) for tt in tuples]
    t1 = device_time(lambda: [pl.execute(out=dev_res, stream=sh) for pl in plans], stream, reps=2)
    out["c3_batch_256_sectors"] = {"evals": evals, "evals_per_s_graph": evals / t, "ms_graph": 1e3 * t,
                                   "ms_one_by_one": 1e3 * t1, "speedup_vs_one_by_one": t1 / t,
                                   "work_per_cta": w, "plan_build_s": build_s, "launches": bp.launches(),
                                   "note": "CBC generating vectors (product weights 1/i^2, d = 8, restricted)"}
    for pl in plans:
        pl.destroy()
    # the same 256 sectors as one persistent launch: work items from a device
    # counter, each dispatched to its sector's run-time specialised code
    t0 = time.perf_counter()
    pp = qmc.BatchPlan(tuples, persistent=True)
    pbuild_s = time.perf_counter() - t0
    pw = pp.tune(sh)
    tpp = device_time(lambda: pp.execute(out=dev_res, stream=sh), stream, reps=3)
    rp = [r.as_dict() for r in pp.execute()]
    rg = [r.as_dict() for r in bp.execute()]
    out["c3_batch_256_sectors_persistent"] = {
        "evals_per_s": evals / tpp, "ms": 1e3 * tpp, "points_per_item": pw, "plan_build_s": pbuild_s,
        "launches": pp.launches(), "ms_graph": 1e3 * t, "graph_plan_build_s": build_s,
        "max_rel_diff_vs_graph": max(abs(a["mean"][0] - b["mean"][0]) / abs(b["mean"][0]) for a, b in zip(rp, rg)),
        "plan": pp.describe()}
    pp.destroy()
    # the generic persistent kernel (no run-time compilation: every sector's
    # dense coefficient slots staged in shared memory), tuned the same way
    # the same batch under Korobov 3 (the transform of the walks to 1e-8)
    sect_k = I.config3(transform="korobov", alpha=3)
    tuples_k = [(q.d, q.n, q.m, gg, q.shifts, qmc.transform(q.transform, q.alpha), qmc.integrand_from_problem(q))
                for q, gg in zip(sect_k, gs)]
    bk = qmc.BatchPlan(tuples_k)
    wk = bk.tune(sh)
    tk = device_time(lambda: bk.execute(out=dev_res, stream=sh), stream, reps=3)
    out["c3_batch_256_sectors_korobov3"] = {"evals_per_s_graph": evals / tk, "ms_graph": 1e3 * tk, "work_per_cta": wk}
    bk.destroy()
    saved_env = os.environ.get("QMC_PERSIST_JIT")
    os.environ["QMC_PERSIST_JIT"] = "0"
    try:
        pg = qmc.BatchPlan(tuples, persistent=True)
        pgw = pg.tune(sh)
        tpg = device_time(lambda: pg.execute(out=dev_res, stream=sh), stream, reps=3)
        out["c3_batch_256_sectors_persistent_generic"] = {"evals_per_s": evals / tpg, "ms": 1e3 * tpg,
                                                          "points_per_item": pgw, "plan": pg.describe()}
        pg.destroy()
    finally:
        if saved_env is None:
            del os.environ["QMC_PERSIST_JIT"]
        else:
            os.environ["QMC_PERSIST_JIT"] = saved_env
    bp.destroy()
    # control-variate estimator Q[f - g] + int g (surrogate contracted on tensor
    # cores) on the configuration-5 integrand at n = 16777213, m = 16: one fit
    # (2000 Adam steps, pilot n = 65537), then the estimator per transform
    # beside the plain rule on the same points
    p = I.config5(n=16777213, m=16)
    g = I.random_generating_vector(I.SplitMix64(5), p.d, p.n)
    gp = qmc.qmc_make_lattice(p.d, I.N_PILOT, p.gamma)
    f_ = qmc.integrand_from_problem(p, "fp32")
    cfg = qmc.qmc_cv_config()
    cfg.R, cfg.K, cfg.freq_step, cfg.steps, cfg.lr, cfg.seed = 16, 32, 1, 2000, 1e-2, 7
    a, _ = qmc.qmc_cv_train(p.d, I.N_PILOT, gp, I.make_shifts(I.SplitMix64(54), 1, p.d)[0], qmc.transform("none"),
                            f_, cfg, stream=sh)
    # the estimator's two engines: the contraction as warp-level mma.sync
    # (cv_tc_kernel) and as tcgen05.mma with the basis in tensor memory
    # (cv_tc5_kernel), the same arithmetic to FP32 accuracy
    saved_engine = os.environ.get("QMC_CV_ENGINE")
    for name, tt in (("none", qmc.transform("none")), ("korobov3", qmc.transform("korobov", 3))):
        plan = qmc.Plan(p.d, p.n, p.m, g, p.shifts, tt, f_)
        tp = device_time(lambda: plan.execute(out=dev_res, stream=sh), stream, reps=3)
        plan.destroy()
        row = {}
        for engine in ("mma", "tcgen05"):
            os.environ["QMC_CV_ENGINE"] = engine
            res = {}
            t = device_time(lambda: res.update(r=qmc.qmc_integrate_cv(p.d, p.n, p.m, g, p.shifts, tt, f_, cfg, a,
                                                                      stream=sh)[0]), stream, reps=3)
            r = res["r"]
            executed = p.d * 2048 * p.n * p.m / t / 1e12
            if engine == "mma":
                peak = out["peaks_measured"]["mma_sync_tf32_tflops"]  # the instruction this kernel issues
                src = ("measured warp-level TF32 mma.sync m16n8k8 throughput on this GPU (qmc_measure_peaks); "
                       "achieved counts both MMAs (basis head and remainder)")
            else:
                peak = measured_peaks()["bf16_tflops"] * 1.1 / 2.25
                src = ("dense TF32 tensor peak taken as the measured cuBLAS BF16 peak x 1.1/2.25 (nominal ratio); "
                       "achieved counts both MMAs (basis head and remainder)")
            row[engine] = {
                "evals_per_s": p.n * p.m / t, "ms": 1e3 * t, "cost_vs_plain_rule": t / tp,
                "roofline": {"bound": "tensor", "achieved": executed, "peak": peak, "unit": "TFLOP/s",
                             "frac": executed / peak,
                             "algorithmic_tflops": p.d * 2 * 16 * 31 * p.n * p.m / t / 1e12, "peak_source": src},
                "err_cv": r.err[0], "err_plain_same_points": r.err[1], "mean_cv": r.mean[0]}
        out[f"c5_cv_estimator_{name}"] = dict(
            row, plain_rule_ms=1e3 * tp, speedup_tcgen05_vs_mma=row["mma"]["ms"] / row["tcgen05"]["ms"],
            gain_same_points=row["mma"]["err_plain_same_points"] / row["mma"]["err_cv"],
            note="2048 TF32 MMA flops per point and dimension: head and remainder of the 32-degree basis x 16 ranks")
    if saved_engine is None:
        os.environ.pop("QMC_CV_ENGINE", None)
    else:
        os.environ["QMC_CV_ENGINE"] = saved_engine
    # gain of the control variate per surrogate design and transform, from the
    # same points (n = 1048573, m = 16): plain error / control-variate error.
    # band > 0 holds the cosine degrees k >= band at zero (band-limited fit)
    gains = {}
    n1 = 1048573
    g1 = qmc.qmc_make_lattice(p.d, n1, p.gamma)
    for band in (0, 4, 8, 16):
        cfg.band = band
        a, losses = qmc.qmc_cv_train(p.d, I.N_PILOT, gp, I.make_shifts(I.SplitMix64(54), 1, p.d)[0],
                                     qmc.transform("none"), f_, cfg, stream=sh)
        row = {"loss": float(losses[1])}
        for name, tt in (("none", qmc.transform("none")), ("baker", qmc.transform("baker")),
                         ("korobov3", qmc.transform("korobov", 3))):
            r, _ = qmc.qmc_integrate_cv(p.d, n1, p.m, g1, p.shifts, tt, f_, cfg, a, stream=sh)
            row[name] = {"gain": r.err[1] / r.err[0], "err_cv": r.err[0], "err_plain": r.err[1]}
        gains[f"band{band}"] = row
    cfg.band = 0
    out["c5_cv_gain_by_band_and_transform"] = dict(gains, n=n1, m=p.m,
                                                   note="same points; gain = plain Eq. (3) error / control-variate "
                                                        "error; band 0 = all 32 cosine degrees fitted")
    return out


def _short(cfg):
    """A copy of a control-variate config with 5 Adam steps (warm-up runs)."""
    import copy
    c = copy.copy(cfg)
    c.steps = 5
    return c


_CBC8 = {}  # n -> the d = 8 CBC vector (product weights 1/i^2); its first d components are the d-dim one


def cbc8(qmc, I, ns):
    """CBC vectors for the primes ns (host precompute, computed once per n)."""
    from concurrent.futures import ThreadPoolExecutor
    need = sorted(n for n in ns if n not in _CBC8)
    with ThreadPoolExecutor(max_workers=4) as ex:
        for n, g in zip(need, ex.map(lambda n: qmc.qmc_make_lattice(8, n, I.product_weights(8)), need)):
            _CBC8[n] = g
    return _CBC8


def c3_time_to_tolerance(qmc, I, sh, tol, ladder_max=11863279, start="own"):
    """The 256 Korobov-3 sectors summed to tol.  Every sector starts on its own
    table prime (start="own") or on the ladder's first prime (start="ladder")
    and climbs the prime ladder (up to ladder_max) while its error is above
    its share tol |sum| / sqrt(256) of the tolerance on the sum.  Batched:
    qmc_integrate_batch_to_tolerance, one batched launch per pass.  One by
    one: the same walk with one qmc_integrate call per sector and level.  CBC
    vectors (d = 8, restricted to each sector's d) are host precomputes and
    not timed."""
    import numpy as np
    sect = I.config3(transform="korobov", alpha=3)
    S = len(sect)
    ladder = [n for n in I.ladder_primes() if min(q.n for q in sect) < n <= ladder_max]
    if start == "ladder":
        n0 = [ladder[0]] * S
        ladder = ladder[1:]
    else:
        n0 = [q.n for q in sect]
    cbc = cbc8(qmc, I, set(ladder) | set(n0))
    fs = [qmc.integrand_from_problem(q) for q in sect]
    ts = [qmc.transform(q.transform, q.alpha) for q in sect]
    tuples = [(q.d, n, q.m, cbc[n][:q.d].copy(), q.shifts, t_, f_) for q, n, t_, f_ in zip(sect, n0, ts, fs)]
    ladder_n = np.array(ladder, dtype=np.uint64)
    ladder_g = np.stack([cbc[n] for n in ladder]).astype(np.uint64)
    # run-time compilation of every sector's kernel (independent of n): a precompute
    g1009 = qmc.qmc_make_lattice(8, 1009, I.product_weights(8))
    qmc.qmc_integrate_batch([(q.d, 1009, q.m, g1009[:q.d].copy(), q.shifts, t_, f_)
                             for q, t_, f_ in zip(sect, ts, fs)], stream=sh)
    res = {}
    # batched: the library's walk (best of 3 runs; the first also warms the allocator)
    walls = []
    for _ in range(3):
        t0 = time.perf_counter()
        rs, lv, passes, reached = qmc.qmc_integrate_batch_to_tolerance(tuples, ladder_n, ladder_g, tol,
                                                                       qmc.WALK_SUM, stream=sh)
        walls.append(time.perf_counter() - t0)
    mean = np.array([r.mean[0] for r in rs])
    err = np.array([r.err[0] for r in rs])
    ns = [n if l < 0 else ladder[l] for n, l in zip(n0, lv)]
    evals = 0
    for q, n, l in zip(sect, n0, lv):  # every lattice a sector visited
        evals += n * q.m + sum(ladder[k] * q.m for k in range(int(np.searchsorted(ladder_n, n, "right")), l + 1))
    total, total_err = mean.sum(), math.sqrt(float(np.sum(err ** 2)))
    res["batched"] = {"rel_err": float(total_err / abs(total)), "sum": float(total), "wall_s": min(walls),
                      "wall_s_runs": walls, "passes": int(passes), "evals": int(evals), "reached": bool(reached),
                      "largest_n": int(max(ns)), "api": "qmc_integrate_batch_to_tolerance"}
    # the same walk with QMC_WALK_JUMP: a sector moves up as far as an error
    # falling like n^-6 would need, skipping the lattices in between
    walls = []
    for _ in range(3):
        t0 = time.perf_counter()
        rj, lvj, pj, okj = qmc.qmc_integrate_batch_to_tolerance(tuples, ladder_n, ladder_g, tol,
                                                                qmc.WALK_SUM | qmc.WALK_JUMP, stream=sh)
        walls.append(time.perf_counter() - t0)
    mj = np.array([r.mean[0] for r in rj])
    ej = np.array([r.err[0] for r in rj])
    res["batched_jump"] = {"rel_err": float(math.sqrt(float(np.sum(ej ** 2))) / abs(mj.sum())), "sum": float(mj.sum()),
                           "wall_s": min(walls), "wall_s_runs": walls, "passes": int(pj), "reached": bool(okj),
                           "largest_n": int(max(n if l < 0 else ladder[l] for n, l in zip(n0, lvj))),
                           "speedup_vs_batched": res["batched"]["wall_s"] / min(walls),
                           "api": "qmc_integrate_batch_to_tolerance, QMC_WALK_JUMP"}
    # one by one: the same decisions, one rule call per sector and level
    steps = [[n] + [m_ for m_ in ladder if m_ > n] for n in n0]
    level = [0] * S
    mean = np.zeros(S)
    err = np.zeros(S)
    todo = list(range(S))
    wall, passes, evals = 0.0, 0, 0
    while True:
        t0 = time.perf_counter()
        rs = [qmc.qmc_integrate(sect[i].d, steps[i][level[i]], sect[i].m, cbc[steps[i][level[i]]][:sect[i].d].copy(),
                                sect[i].shifts, ts[i], fs[i], stream=sh)[0] for i in todo]
        wall += time.perf_counter() - t0
        passes += 1
        for i, r in zip(todo, rs):
            mean[i], err[i] = r.mean[0], r.err[0]
            evals += steps[i][level[i]] * sect[i].m
        total, total_err = mean.sum(), math.sqrt(float(np.sum(err ** 2)))
        if total_err <= tol * abs(total):
            break
        share = tol * abs(total) / math.sqrt(S)
        todo = [i for i in range(S) if err[i] > share and level[i] + 1 < len(steps[i])]
        if not todo:
            break
        for i in todo:
            level[i] += 1
    res["one_by_one"] = {"rel_err": float(total_err / abs(total)), "sum": float(total), "wall_s": wall,
                         "passes": passes, "evals": int(evals), "reached": bool(total_err <= tol * abs(total)),
                         "largest_n": int(max(steps[i][level[i]] for i in range(S))), "api": "qmc_integrate per call"}
    res["batched"]["speedup_vs_one_by_one"] = res["one_by_one"]["wall_s"] / res["batched"]["wall_s"]
    res["batched_jump"]["speedup_vs_one_by_one"] = res["one_by_one"]["wall_s"] / res["batched_jump"]["wall_s"]
    tag = "c3_256_sectors_korobov3_sum" + ("_from_ladder_start" if start == "ladder" else "")
    return {f"{tag}_batched": res["batched"], f"{tag}_batched_jump": res["batched_jump"],
            f"{tag}_one_by_one": res["one_by_one"]}


def c3_time_to_tolerance_embedded(qmc, I, sh, tol, log2_n0=16, log2_nmax=24):
    """The 256 Korobov-3 sectors summed to tol on embedded base-2 lattices:
    every sector starts with 2^log2_n0 points and doubles (up to
    2^log2_nmax) while its error is above its share tol |sum| / sqrt(256);
    a doubling evaluates only the new half of the points.  Batched:
    qmc_integrate_batch_extensible, one batched launch per pass.  One by one:
    the same walk with one qmc_integrate call per sector and pass on the new
    points, per-shift values averaged and combined (qmc_combine_shifts) on
    the host.  The embedded vector (d = 8, restricted to each sector's d) is
    a host precompute and not timed."""
    import numpy as np
    sect = I.config3(transform="korobov", alpha=3)
    S = len(sect)
    levels = log2_nmax - log2_n0
    g = qmc.qmc_make_lattice_embedded(8, log2_n0, log2_nmax, I.product_weights(8))
    n0 = 1 << log2_n0
    fs = [qmc.integrand_from_problem(q) for q in sect]
    ts = [qmc.transform(q.transform, q.alpha) for q in sect]
    tuples = [(q.d, n0, q.m, g[:q.d] % np.uint64(n0), q.shifts, t_, f_) for q, t_, f_ in zip(sect, ts, fs)]
    qmc.qmc_integrate_batch(tuples, stream=sh)  # run-time compilation of every sector's kernel: a precompute
    res = {}
    walls = []
    for _ in range(3):
        t0 = time.perf_counter()
        rs, lv, passes, reached = qmc.qmc_integrate_batch_extensible(tuples, levels, g, tol, qmc.WALK_SUM, stream=sh)
        walls.append(time.perf_counter() - t0)
    mean = np.array([r.mean[0] for r in rs])
    err = np.array([r.err[0] for r in rs])
    total, total_err = mean.sum(), math.sqrt(float(np.sum(err ** 2)))
    res["batched"] = {"rel_err": float(total_err / abs(total)), "sum": float(total), "wall_s": min(walls),
                      "wall_s_runs": walls, "passes": int(passes), "reached": bool(reached),
                      "evals": int(sum((n0 << int(l)) * q.m for q, l in zip(sect, lv))),
                      "largest_n": int(n0 << int(max(lv))), "api": "qmc_integrate_batch_extensible"}
    walls = []
    for _ in range(3):
        t0 = time.perf_counter()
        rj, lvj, pj, okj = qmc.qmc_integrate_batch_extensible(tuples, levels, g, tol, qmc.WALK_SUM | qmc.WALK_JUMP,
                                                              stream=sh)
        walls.append(time.perf_counter() - t0)
    mj = np.array([r.mean[0] for r in rj])
    ej = np.array([r.err[0] for r in rj])
    res["batched_jump"] = {"rel_err": float(math.sqrt(float(np.sum(ej ** 2))) / abs(mj.sum())), "sum": float(mj.sum()),
                           "wall_s": min(walls), "wall_s_runs": walls, "passes": int(pj), "reached": bool(okj),
                           "largest_n": int(n0 << int(max(lvj))),
                           "speedup_vs_batched": res["batched"]["wall_s"] / min(walls),
                           "api": "qmc_integrate_batch_extensible, QMC_WALK_JUMP"}
    # one by one: the same decisions, one rule call per sector and pass
    size = [n0] * S
    dbl = [0] * S
    q = [None] * S
    mean = np.zeros(S)
    err = np.zeros(S)
    todo = list(range(S))
    wall, passes, evals = 0.0, 0, 0
    while True:
        t0 = time.perf_counter()
        for i in todo:
            p, n = sect[i], size[i]
            shifts = p.shifts
            if passes:
                v = p.shifts + (g[:p.d] % np.uint64(2 * n)).astype(np.float64) / float(2 * n)
                shifts = np.where(v >= 1.0, v - 1.0, v)
            _, ps = qmc.qmc_integrate(p.d, n, p.m, g[:p.d] % np.uint64(n), shifts, ts[i], fs[i], stream=sh,
                                      want_per_shift=True)
            if passes:
                q[i] = 0.5 * (q[i] + ps)
                size[i] *= 2
                dbl[i] += 1
            else:
                q[i] = ps
            r = qmc.qmc_combine_shifts(q[i])
            mean[i], err[i] = r.mean[0], r.err[0]
            evals += n * p.m
        wall += time.perf_counter() - t0
        passes += 1
        total, total_err = mean.sum(), math.sqrt(float(np.sum(err ** 2)))
        if total_err <= tol * abs(total):
            break
        share = tol * abs(total) / math.sqrt(S)
        todo = [i for i in range(S) if err[i] > share and dbl[i] < levels]
        if not todo:
            break
    res["one_by_one"] = {"rel_err": float(total_err / abs(total)), "sum": float(total), "wall_s": wall,
                         "passes": passes, "evals": int(evals), "reached": bool(total_err <= tol * abs(total)),
                         "largest_n": int(max(size)), "api": "qmc_integrate per call"}
    res["batched"]["speedup_vs_one_by_one"] = res["one_by_one"]["wall_s"] / res["batched"]["wall_s"]
    res["batched_jump"]["speedup_vs_one_by_one"] = res["one_by_one"]["wall_s"] / res["batched_jump"]["wall_s"]
    tag = "c3_256_sectors_korobov3_sum_embedded"
    return {f"{tag}_batched": res["batched"], f"{tag}_batched_jump": res["batched_jump"],
            f"{tag}_one_by_one": res["one_by_one"]}


def time_to_tolerance(qmc, I, torch, tol=1e-8, budget_s=60.0):
    """Wall time until err/|Qbar| <= tol walking the lattice ladder (largest prime
    <= 2^(e/2)), each level a fresh rule with its CBC vector; lattice
    construction is a precompute and is not timed, everything else is.
    Compares the plain rule on the prime ladder, the embedded base-2 lattices
    (each level adds only the new half of the points), the sum of 32 sectors as
    one fused sweep against one rule per sector, and the control variate
    (training included)."""
    import numpy as np
    out = {}
    ladder = [n for n in I.ladder_primes() if n >= 65521]
    sh = torch.cuda.current_stream().cuda_stream

    class lattices(dict):
        """CBC vectors built on first use (host precompute, not timed)."""

        def __init__(self, d, gamma):
            super().__init__()
            self.d, self.gamma = d, gamma

        def __missing__(self, n):
            self[n] = qmc.qmc_make_lattice(self.d, n, self.gamma)
            return self[n]

    caches = {}

    def lat_for(p):
        if p.d not in caches:
            caches[p.d] = lattices(p.d, p.gamma)
        return caches[p.d]

    # plain rule on the single-sector workload and on the d=8 Korobov-3 sector
    for name, p in (("sector_d6_baker_fp32", I.config2()), ("sector_d8_korobov3_fp32", I.config5())):
        lat = lat_for(p)
        f = qmc.integrand_from_problem(p, "fp32")
        t = qmc.transform(p.transform, p.alpha)
        # the integrand's kernel is compiled at run time on first use: a precompute, like the lattices
        qmc.qmc_integrate(p.d, ladder[0], p.m, lat[ladder[0]], p.shifts, t, f, stream=sh)
        wall, rec = 0.0, None
        for n in ladder:
            gn = lat[n]
            t0 = time.perf_counter()
            r, _ = qmc.qmc_integrate(p.d, n, p.m, gn, p.shifts, t, f, stream=sh)
            wall += time.perf_counter() - t0
            rel = r.err[0] / abs(r.mean[0])
            rec = {"n": n, "rel_err": rel, "mean": r.mean[0], "wall_s": wall}
            if rel <= tol or wall > budget_s:
                break
        rec["reached"] = rec["rel_err"] <= tol
        out[name] = rec
        # embedded lattices: n = 2^16, 2^17, ... each level adds only the new half of the points
        ge = qmc.qmc_make_lattice_embedded(p.d, 16, 25, p.gamma)  # precompute (all odd candidates)
        t0 = time.perf_counter()
        r, lvl, _, ok = qmc.qmc_integrate_extensible(p.d, 16, 10, ge, p.m, p.shifts, t, f, tol, stream=sh)
        out[name + "_embedded"] = {"n": 1 << (16 + lvl), "rel_err": r.err[0] / abs(r.mean[0]), "mean": r.mean[0],
                                   "wall_s": time.perf_counter() - t0, "reached": bool(ok),
                                   "points_evaluated_per_shift": 1 << (16 + lvl)}
    # integrand-sum batching: the sum of the 32 d = 6 sectors of the shared-lattice
    # variant of configuration 3 (Korobov 3), one fused sweep per level
    # (qmc_integrate_multi) against one rule per sector (qmc_integrate, per-shift
    # values summed, Eq. (3) by qmc_combine_shifts); the same points either way
    probs = I.config3_shared(transform="korobov", alpha=3)
    fs = [qmc.integrand_from_problem(q) for q in probs]
    sh6, m6, tb = probs[0].shifts, probs[0].m, qmc.transform("korobov", 3)
    lat = lat_for(probs[0])
    n0 = ladder[0]
    qmc.qmc_integrate_multi(6, n0, m6, lat[n0], sh6, tb, fs, stream=sh)  # run-time compilation: a precompute
    for f_ in fs:
        qmc.qmc_integrate(6, n0, m6, lat[n0], sh6, tb, f_, stream=sh)
    for mode in ("fused", "one_rule_per_sector"):
        wall, rec = 0.0, None
        for n in ladder:
            gn = lat[n]
            t0 = time.perf_counter()
            if mode == "fused":
                r = qmc.qmc_integrate_multi(6, n, m6, gn, sh6, tb, fs, stream=sh)[0][-1]
            else:
                tot = np.zeros((m6, 2))
                for f_ in fs:
                    tot += qmc.qmc_integrate(6, n, m6, gn, sh6, tb, f_, stream=sh, want_per_shift=True)[1]
                r = qmc.qmc_combine_shifts(tot)
            wall += time.perf_counter() - t0
            rel = r.err[0] / abs(r.mean[0])
            rec = {"n": n, "rel_err": rel, "mean": r.mean[0], "wall_s": wall}
            if rel <= tol or wall > budget_s:
                break
        rec["reached"] = rec["rel_err"] <= tol
        out[f"sum_32_sectors_d6_korobov3_fp32_{mode}"] = rec
    # configuration 3's 256 sectors (Korobov 3 variant), their sum to 1e-8
    # relative error: every sector walks its own ladder (its table prime, then
    # the ladder primes above it, CBC vectors from the library, untimed).  A
    # pass refines only the sectors whose Eq. (3) error exceeds their share
    # tol |sum| / sqrt(256) of the total's budget; the total error is the
    # quadrature sum of the sectors'.  Batched: the library's walk
    # (qmc_integrate_batch_to_tolerance, one batched launch per pass); one by
    # one: one qmc_integrate call per refined sector.  Same lattices, shifts
    # and decisions.
    out.update(c3_time_to_tolerance(qmc, I, sh, tol))
    # the same sum with every sector started on the ladder's first prime: the
    # walk then chooses each sector's n from the bottom of the ladder
    out.update(c3_time_to_tolerance(qmc, I, sh, tol, start="ladder"))
    # the same sum on embedded base-2 lattices: every sector starts at 2^16
    # points and doubles, each doubling evaluating only the new half
    out.update(c3_time_to_tolerance_embedded(qmc, I, sh, tol))
    lad = out.get("c3_256_sectors_korobov3_sum_from_ladder_start_batched")
    if lad:
        emb = out["c3_256_sectors_korobov3_sum_embedded_batched"]
        emb["speedup_vs_prime_ladder_batched"] = lad["wall_s"] / emb["wall_s"]
    # control variate on the d=8 sector (pilot n=65537, 2000 Adam steps).  The
    # library's judged walk (qmc_integrate_cv_to_tolerance): the first ladder
    # lattice is the pilot where the control variate and the plain rule meet at
    # equal cost; the loser is dropped.  Fit included in the wall time.  Beside
    # it, the control variate forced through every level (no judge).
    p = I.config5()
    lat = lat_for(p)
    gp = qmc.qmc_make_lattice(p.d, I.N_PILOT, p.gamma)
    f = qmc.integrand_from_problem(p, "fp32")
    t = qmc.transform(p.transform, p.alpha)
    pilot_shift = I.make_shifts(I.SplitMix64(54), 1, p.d)[0]
    # the ladder up to one level past the plain walk's stopping point
    stop = ladder.index(out["sector_d8_korobov3_fp32"]["n"]) + 2
    ns = np.array(ladder[:stop], dtype=np.uint64)
    gs = np.concatenate([lat[n] for n in ladder[:stop]])
    for band in (0, 8):
        cfg = qmc.qmc_cv_config()
        cfg.R, cfg.K, cfg.freq_step, cfg.steps, cfg.lr, cfg.band, cfg.seed = 16, 32, 1, 2000, 1e-2, band, 7
        # first-use work outside the timing: one short fit and one estimator call
        a0, _ = qmc.qmc_cv_train(p.d, I.N_PILOT, gp, pilot_shift, t, f, _short(cfg))
        qmc.qmc_integrate_cv(p.d, ladder[0], p.m, lat[ladder[0]], p.shifts, t, f, cfg, a0, stream=sh)
        t0 = time.perf_counter()
        a, losses = qmc.qmc_cv_train(p.d, I.N_PILOT, gp, pilot_shift, t, f, cfg)
        train_s = time.perf_counter() - t0
        r, lvl, mode, judge, ok = qmc.qmc_integrate_cv_to_tolerance(p.d, ns, gs, p.m, p.shifts, t, f, cfg, a, tol,
                                                                     stream=sh)
        wall = time.perf_counter() - t0
        out[f"sector_d8_korobov3_cv_band{band}_judged"] = {
            "n": int(ns[lvl]), "rel_err": r.err[0] / abs(r.mean[0]), "mean": r.mean[0], "wall_s": wall,
            "train_s": train_s, "reached": bool(ok), "kept": "control variate" if mode == 1 else "plain rule",
            "pilot": dict(judge, n=int(ladder[0])), "loss": [float(losses[0]), float(losses[1])],
            "plain_ladder_wall_s": out["sector_d8_korobov3_fp32"]["wall_s"],
            "speedup_vs_plain_ladder": out["sector_d8_korobov3_fp32"]["wall_s"] / wall}
        if band == 0:  # the control variate forced through every level, for comparison
            wall, rec = train_s, None
            for n in ladder:
                gn = lat[n]
                t1 = time.perf_counter()
                rr, _ = qmc.qmc_integrate_cv(p.d, n, p.m, gn, p.shifts, t, f, cfg, a, stream=sh)
                wall += time.perf_counter() - t1
                rel = rr.err[0] / abs(rr.mean[0])
                rec = {"n": n, "rel_err": rel, "plain_rel_err_same_points": rr.err[1] / abs(rr.mean[1]),
                       "mean": rr.mean[0], "wall_s": wall, "train_s": train_s}
                if rel <= tol or wall > budget_s:
                    break
            rec["reached"] = rec["rel_err"] <= tol
            out["sector_d8_korobov3_cv_forced"] = rec
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner (profiler captures)")
    ap.add_argument("--no-extras", action="store_true", help="skip the other configurations' throughput")
    ap.add_argument("--no-time-to-tol", action="store_true",
                    help="skip the wall time to 1e-8 relative error (plain, embedded lattices, control variate)")
    ap.add_argument("--n", type=int, default=None,
                    help="smaller prime lattice size, for profiler captures only (changes the workload)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1811_11722_gb300 import build, qmc
    build.build_library()
    p = workload(rank, args.n)
    g = qmc.qmc_make_lattice(p.d, p.n, p.gamma)          # host CBC, untimed
    f = qmc.integrand_from_problem(p, "fp32")
    t = qmc.transform(p.transform, p.alpha)
    plan = qmc.Plan(p.d, p.n, p.m, g, p.shifts, t, f)
    shifts_per_launch = 32 if args.no_tune else plan.tune(torch.cuda.current_stream().cuda_stream)  # untimed
    launches_per_step = plan.launches()
    desc = plan.describe()

    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    out = torch.zeros(qmc.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    per = torch.zeros(2 * p.m, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        plan.execute(out=out, per_shift=per, stream=sh)
    torch.cuda.synchronize()

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    for e4 in ev:  # torch creates the CUDA event on first record; the library re-records it
        for e in e4:
            e.record(stream)
    torch.cuda.synchronize()
    assert all(e.cuda_event for e4 in ev for e in e4)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for s in range(K):
            flush.zero_()                                    # L2 flush between steps, outside the events
            e_step0, e_rule0, e_rule1, e_step1 = ev[s]
            plan.record_events(e_rule0.cuda_event, e_rule1.cuda_event)
            e_step0.record(stream)
            plan.execute(out=out, per_shift=per, stream=sh)
            e_step1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    plan.record_events(None, None)
    step_ms = [e[0].elapsed_time(e[3]) for e in ev]
    rule_ms = [e[1].elapsed_time(e[2]) for e in ev]
    total_s = sum(step_ms) / 1e3
    if dist:
        tt = torch.tensor([total_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_s = float(tt.item())
    evals = p.n * p.m
    value = world * evals * K / total_s

    res = qmc.qmc_result.from_buffer_copy(out.cpu().numpy().tobytes()).as_dict()
    assert res["status"] == 0 and np.isfinite(res["mean"][0]), res

    # end to end: public C-ABI call with host inputs and a host result
    e2e_times = []
    for s in range(args.warmup + K):
        t0 = time.perf_counter()
        r, _ = qmc.qmc_integrate(p.d, p.n, p.m, g, p.shifts, t, f, stream=sh)
        if s >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    e2e_total = sum(e2e_times)
    if dist:
        tt = torch.tensor([e2e_total], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_total = float(tt.item())
    h2d = int(g.nbytes + p.shifts.nbytes + p.U.coef.nbytes + p.U.expo.nbytes + p.F.coef.nbytes + p.F.expo.nbytes)

    rule_avg_s = statistics.mean(rule_ms) / 1e3
    achieved = FLOPS_PER_EVAL * evals / rule_avg_s / 1e12
    clocks = clk.summary()
    sms = device_sms(torch, local)
    sm_max_mhz = clocks.get("sm_max_mhz") or device_max_sm_mhz(local)
    peak = fp32_peak_tflops(sms, sm_max_mhz)
    sha = kernel_sha()
    traffic = NCU_TRAFFIC["bytes_per_launch"] if NCU_TRAFFIC["kernel_sha"] == sha else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": config_dict(world, p.n),
        "e2e": {"value": world * evals * K / e2e_total, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": qmc.RESULT_BYTES},
        "gpu_launches": launches_per_step * K,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": (("qmc_jit_sector = sector_body specialised at run time for this U, F; "
                                 if desc.get("specialised") == "1" else "sector_kernel ")
                                + f"<float, D=6, MC={shifts_per_launch}, baker, U deg 1, F deg 2>"),
                     "plan": desc,
                     "kernel_ms": 1e3 * rule_avg_s, "flops_per_eval": FLOPS_PER_EVAL,
                     "peak_source": f"{sms} SMs (device) x {LANES} FP32 lanes x 2 flops x {sm_max_mhz:g} MHz "
                                    "(maximum SM clock, nvidia-smi)",
                     "frac_at_observed_clock": (achieved / fp32_peak_tflops(sms, clocks["sm_mhz"])
                                                if clocks.get("sm_mhz") else None)},
        "clocks": clocks,
        "result": {"mean": res["mean"][0], "err": res["err"][0]},
        "kernel_sha": sha,
    }
    if dist:  # one exchange, after timing: every rank's per-shift values -> one Eq. (3) estimate
        from paper_1811_11722_gb300.distributed import combine_across_ranks
        comb = combine_across_ranks(per.view(-1, 2).cpu().numpy()).as_dict()
        line["combined_estimate"] = {"shifts": p.m * world, "mean": comb["mean"][0], "err": comb["err"][0]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, g)
    if rank == 0 and world == 1 and not args.no_extras and args.n is None:
        from paper_1811_11722_gb300 import inputs as I
        line["extras"] = extras(qmc, I, torch)
        pk = line["extras"]["peaks_measured"]["fp32_tflops"]
        line["roofline"]["peak_measured_probe"] = pk
        line["roofline"]["frac_of_measured_probe"] = achieved / pk
    if not args.no_time_to_tol and rank == 0 and world == 1 and args.n is None:
        from paper_1811_11722_gb300 import inputs as I
        line["time_to_1e-8"] = time_to_tolerance(qmc, I, torch)
    if rank == 0:  # numpy scalars in the extras print as plain numbers
        print(json.dumps(line, default=lambda o: o.item() if hasattr(o, "item") else str(o)), flush=True)
    plan.destroy()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
