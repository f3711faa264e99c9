#!/usr/bin/env python
"""Zolo-PD / Zolo-SVD throughput on GB300 through libzolo's C ABI.

Default workload: the batch of 512 square matrices (n uniform in {64,...,1024},
kappa log-uniform in [1e2, 1e12], r per matrix from kappa) through one
zolo_pd_batched call per step.  The split-precision form (the iterations'
products on the BF16 tensor cores as nine Ozaki slices) is the timed headline
(`value`, matrices/s); the plain FP64 form runs on the same matrices in the same
process (`fp64`, `fp64_value`), and `split_over_fp64` is their ratio.  Every
result's backward error and orthogonality are checked against 1e-13 (exit code
3 if either arm misses it).  `e2e` times the same call with the inputs copied
in from pinned host memory and both factors copied back inside the timed region.
The 1.6 GB of inputs per step exceed the 129 MB L2, so no flush is needed.

Single-matrix workloads (--workload svd4096, pd4096, ...) time one Zolo-SVD or
Zolo-PD per step in the precision --prec names.

Multi-GPU: every rank decomposes its own replica of the workload (weak scaling,
no collective on the data path); value = total matrices / slowest rank's time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload batch512|svd4096|...]
  python bench.py --impl reference ...   (the CPU oracle on a bounded sample)
"""
from __future__ import annotations

import argparse
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

METRIC = "Zolo-PD matrices/s & eff. TFLOP/s, split-prec vs FP64, at bwd err <= 1e-13"
# FP64 FMA pipe: 152 SMs x 2 DFMA (4 flops) per clock x 2.07 GHz max SM clock.
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12

WORKLOADS = {
    "svd4096": dict(kind="svd", m=4096, n=4096, kappa=1e12, r=8, sample_n=384,
                    desc="Plain FP64 Zolo-SVD of one 4096x4096 matrix, sigma geometric 1..1e-12 "
                         "(kappa 1e12), r=8, QR-form then Cholesky-form iteration, eig(H) included"),
    "pd4096": dict(kind="pd", m=4096, n=4096, kappa=1e12, r=8, sample_n=384,
                   desc="Plain FP64 Zolo-PD of one 4096x4096 matrix, kappa 1e12, r=8"),
    # r = 1: the Zolotarev step is the dynamically weighted Halley step, i.e. QDWH-PD
    # on the same kernels (5 iterations at kappa 1e12: 2 QR form, 3 Cholesky form)
    "qdwh4096": dict(kind="pd", m=4096, n=4096, kappa=1e12, r=1, sample_n=384,
                     desc="QDWH-PD (Zolo-PD with r=1) of one 4096x4096 matrix, kappa 1e12"),
    "pd256": dict(kind="pd", m=256, n=256, kappa=1e8, r=3, sample_n=256,
                  desc="Plain FP64 Zolo-PD of one 256x256 matrix, kappa 1e8, r=3"),
    "svd256": dict(kind="svd", m=256, n=256, kappa=1e8, r=3, sample_n=256,
                   desc="Plain FP64 Zolo-SVD of one 256x256 matrix, kappa 1e8, r=3"),
    "svd1024": dict(kind="svd", m=1024, n=1024, kappa=1e8, r=6, sample_n=256,
                    desc="Plain FP64 Zolo-SVD of one 1024x1024 matrix, kappa 1e8, r=6"),
    "pd16384x4096": dict(kind="pd", m=16384, n=4096, kappa=1e6, r=6, sample_n=384, tall=True,
                         desc="Zolo-PD of one 16384x4096 matrix, sigma uniform in [1e-6, 1], r=6"),
    # panels taller than 8 x 768 rows: the QR panel runs in the global-memory cluster kernel
    "pd8192x512": dict(kind="pd", m=8192, n=512, kappa=1e8, r=6, sample_n=256, tall=True,
                       desc="Zolo-PD of one 8192x512 matrix, sigma uniform in [1e-8, 1], r=6"),
    "pd1024": dict(kind="pd", m=1024, n=1024, kappa=1e8, r=6, sample_n=256,
                   desc="Zolo-PD of one 1024x1024 matrix, kappa 1e8, r=6"),
    # beta = sigma_min / 100: forming A in FP64 perturbs its singular values by about
    # sqrt(n) eps ||A|| ~ 1e-14, so the designed sigma_min = 1e-16 is no lower bound
    # of the stored matrix's (with beta = 1e-16, directions below it stay short of 1)
    "pd16384": dict(kind="pd", m=16384, n=16384, kappa=1e16, r=8, sample_n=384, clustered=True,
                    beta_scale=0.01,
                    desc="Zolo-PD of one 16384x16384 matrix, sigma geometric 1..1e-16 plus 64 equal "
                         "singular values at 1e-3, r=8, beta = sigma_min/100 (about 80 GB working "
                         "set)"),
    "batch512": dict(kind="batch", count=512, m=1024, n=1024, kappa=1e12, r=0,
                     desc="Zolo-PD of a batch of 512 square matrices, n uniform in {64,...,1024}, "
                          "sigma geometric over kappa log-uniform in [1e2, 1e12], r chosen per "
                          "matrix, one zolo_pd_batched call (graph-captured, replayed)"),
}


def pd_model_flops(m, n, r, used_qr):
    """Zolo-PD flops credited per matrix: 5 r m n^2 per QR-form iteration (structured
    QR 2mn^2 + structured Q 2mn^2 + Q1 Q2^T mn^2), m n^2 + r (n^3/3 + 2 m n^2) per
    Cholesky-form iteration, 2 m n^2 for H."""
    f = 2.0 * m * n * n
    for qr in used_qr:
        f += 5.0 * r * m * n * n if qr else m * n * n + r * (n ** 3 / 3.0 + 2.0 * m * n * n)
    return f


def make_input(w, seed):
    from paper_1806_06204_gb300 import synth
    if w.get("tall"):
        return synth.tall_uniform(w["m"], w["n"], lo=1.0 / w["kappa"], seed=seed)
    if w.get("clustered"):
        return synth.clustered_square_device(w["n"], 64, seed=5000 + seed)
    return synth.make_matrix(w["m"], w["n"], synth.geometric_sigma(w["n"], w["kappa"]), seed)


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "samples": len(sm), "reasons": sorted(reasons)}


def accuracy(w, sm, outs):
    """Backward error / orthogonality / sigma error of one result, on the device
    with torch (a check of the output, not part of the timed path)."""
    import torch
    A = torch.from_numpy(sm.A).cuda()
    nA = torch.linalg.norm(A)
    n = w["n"]
    I = torch.eye(n, dtype=torch.float64, device="cuda")
    if w["kind"] == "svd":
        U, S, V = outs
        res = torch.linalg.norm(A - (U * S) @ V.T)
        sig = torch.from_numpy(sm.sigma).cuda()
        orth_u = float(torch.linalg.norm(U.T @ U - I))
        orth_v = float(torch.linalg.norm(V.T @ V - I))
        return {"bwd_err": float(res / nA),
                "orth_U": orth_u / math.sqrt(n),
                "orth_V": orth_v / math.sqrt(n),
                "max_sigma_err": float(torch.max(torch.abs(S - sig)) / sig[0]),
                # Section 4's own measures: the residual over ||A||_2 (sigma_1 of
                # the generator) and ||I - U^T U||_F / n, ||I - V^T V||_F / n
                "paper_Res": float(res) / float(sm.sigma[0]),
                "paper_OrthL": orth_u / n,
                "paper_OrthR": orth_v / n}
    Qp, H = outs
    return {"bwd_err": float(torch.linalg.norm(A - Qp @ H) / nA),
            "orth_Qp": float(torch.linalg.norm(Qp.T @ Qp - I) / math.sqrt(n)),
            "H_symmetric": bool(torch.equal(H, H.T))}


def oracle_sample(w, seed=None):
    """Time the CPU oracle on bounded samples of the workload: the same method,
    kappa and r on matrices of two sizes, n_s and 2 n_s / 3 (rows scaled with
    the workload's aspect ratio).  The oracle's seconds per model flop fall as n
    grows (per-column Python overhead), so the full-size rate is scaled from the
    larger sample's, and both are stated.  Returns (matrices/s at full size,
    seconds of CPU work, description)."""
    from oracle import zolo_oracle as zo
    from paper_1806_06204_gb300 import synth
    rates, parts, spent = [], [], 0.0
    for ns in (w["sample_n"], max(64, (2 * w["sample_n"] // 3) // 32 * 32)):
        ms = int(round(ns * w["m"] / w["n"]))
        sm = synth.make_matrix(ms, ns, synth.geometric_sigma(ns, w["kappa"]), seed or 7000)
        t0 = time.perf_counter()
        if w["kind"] == "svd":
            _, _, _, info = zo.zolo_svd(sm.A, 1.0, float(sm.sigma[-1]), r=w["r"])
        else:
            _, _, info = zo.zolo_pd(sm.A, 1.0, float(sm.sigma[-1]), r=w["r"])
        dt = time.perf_counter() - t0
        spent += dt
        f = pd_model_flops(ms, ns, w["r"], info.used_qr)
        rates.append(dt / f)
        parts.append(f"{ms}x{ns}: {dt:.1f} s ({1e9 * dt / f:.2f} s per model Gflop)")
    full = pd_model_flops(w["m"], w["n"], w["r"], info.used_qr)
    desc = (f"oracle zolo_{w['kind']} (kappa {w['kappa']:.0e}, r={w['r']}) on " + "; ".join(parts) +
            f"; scaled by the Zolo-PD flop model to {w['m']}x{w['n']} at the first (larger) "
            f"sample's rate")
    return 1.0 / (rates[0] * full), spent, desc


def max_over_ranks(x, dist):
    """The largest value of x over all ranks (the slowest rank sets the job's time);
    x itself without a process group."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def used_threads(fn):
    """Run fn() and return (its result, the most threads this process had while it
    ran), sampled from /proc every 50 ms: the cores the oracle actually used."""
    peak = [threading.active_count()]
    done = threading.Event()

    def watch():
        while not done.is_set():
            try:
                with open("/proc/self/status") as f:
                    for ln in f:
                        if ln.startswith("Threads:"):
                            peak[0] = max(peak[0], int(ln.split()[1]) - 1)   # minus the watcher
            except OSError:
                return
            done.wait(0.05)

    t = threading.Thread(target=watch, daemon=True)
    t.start()
    try:
        out = fn()
    finally:
        done.set()
        t.join()
    return out, min(peak[0], os.cpu_count() or peak[0])


def batch_oracle_sample(w, budget_s=12.0):
    """Time the CPU oracle on matrices of the batch itself and scale to all of it.

    The oracle's time per model flop falls as n grows (its per-column Python
    overhead is amortised), so one small size alone would understate the CPU.
    The sample takes the batch's matrices in order, at the two largest sizes
    that fit the time budget (n = 192 and 256), times each, and scales every
    matrix of the batch by the lower of the two measured seconds per model flop.
    Returns (matrices/s, seconds of CPU work, description, threads used)."""
    from oracle import zolo_oracle as zo
    from paper_1806_06204_gb300 import synth
    ns, kap = synth.batch_sizes_and_kappas(w["count"])
    tot_f = 0.0
    plan = []
    for i, (n, kp) in enumerate(zip(ns, kap)):
        r = zo.choose_r(1.0 / kp)
        it = zo.ell_schedule(1.0 / kp, r)
        used_qr = [zo.uses_qr(zo.zolotarev_coeffs(l, r), l) for l in it[:-1]]
        f = pd_model_flops(n, n, r, used_qr)
        tot_f += f
        plan.append((i, n, kp, r, f))
    per_size = {}
    spent = [0.0]

    def run():
        for size in (192, 256):
            t, fl, k = 0.0, 0.0, 0
            for i, n, kp, r, f in plan:
                if n != size:
                    continue
                if k >= 1 and t > budget_s / 2:
                    break
                sm = synth.make_matrix(n, n, synth.geometric_sigma(n, kp), 4000 + 1 + i)
                t0 = time.perf_counter()
                zo.zolo_pd(sm.A, 1.0, float(sm.sigma[-1]), r=r)
                t += time.perf_counter() - t0
                fl += f
                k += 1
            per_size[size] = (t, fl, k)
            spent[0] += t

    _, cores = used_threads(run)
    rate = {sz: t / fl for sz, (t, fl, k) in per_size.items()}
    best = min(rate.values())
    desc = ("oracle zolo_pd on matrices of the batch itself: " +
            ", ".join(f"{k} at n={sz} ({t:.1f} s, {1e9 * t / fl:.2f} s per Gflop)"
                      for sz, (t, fl, k) in sorted(per_size.items())) +
            f"; every matrix of the batch scaled by the lower rate (model flops) to all "
            f"{w['count']}")
    return 1.0 / (best * tot_f / w["count"]) if best > 0 else None, spent[0], desc, cores


def run_reference(args, w, rank):
    if rank != 0:
        return
    vals, tot, cores = [], 0.0, 1
    desc = ""
    if w["kind"] == "batch":
        # each step a bounded sample, sized so that the whole run stays within minutes
        budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
        sample = lambda: batch_oracle_sample(w, budget_s=budget)
    else:
        def sample():
            (v, dt, d), c = used_threads(lambda: oracle_sample(w))
            return v, dt, d, c
    for _ in range(args.warmup):
        sample()
    for _ in range(args.steps):
        v, dt, desc, cores = sample()
        vals.append(v)
        tot += dt
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "matrices/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * tot / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"]},
            "cpu_baseline": {"value": value, "unit": "matrices/s", "cores": cores,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "matrices/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# Builder's DFMA microbenchmark on this GPU (a register-resident FMA chain on all
# SMs, CUDA events): the FP64 pipe's measured ceiling beside the derived peak.
FP64_DFMA_MEASURED_TFLOPS = 1.20
# Tensor-core products issued per FP64-equivalent flop on the split path: nine
# BF16 slices per operand, slice pairs (s, t) with s + t <= 11: 53; eight FP16
# slices, s + t <= 9: 36; eleven FP8 (E4M3) slices, s + t <= 13: 76.  The FP8
# products run at twice the 16-bit rate (nominal 4.5 against 2.25 PFLOP/s), so
# their peak is the measured BF16 peak times 2.
SPLIT_PAIRS = 53
SPLIT_PAIRS_OF = {"bf16": 53, "fp16": 36, "fp8": 76}
SLICE_PEAK_RATIO = {"bf16": 1.0, "fp16": 1.0, "fp8": 2.0}
SLICE_DTYPE = {"bf16": "bf16x9-slices->f64", "fp16": "fp16x8-slices->f64",
               "fp8": "e4m3x11-slices->f64"}
SLICE_DESC = {"bf16": "nine BF16 slices", "fp16": "eight FP16 slices",
              "fp8": "eleven FP8 (E4M3) slices"}


def split_prec(zb, slices):
    return {"bf16": zb.ZOLO_SPLIT_BF16, "fp16": zb.ZOLO_SPLIT_FP16,
            "fp8": zb.ZOLO_SPLIT_FP8}[slices]


# DRAM bytes per algorithmic byte of a kernel class, from an ncu capture of that
# class (dram__bytes_read.sum + dram__bytes_write.sum over the bytes its launches
# state); bench.py scales it by the bytes its own launches state.  Set to None
# when the kernel changes.
TRAFFIC_PER_STATED_BYTE = {
    # qr_panel_smem_kernel, 12 launches at n = 960, r = 5: 1.313 MB read, 0
    # written, of 2.54 MB stated (profiles/traffic_batch4_split.md)
    "qr_panel": 0.517,
}


def sm_time(kstats):
    """Per kernel class, the SM-time of the profiled call: each launch's device
    time times the share of the GPU's resident-block slots its blocks take (the
    library's zolo_profile_read); with the batch's lanes in flight these shares
    add up to about the timed step, the plain device times to several times it."""
    return {k: round(v.get("sm_ms", 0.0), 3) for k, v in kstats.items() if v["launches"]}


# Kernel classes whose work the Zolo-PD flop model does not count (Zolo-SVD's
# eigensolver sweeps; its three n^3 products run in the gemm_f64 class).
OUTSIDE_PD_MODEL = {"jacobi_round", "jacobi32_sweep"}


def roofline(kstats, step_ms, model_flops=None, split_pairs=SPLIT_PAIRS, peak_ratio=1.0,
             by="ms"):
    """Roofline entry of the dominant kernel class (by device time in one step,
    or with by="sm_ms" by SM-time: device time times the share of the GPU the
    launches' blocks take).

    With model_flops (the Zolo-PD flops of the step), the algorithmic work of a
    flop-carrying class is the model's, shared out between the classes in
    proportion to the flops each launch site states for its launch; achieved =
    that share / the class's device time.  On the split path a model flop is
    issued as `split_pairs` tensor-core products of the slice type, whose peak is
    `peak_ratio` times the measured BF16 one.  The flops the launches
    state themselves (padding, T factors, the explicit Q's full rows included)
    are kept beside it as `issued_*`."""
    dom_name, dom = max(((k, v) for k, v in kstats.items() if v["launches"] > 0),
                        key=lambda kv: kv[1].get(by, kv[1]["ms"]))
    sec = dom["ms"] / 1000.0
    bound = {"combine": "hbm", "slice": "hbm", "gemm_split": "tensor"}.get(dom_name, "alu")
    # the eigensolver's sweeps are outside the Zolo-PD flop model: they take no share
    flop_classes = {k: v for k, v in kstats.items()
                    if v["launches"] > 0 and v["flops"] > 0 and k not in OUTSIDE_PD_MODEL}
    stated = sum(v["flops"] for v in flop_classes.values())
    if model_flops and dom_name in flop_classes and stated > 0:
        work = model_flops * dom["flops"] / stated
        basis = ("Zolo-PD model flops of the step, shared between kernel classes in proportion "
                 "to their launches' stated flops")
    else:
        work = dom["flops"]
        basis = "flops stated by the launches"
    if bound == "tensor":
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak = peaks["bf16_tflops_sustained"] * peak_ratio
        achieved = work * split_pairs / sec / 1e12
        roof = {"bound": "tensor", "kernel": dom_name, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": ("MEASURED_PEAKS.json bf16_tflops_sustained (of measured)" +
                                (f" x {peak_ratio:g} (nominal FP8/BF16 ratio)"
                                 if peak_ratio != 1.0 else "")),
                "work_basis": basis + f"; x{split_pairs} slice-pair products per flop",
                "fp64_equivalent_tflops": work / sec / 1e12,
                "issued_tflops": dom["flops"] * split_pairs / sec / 1e12}
    elif bound == "alu":
        achieved = work / sec / 1e12
        roof = {"bound": "alu", "kernel": dom_name, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "derived: 152 SMs x 4 FP64 flops/clk x 2.07 GHz (MEASURED_PEAKS.json "
                               "has no FP64 entry); DFMA microbenchmark measured "
                               f"{FP64_DFMA_MEASURED_TFLOPS} TFLOP/s",
                "frac_of_measured_dfma": achieved / FP64_DFMA_MEASURED_TFLOPS,
                "work_basis": basis, "issued_tflops": dom["flops"] / sec / 1e12}
    else:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        gbs = dom["bytes"] / sec / 1e9
        roof = {"bound": "hbm", "kernel": dom_name, "achieved": gbs, "peak": peak, "unit": "GB/s",
                "frac": gbs / peak, "traffic": None, "work_basis": "bytes stated by the launches"}
    ratio = TRAFFIC_PER_STATED_BYTE.get(dom_name)
    if ratio is not None and dom["bytes"] > 0:
        roof["traffic"] = ratio * dom["bytes"] / dom["launches"]
        roof["traffic_source"] = ("DRAM bytes per launch: ncu capture of the class "
                                  "(profiles/traffic_batch4_split.md) scaled by the algorithmic "
                                  "bytes these launches state")
        roof["algorithmic_bytes_per_launch"] = dom["bytes"] / dom["launches"]
    roof["launches"] = dom["launches"]
    roof["avg_launch_ms"] = dom["ms"] / dom["launches"]
    roof["share_of_step"] = dom["ms"] / step_ms
    return roof


def batch_arm(args, w, h, mats, As, Qps, Hs, split, steps, warmup, local, dist, slices=None):
    """One precision of the batch: warm-up, K timed zolo_pd_batched calls (CUDA
    events on the calling stream, barrier and synchronise on both sides), then
    one more call with per-launch events for the kernel classes, and the
    accuracy of every result."""
    import torch
    from paper_1806_06204_gb300 import binding as zb
    slices = slices or args.slices
    sp = split_prec(zb, slices)
    os_ = [zb.opts(beta=float(sm.sigma[-1]), alpha=1.0, r=0,
                   prec=sp if split else zb.ZOLO_FP64, ns_steps=1 if split else 0,
                   chol_form=args.chol_form)
           for sm in mats]

    def step():
        _, _, infos, st = zb.zolo_pd_batched(h, As, os_, Qps=Qps, Hs=Hs)
        return infos

    def barrier():
        if dist:
            dist.barrier()

    infos = None
    # --autotune-batch: the first warm-up call measures the batch's contraction
    # shapes (zolo_autotune) and the timed calls replay the kept kernels.  Off by
    # default: on the batch of 512 the kept kernels measured no faster (split
    # 275.3 vs 275.1 matrices/s, FP64 71.0 vs 71.8) -- they win alone on the GPU,
    # but 32 lanes in flight already fill it
    tuning = args.autotune_batch and warmup > 0
    if tuning:
        zb.autotune(h, True)
    for _ in range(warmup):
        infos = step()
    torch.cuda.synchronize()
    if tuning:
        zb.autotune(h, False)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = zb.kernel_launches()
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            infos = step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = zb.kernel_launches() - launches0
    ms_step = max_over_ranks(e0.elapsed_time(e1) / steps, dist)
    flops = sum(pd_model_flops(a.shape[0], a.shape[1], i.r, i.used_qr) for a, i in zip(As, infos))

    # per-kernel device times: one more call, outside the timed steps, with
    # event-bracketed launches (a replayed graph cannot be bracketed kernel by kernel)
    zb.profile(True)
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    step()
    e3.record(stream)
    torch.cuda.synchronize()
    kstats = zb.profile_read()
    zb.profile(False)
    prof_ms = e2.elapsed_time(e3)
    roof = roofline(kstats, prof_ms, flops, split_pairs=SPLIT_PAIRS_OF[slices],
                    peak_ratio=SLICE_PEAK_RATIO[slices])
    roof["measured"] = ("one extra call after the timed steps with the batch's lanes "
                        "serialised and every launch bracketed by CUDA events (no graph replay): "
                        "each launch timed alone on the GPU")
    # the same class inside the timed steps, where 32 lanes overlap: its work over
    # the whole timed step is a lower bound of its rate there (it runs at most that long)
    work = roof["achieved"] * roof["launches"] * roof["avg_launch_ms"] / 1000.0
    rate = work / (ms_step / 1000.0)
    roof["in_step_lower_bound"] = {
        "achieved": rate, "frac": rate / roof["peak"],
        "basis": "the class's work divided by the whole timed step (its lanes overlap there)"}
    # the class that holds the most of the GPU: with 32 lanes in flight the
    # classes' SM-times add up to about the step, so this one sets the pace
    # (the class above has the most device time alone, on a few SMs)
    roof_sm = roofline(kstats, prof_ms, flops, split_pairs=SPLIT_PAIRS_OF[slices],
                       peak_ratio=SLICE_PEAK_RATIO[slices], by="sm_ms")
    roof_sm["sm_time_share"] = (kstats[roof_sm["kernel"]].get("sm_ms", 0.0) /
                                max(1e-9, sum(v.get("sm_ms", 0.0) for v in kstats.values())))

    # accuracy of every result, on the device with torch (a check, not timed)
    bwd, orth = 0.0, 0.0
    for a, q, hh in zip(As, Qps, Hs):
        n = a.shape[1]
        bwd = max(bwd, float(torch.linalg.norm(a - q @ hh) / torch.linalg.norm(a)))
        I = torch.eye(n, dtype=torch.float64, device="cuda")
        orth = max(orth, float(torch.linalg.norm(q.T @ q - I) / math.sqrt(n)))
    acc = {"max_bwd_err": bwd, "max_orth_Qp": orth, "matrices": len(As),
           "statuses_nonzero": sum(1 for i in infos if i.status),
           "bar": 1e-13, "bar_met": bool(bwd <= 1e-13 and orth <= 1e-13)}
    return {"os": os_, "ms_step": ms_step, "flops": flops, "infos": infos, "launches": launches,
            "autotune": bool(tuning),
            "kstats": kstats, "roof": roof, "roof_sm": roof_sm, "acc": acc, "clocks": clk.summary(),
            "steps": steps, "warmup": warmup}


def run_batch(args, w, rank, world, dist, local):
    """The uneven batch through zolo_pd_batched.  By default both precisions run
    on the same matrices: `value` is the split-precision matrices/s over all
    ranks, `fp64` the plain FP64 arm, `split_over_fp64` their ratio."""
    import torch
    from paper_1806_06204_gb300 import binding as zb, synth
    prec = args.prec if args.prec != "auto" else "both"
    if args.count:   # the first `count` matrices of the same seeded batch (for profiling)
        w = dict(w, count=args.count)
    mats = synth.batch(w["count"], seed=4000 + 100000 * rank)
    if args.count:
        mats = mats[:args.count]
    As = [torch.from_numpy(sm.A).cuda() for sm in mats]
    Qps = [zb.empty_colmajor(a.shape[0], a.shape[1]) for a in As]
    Hs = [zb.empty_colmajor(a.shape[1], a.shape[1]) for a in As]
    h = zb.Handle(local)
    if args.no_graph:
        zb.batch_graphs(h, False)
    head_split = prec in ("split", "both")
    arm = batch_arm(args, w, h, mats, As, Qps, Hs, head_split, args.steps, args.warmup, local,
                    dist)
    fp64 = None
    others = []
    if prec == "both":
        fs = args.fp64_steps if args.fp64_steps is not None else max(1, min(args.steps, 5))
        fw = args.fp64_warmup if args.fp64_warmup is not None else min(args.warmup, 3)
        fp64 = batch_arm(args, w, h, mats, As, Qps, Hs, False, fs, fw, local, dist)
        if not args.no_other_slices:
            # the other slice forms on the same matrices, for comparison
            for oth in SLICE_DTYPE:
                if oth == args.slices:
                    continue
                other = batch_arm(args, w, h, mats, As, Qps, Hs, True, fs, fw, local, dist,
                                  slices=oth)
                other["slices"] = oth
                others.append(other)
    value = world * w["count"] / (arm["ms_step"] / 1000.0)
    os_ = arm["os"]

    e2e = None
    if not args.no_e2e:
        # host (pinned) inputs copied in and both factors copied back inside the timed region
        Ah = [torch.from_numpy(sm.A.T.copy()).pin_memory().t() for sm in mats]
        Qh = [torch.empty((a.shape[1], a.shape[0]), dtype=torch.float64).pin_memory().t() for a in As]
        Hh = [torch.empty((a.shape[1], a.shape[1]), dtype=torch.float64).pin_memory().t() for a in As]
        Ad = [zb.empty_colmajor(a.shape[0], a.shape[1]) for a in As]

        def host_step():
            for d, src in zip(Ad, Ah):
                d.copy_(src, non_blocking=True)
            zb.zolo_pd_batched(h, Ad, os_, Qps=Qps, Hs=Hs)
            for dst, q in zip(Qh, Qps):
                dst.copy_(q, non_blocking=True)
            for dst, hh in zip(Hh, Hs):
                dst.copy_(hh, non_blocking=True)
            torch.cuda.synchronize()

        host_step()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_step()
        if dist:
            dist.barrier()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, dist)
        nb = sum(a.numel() for a in As) * 8
        e2e = {"value": world * w["count"] / e2e_s, "unit": "matrices/s", "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb + sum(x.numel() for x in Hs) * 8}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, desc, cores = batch_oracle_sample(w)
        cpu = {"value": v, "unit": "matrices/s", "cores": cores, "kind": "oracle", "sample": desc}
    if rank == 0:
        ns = [a.shape[1] for a in As]
        infos = arm["infos"]
        sl = SLICE_DESC[args.slices]
        desc = w["desc"] + (f": split precision ({sl}, FP32 level sums) timed, plain "
                            "FP64 beside it" if prec == "both" else
                            (f": split precision ({sl})" if head_split else
                             ": plain FP64"))
        line = {"metric": METRIC, "value": value, "unit": "matrices/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": arm["ms_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": (SLICE_DTYPE[args.slices] if head_split else "f64"),
                "data": "synthetic",
                "config": {"workload": args.workload, "desc": desc, "count": w["count"],
                           "n_min": min(ns), "n_max": max(ns), "prec": "split" if head_split else "fp64",
                           "r_hist": {str(r): sum(1 for i in infos if i.r == r)
                                      for r in sorted({i.r for i in infos})},
                           "l2": "inputs larger than L2 (1.6 GB of A per step; no flush)",
                           "autotune": arm["autotune"],
                           "parallelism": "replicas" if world > 1 else "single"},
                "eff_tflops": world * arm["flops"] / (arm["ms_step"] / 1000.0) / 1e12,
                "pd_model_flops": arm["flops"], "accuracy": arm["acc"], "roofline": arm["roof"],
                "roofline_by_sm_time": arm["roof_sm"],
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": arm["launches"],
                "kernel_ms": {k: round(v["ms"], 3) for k, v in arm["kstats"].items() if v["launches"]},
                "kernel_sm_ms": sm_time(arm["kstats"]),
                "kernel_gflop": {k: round(v["flops"] / 1e9, 1) for k, v in arm["kstats"].items()
                                 if v["launches"]},
                "clocks": arm["clocks"]}
        if fp64 is not None:
            fv = world * w["count"] / (fp64["ms_step"] / 1000.0)
            line["fp64_value"] = fv
            line["split_over_fp64"] = value / fv
            line["fp64"] = {"value": fv, "unit": "matrices/s", "ms_per_step": fp64["ms_step"],
                            "steps": fp64["steps"], "warmup": fp64["warmup"],
                            "eff_tflops": world * fp64["flops"] / (fp64["ms_step"] / 1000.0) / 1e12,
                            "accuracy": fp64["acc"], "roofline": fp64["roof"],
                            "gpu_launches": fp64["launches"],
                            "kernel_ms": {k: round(v["ms"], 3) for k, v in fp64["kstats"].items()
                                          if v["launches"]},
                            "clocks": fp64["clocks"]}
        for other in others:
            ov = world * w["count"] / (other["ms_step"] / 1000.0)
            line[other["slices"] + "_slices"] = {
                "value": ov, "unit": "matrices/s", "dtype": SLICE_DTYPE[other["slices"]],
                "ms_per_step": other["ms_step"], "steps": other["steps"],
                "warmup": other["warmup"],
                "split_over_fp64": ov / line["fp64_value"] if fp64 is not None else None,
                "eff_tflops": world * other["flops"] / (other["ms_step"] / 1000.0) / 1e12,
                "accuracy": other["acc"], "roofline": other["roof"],
                "gpu_launches": other["launches"],
                "kernel_ms": {k: round(v["ms"], 3) for k, v in other["kstats"].items()
                              if v["launches"]},
                "clocks": other["clocks"]}
        print(json.dumps(line), flush=True)
        bad = [a for a in (arm, fp64, *others) if a is not None and not a["acc"]["bar_met"]]
        if bad:
            print("accuracy bar (1e-13) not met", file=sys.stderr)
            h.close()
            raise SystemExit(3)
    h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch512", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="auto", choices=["auto", "fp64", "split", "both"],
                    help="split: the iterations' products on the BF16 tensor cores (Ozaki slices); "
                         "both (batch only): split timed, FP64 beside it; auto: both for the "
                         "batch, fp64 otherwise")
    ap.add_argument("--slices", default="bf16", choices=sorted(SLICE_DTYPE),
                    help="split precision's slices: nine BF16 six-bit slices (53 slice-pair "
                         "products), eight FP16 seven-bit slices (36) or eleven FP8 "
                         "five-bit slices (76 at twice the rate)")
    ap.add_argument("--no-graph", action="store_true",
                    help="batch workload: queue the lanes directly every step instead of replaying "
                         "a recorded CUDA graph (for kernel profilers)")
    ap.add_argument("--count", type=int, default=None,
                    help="batch workload: only its first COUNT matrices (for profiler captures)")
    ap.add_argument("--no-other-slices", action="store_true",
                    help="with --prec both: skip the arms of the other slice forms")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="timed steps of the FP64 arm with --prec both (default min(steps, 5))")
    ap.add_argument("--fp64-warmup", type=int, default=None,
                    help="warm-up steps of the FP64 arm with --prec both (default min(warmup, 3))")
    ap.add_argument("--beta-scale", type=float, default=None,
                    help="beta = sigma_min times this (default: the workload's own, else 1)")
    ap.add_argument("--r", type=int, default=None,
                    help="override the workload's r; -1 = the r measured fastest on this GPU "
                         "(tuned during the warm-up steps)")
    ap.add_argument("--chol-form", type=int, default=0, choices=[0, 1, 2],
                    help="Cholesky-form iterations: 1 triangular solves, 2 explicit inverse, "
                         "0 by the flop model")
    ap.add_argument("--autotune", dest="autotune", action="store_true", default=True,
                    help="measure the contraction kernels per shape during the warm-up steps "
                         "(default)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="built-in kernel rules only")
    ap.add_argument("--autotune-batch", action="store_true",
                    help="batch workload: measure the contraction kernels during the warm-up "
                         "steps (off by default: no gain measured on the batch of 512)")
    ap.add_argument("--tune-cache", default=None,
                    help="tuning-cache file: loaded before the warm-up steps when it exists, "
                         "written after them")
    ap.add_argument("--shard-shifts", action="store_true",
                    help="Zolo-PD workloads under torchrun: the ranks decompose one matrix "
                         "together, each taking a block of every iteration's r shifts, with one "
                         "NCCL sum of S per iteration (zolo_pd_sharded; strong scaling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if args.impl == "ours" and torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)

    if args.impl == "reference":
        run_reference(args, w, rank)
        if dist:
            dist.destroy_process_group()
        return

    import numpy as np
    import torch
    from paper_1806_06204_gb300 import build
    build.build()
    from paper_1806_06204_gb300 import binding as zb

    torch.cuda.set_device(local)
    if w["kind"] == "batch":
        run_batch(args, w, rank, world, dist, local)
        if dist:
            dist.destroy_process_group()
        return
    shard = args.shard_shifts and world > 1 and w["kind"] == "pd"
    if args.shard_shifts and not shard:
        raise SystemExit("--shard-shifts needs torchrun with N > 1 and a Zolo-PD workload")
    # sharded: every rank holds the same matrix; replicas: each rank its own
    sm = make_input(w, seed=2000 + (0 if shard else rank))
    A = torch.from_numpy(sm.A).cuda()
    h = zb.Handle(local)
    if args.tune_cache and os.path.exists(args.tune_cache):
        if zb.tune_load(h, args.tune_cache) != 0:
            raise SystemExit(f"tuning cache {args.tune_cache} refused (other GPU or malformed)")
    # kernels are measured during the warm-up steps only, never inside the timed region
    tuning = args.autotune and args.warmup > 0
    if tuning:
        zb.autotune(h, True)
    if args.prec == "both":
        raise SystemExit("--prec both applies to the batch workload only")
    split = args.prec == "split"
    beta_scale = args.beta_scale if args.beta_scale is not None else w.get("beta_scale", 1.0)
    r_req = args.r if args.r is not None else w["r"]
    sp = split_prec(zb, args.slices)
    o = zb.opts(beta=float(np.min(sm.sigma)) * beta_scale, alpha=1.0, r=r_req,
                prec=sp if split else zb.ZOLO_FP64, ns_steps=1 if split else 0,
                chol_form=args.chol_form)
    m, n = w["m"], w["n"]

    def step():
        if w["kind"] == "svd":
            U, S, V, info = zb.zolo_svd(h, A, o)
            return (U, S, V), info
        if shard:
            Qp, H, info = zb.zolo_pd_sharded(h, A, o, rank, world, zb.torch_allreduce())
        else:
            Qp, H, info = zb.zolo_pd(h, A, o)
        return (Qp, H), info

    for _ in range(args.warmup):
        outs, info = step()
    torch.cuda.synchronize()
    if tuning:
        zb.autotune(h, False)   # the timed steps use the kept kernels
    if args.tune_cache:
        zb.tune_save(h, args.tune_cache)

    def barrier():
        if dist:
            dist.barrier()

    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = zb.kernel_launches()
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            outs, info = step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = zb.kernel_launches() - launches0
    ms_step = e0.elapsed_time(e1) / args.steps
    ms_step = max_over_ranks(ms_step, dist)
    # matrices/s over all ranks (sharded: the ranks decompose one matrix together)
    value = (1 if shard else world) / (ms_step / 1000.0)
    flops = pd_model_flops(m, n, info.r, info.used_qr)
    acc = accuracy(w, sm, outs)

    # roofline of the dominant kernel class: one more step after the timed ones,
    # every launch bracketed by CUDA events on its stream
    zb.profile(True)
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    step()
    e3.record(stream)
    torch.cuda.synchronize()
    kstats = zb.profile_read()
    zb.profile(False)
    roof = roofline(kstats, e2.elapsed_time(e3), flops, split_pairs=SPLIT_PAIRS_OF[args.slices],
                    peak_ratio=SLICE_PEAK_RATIO[args.slices])
    roof["measured"] = "one extra step after the timed ones, per-launch CUDA events"

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        Ah = torch.from_numpy(sm.A).pin_memory().numpy()
        Ah = np.asfortranarray(Ah)
        if w["kind"] == "svd":
            Uh = torch.empty((n, m), dtype=torch.float64).pin_memory().numpy().T
            Vh = torch.empty((n, n), dtype=torch.float64).pin_memory().numpy().T
            Sh = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
            host_step = lambda: zb.zolo_svd_host(h, Ah, o, Uh, Sh, Vh)
            d2h = 8 * (m * n + n * n + n)
        elif shard:
            # pinned host copies in and out around the sharded call
            Ap = torch.from_numpy(sm.A.T.copy()).pin_memory().t()
            Qt = torch.empty((n, m), dtype=torch.float64).pin_memory().t()
            Ht = torch.empty((n, n), dtype=torch.float64).pin_memory().t()
            Ad = zb.empty_colmajor(m, n)
            sum_fn = zb.torch_allreduce()

            def host_step():
                Ad.copy_(Ap, non_blocking=True)
                Qd, Hd, _ = zb.zolo_pd_sharded(h, Ad, o, rank, world, sum_fn)
                Qt.copy_(Qd, non_blocking=True)
                Ht.copy_(Hd, non_blocking=True)
                torch.cuda.synchronize()
            d2h = 8 * (m * n + n * n)
        else:
            Qh = torch.empty((n, m), dtype=torch.float64).pin_memory().numpy().T
            Hh = torch.empty((n, n), dtype=torch.float64).pin_memory().numpy().T
            host_step = lambda: zb.zolo_pd_host(h, Ah, o, Qh, Hh)
            d2h = 8 * (m * n + n * n)
        host_step()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_step()
        torch.cuda.synchronize()
        barrier()
        e2e_s = (time.perf_counter() - t0) / args.steps
        e2e_s = max_over_ranks(e2e_s, dist)
        e2e = {"value": (1 if shard else world) / e2e_s, "unit": "matrices/s",
               "h2d_bytes_per_step": 8 * m * n, "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        (v, dt, desc), cores = used_threads(lambda: oracle_sample(w))
        cpu = {"value": v, "unit": "matrices/s", "cores": cores, "kind": "oracle",
               "sample": desc}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "matrices/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "strong" if shard else "weak",
                "vs_baseline": None,
                "dtype": "f64" if not split else SLICE_DTYPE[args.slices],
                "data": "synthetic",
                "config": {"workload": args.workload, "desc": w["desc"], "m": m, "n": n,
                           "kappa": w["kappa"], "r": info.r, "r_requested": r_req,
                           "chol_form": info.chol_form, "autotune": bool(tuning),
                           "prec": "split" if split else "fp64",
                           "beta_over_sigma_min": beta_scale,
                           "l2": "inputs larger than L2 (no flush)",
                           "parallelism": (f"shifts sharded over {world} ranks, one NCCL sum of S "
                                           "per iteration" if shard else
                                           "replicas" if world > 1 else "single")},
                "eff_tflops": world * flops / (ms_step / 1000.0) / 1e12,
                "pd_model_flops": flops, "iters": info.iters, "used_qr": info.used_qr,
                "eig_sweeps": info.eig_sweeps, "accuracy": acc,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches,
                "kernel_ms": {k: round(v["ms"], 3) for k, v in kstats.items() if v["launches"]},
                "kernel_sm_ms": sm_time(kstats),
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
