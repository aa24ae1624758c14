#!/usr/bin/env python
"""Throughput of the whole PROJECTION hot path (Algorithm 2 + Section 5.1 EM)
on one GB300, on seeded synthetic planted-motif inputs.

A step is one motif search over one instance: pack-resident 2-bit input ->
Philox positions, projection, hashing and bucket counts for all m trials ->
enriched-bucket lists -> theta^0 -> EM for every enriched bucket -> FP64
ranking, consensus, sites.  Default workload: planted (15,4), t = 20 x n = 600,
k = 7, s = 4, m = 172 (the Section 5 bound at q = 0.95), 5 EM iterations,
pseudocount 0.25.  EM runs on the tensor cores with the BF16 hi + lo split
(--precision fp32 selects the plain FP32 SIMT path); the line also gives one
step of the other precision through the same call and, for both, the errors
against the FP64 oracle from identical starting models.

Prints one JSON line.  `value` is EM l-mer x PWM scores per second over the
whole step (scores per step = x * C * (em_iters + 1), C = enriched buckets);
hashes/s and instances/s are reported beside it.

--impl reference times the CPU oracle (the FP64 statement of the method) on
the same workload: all m trials hashed, EM on a deterministic candidate
sample, time extrapolated linearly in the candidate count.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import instance_for_config, mix_instances  # noqa: E402

METRIC = "l-mer hashes/s, EM l-mer×PWM scores/s; batched instances/s vs plain at same motif"
UNIT = "scores/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
SMS = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_NOMINAL = 2070.0
FLUSH_BYTES = 512 << 20  # > 2x the 129 MB L2


def resolve(inst, p):
    """k, s, m as the library resolves them (0 = Section 5 choice)."""
    import paper_1605_06904_gb300 as P
    return P.projection_default_params(inst.lens, inst.l, inst.d, p.get("k", 0), p.get("s", 0),
                                       p.get("m", 0))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_over_ranks(work, seconds, device, world):
    """Whole-job totals of a weak-scaling run: per-rank work summed, wall time
    the slowest rank's (one all-reduce each; no data-path collective)."""
    import torch
    import torch.distributed as dist
    w = torch.tensor([float(v) for v in work], dtype=torch.float64, device=device)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(w, op=dist.ReduceOp.SUM)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in w.tolist()], float(t.item())


def rank_instance(cfg: int, rank: int):
    """Weak scaling: rank r searches instance r of the workload."""
    return instance_for_config(cfg, rank)


def recorded_traffic(profile: str, sources) -> float | None:
    """DRAM bytes per launch from a committed ncu summary, if the kernel sources
    still hash to what the capture was taken with (else None)."""
    import hashlib
    try:
        text = open(os.path.join(ROOT, "profiles", profile)).read()
        h = hashlib.sha256()
        for s in sources:
            h.update(open(os.path.join(ROOT, "paper_1605_06904_gb300", "csrc", s), "rb").read())
        vals = dict(ln.strip().split(": ", 1) for ln in text.splitlines()
                    if ln.strip().startswith(("traffic_bytes_per_launch:", "source_sha256_16:")))
        if vals.get("source_sha256_16") != h.hexdigest()[:16]:
            return None
        return float(vals["traffic_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS, "bf16_tflops": FALLBACK_BF16_TFLOPS}, "fallback"


def em_error_report(P, inst, packed, k, s, seed, iters, beta, dev, n_sample=16, trials=2,
                    site_prob=None):
    """Errors of both EM precisions against the FP64 oracle from identical
    starting models: theta^0 of the n_sample largest buckets of the first
    `trials` trials, hashed and built by the oracle (inputs of the GPU leg are
    the float32 rounding of the oracle's theta^0)."""
    import torch

    import oracle as O
    codes = O.encode(inst.ascii)
    off = inst.seq_off
    h = O.hash_trials(codes, off, inst.l, k, s, seed, 0, trials)
    sel = O.top_candidates(h["cand_cnt"], n_sample)
    th0 = np.stack([O.theta0(codes, off, inst.l, h["members"][h["cand_off"][c]:h["cand_off"][c + 1]],
                             beta) for c in sel]).astype(np.float32)
    if site_prob is None:
        w_pwm, w_ll = O.em(codes, off, inst.l, O.background(codes), th0.astype(np.float64), iters,
                           beta, nthreads=os.cpu_count() or 1)
    else:
        w_pwm, w_ll = O.em_zoops(codes, off, inst.l, O.background(codes), th0.astype(np.float64),
                                 iters, beta, site_prob, nthreads=os.cpu_count() or 1)
    bg = P.projection_background(packed, off[-1])
    out = {}
    for name, prec in (("bf16_split", P.PROJ_EM_BF16_SPLIT), ("fp32", P.PROJ_EM_FP32)):
        t0 = torch.from_numpy(th0).to(dev)
        if site_prob is None:
            g_pwm, g_ll = P.em_refine(packed, off, inst.l, bg, t0, iters, beta, prec)
        else:
            g_pwm, g_ll = P.em_refine_zoops(packed, off, inst.l, bg, t0, iters, beta, site_prob,
                                            prec)
        g_pwm, g_ll = g_pwm.cpu().numpy(), g_ll.cpu().numpy()
        out[name] = {"pwm_max_abs": float(np.abs(g_pwm - w_pwm).max()),
                     "ll_max_rel": float((np.abs(g_ll - w_ll) /
                                          np.maximum(np.abs(w_ll), inst.t)).max()),
                     "consensus_equal_frac": float(np.mean(
                         [O.consensus(g_pwm[q]) == O.consensus(w_pwm[q])
                          for q in range(len(sel))]))}
    return out, int(len(sel))


# ---------------------------------------------------------------------------
# CPU oracle leg
# ---------------------------------------------------------------------------

def oracle_step(inst, k, s, m, seed, iters, beta, max_sample=6000, nthreads=None):
    """One oracle step on a bounded sample; returns (seconds for the whole step,
    extrapolated; details)."""
    import oracle as O
    nthreads = nthreads or os.cpu_count() or 1
    codes = O.encode(inst.ascii)
    off = inst.seq_off
    t0 = time.perf_counter()
    h = O.hash_trials(codes, off, inst.l, k, s, seed, 0, m)
    t_hash = time.perf_counter() - t0
    C = int(h["cand_key"].size)
    stride = max(1, math.ceil(C / max_sample))
    idx = np.arange(0, C, stride)
    t0 = time.perf_counter()
    bg = O.background(codes)
    th0 = np.stack([O.theta0(codes, off, inst.l,
                             h["members"][h["cand_off"][c]:h["cand_off"][c + 1]], beta)
                    for c in idx]) if idx.size else np.zeros((0, inst.l, 4))
    t_th0 = time.perf_counter() - t0
    t0 = time.perf_counter()
    if idx.size:
        O.em(codes, off, inst.l, bg, th0, iters, beta, nthreads=nthreads)
    t_em = time.perf_counter() - t0
    scale = C / max(1, idx.size)
    total = t_hash + (t_th0 + t_em) * scale
    return total, {"C": C, "sample": int(idx.size), "stride": stride, "t_hash": t_hash,
                   "t_theta0": t_th0, "t_em": t_em, "threads": nthreads}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    inst = instance_for_config(args.config, 0)
    p = dict(inst.params)
    import oracle as O
    k, s, m = O.default_params(inst.lens, inst.l, inst.d, p.get("k", 0), p.get("s", 0),
                               p.get("m", 0))
    iters, beta, seed = p["em_iters"], p["beta"], 1000 + args.config
    for _ in range(args.warmup):
        oracle_step(inst, k, s, m, seed, iters, beta, max_sample=args.ref_sample)
    times, det = [], None
    for _ in range(args.steps):
        tt, det = oracle_step(inst, k, s, m, seed, iters, beta, max_sample=args.ref_sample)
        times.append(tt)
    T = float(np.mean(times))
    x = inst.n_lmers
    scores = x * det["C"] * (iters + 1)
    value = scores / T
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": T * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(args, inst, k, s, m, iters, beta),
        "hashes_per_s": m * x / T, "instances_per_s": 1.0 / T,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": det["threads"], "kind": "oracle",
                         "sample": sample_text(det, m)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def sample_text(det, m):
    return (f"all {m} trials hashed; theta0 + EM on every {det['stride']}th candidate "
            f"({det['sample']} of {det['C']}) on {det['threads']} threads, that time scaled "
            f"by C/sample")


def config_dict(args, inst, k, s, m, iters, beta):
    return {"workload": f"planted({inst.l},{inst.d}) t={inst.t} n={int(inst.lens[0])} k={k} s={s} "
                        f"m={m} em_iters={iters} pseudocount={beta}",
            "config_index": args.config, "t": inst.t, "n": int(inst.lens[0]), "l": inst.l,
            "d": inst.d, "k": k, "s": s, "m": m, "em_iters": iters, "x_lmers": inst.n_lmers,
            "precision": args.precision, "l2": "flushed between steps (512 MB write)",
            "parallelism": f"independent instances, one per GPU"}


# ---------------------------------------------------------------------------
# Batched serving mix (config 4)
# ---------------------------------------------------------------------------

def run_batched(args):
    """256 planted instances of uneven t, n, (l,d): one batched call
    (tensor-core EM) per step vs plain per-instance FP32 searches."""
    import torch

    import paper_1605_06904_gb300 as P
    torch.cuda.set_device(0)
    insts = mix_instances(args.n_inst)
    L = [i.l for i in insts]
    D = [i.d for i in insts]
    K = [i.params["k"] for i in insts]
    S = [i.params["s"] for i in insts]
    seeds = [4000 + q for q in range(len(insts))]
    M = [P.projection_default_params(i.lens, i.l, i.d, i.params["k"], i.params["s"], 0)[2]
         for i in insts]

    def step():
        return P.projection_find_batch([i.seqs for i in insts], L, D, K, S, M, seeds, em_iters=5,
                                       pseudocount=0.25, precision=P.PROJ_EM_BF16_SPLIT)

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    P.projection_trace_enable(True)
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = step()  # synchronises
        times.append(time.perf_counter() - t0)
    P.projection_trace_enable(False)
    clk = clocks.stop()
    em_ms, em_launches = P.projection_trace_read("em_tc")
    _, all_launches = P.projection_trace_read("")
    T = float(np.mean(times))
    C = sum(r["n_candidates"] for r in res)
    x = [i.n_lmers for i in insts]
    scores = sum(r["n_candidates"] * xi for r, xi in zip(res, x)) * 6

    # plain: one FP32 search per instance, one after another
    plain_t0 = time.perf_counter()
    plain = []
    for q, inst in enumerate(insts):
        plain.append(P.projection_find(inst.ascii, inst.seq_off, inst.l, inst.d, K[q], S[q], M[q],
                                       seed=seeds[q], em_iters=5, pseudocount=0.25,
                                       precision=P.PROJ_EM_FP32))
    plain_T = time.perf_counter() - plain_t0
    same = float(np.mean([a["consensus"] == b["consensus"] for a, b in zip(res, plain)]))
    planted = float(np.mean([r["consensus"] == i.motif for r, i in zip(res, insts)]))
    pk, pk_kind = peaks()
    flops = sum(r["n_candidates"] * xi * (5 * 16 * i.l + 8 * i.l)
                for r, xi, i in zip(res, x, insts)) * args.steps
    achieved = flops / (em_ms / 1e3) / 1e12 if em_ms > 0 else None
    peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    line = {
        "metric": METRIC, "value": len(insts) / T, "unit": "instances/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": T * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16-split",
        "data": "synthetic",
        "config": {"workload": f"batched mix of {len(insts)} planted instances, t~U[10,40], "
                               "n~U[300,1200], (l,d) in {(11,2),(13,3),(15,4),(17,5),(19,6)}, "
                               "k=min(l-d,ceil(log4(t*n))), s=4, m=bound(q=0.95), 5 EM iters",
                   "config_index": 4, "instances": len(insts), "trials": int(sum(M)),
                   "candidates": int(C), "l2": "inputs copied from host each step"},
        "scores_per_s": scores / T, "hashes_per_s": sum(m * xi for m, xi in zip(M, x)) / T,
        "plain_fp32_instances_per_s": len(insts) / plain_T,
        "batched_vs_plain": plain_T / T, "equal_motif_frac": same,
        "planted_motif_recovered_frac": planted,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if achieved else None, "traffic": None,
                     "kernel": "em_tc_kernel", "launches": em_launches,
                     "avg_launch_ms": em_ms / max(1, em_launches),
                     "peak_source": f"bf16_tflops_sustained ({pk_kind})"},
        "clocks": clk,
        "e2e": {"value": len(insts) / T, "unit": "instances/s",
                "h2d_bytes_per_step": int(sum(i.ascii.size for i in insts)),
                "d2h_bytes_per_step": int(sum(16 * i.l + 4 * i.t + i.l + 32 for i in insts))},
        "gpu_launches": all_launches / max(1, args.steps), "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Serving-scale input, top buckets refined (config 5)
# ---------------------------------------------------------------------------

def run_top(args):
    """t = 2000 x n = 500, Markov GC40 background, (20,5) ZOOPS; m = 500 trials
    hashed, the 1024 largest enriched buckets refined by 10 EM iterations.
    Timed: the whole search with BF16-split EM (and FP32 EM beside it).
    Errors of both EM paths against the FP64 oracle on a sample of the refined
    models are reported."""
    import torch

    import oracle as O
    import paper_1605_06904_gb300 as P
    torch.cuda.set_device(0)
    inst = instance_for_config(5)
    p = inst.params
    k, s, m, iters, beta, top = p["k"], p["s"], p["m"], p["em_iters"], p["beta"], p["top"]
    if args.trials:  # a shorter run of the same instance (profiling captures)
        m = args.trials
    seed = 1005
    dev = torch.device("cuda", 0)
    packed = P.projection_pack(torch.from_numpy(inst.ascii).to(dev))
    off = inst.seq_off
    x = inst.n_lmers
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step(prec):
        if args.zoops:
            return P.projection_find_packed_zoops(packed, off, inst.l, inst.d, k, s, m, seed=seed,
                                                  em_iters=iters, pseudocount=beta,
                                                  precision=prec, site_prob=args.zoops, top=top)
        return P.projection_find_packed_top(packed, off, inst.l, inst.d, k, s, m, seed=seed,
                                            em_iters=iters, pseudocount=beta, precision=prec,
                                            top=top)

    for _ in range(args.warmup):
        res = step(P.PROJ_EM_BF16_SPLIT)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    P.projection_trace_enable(True)
    ms = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res = step(P.PROJ_EM_BF16_SPLIT)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    P.projection_trace_enable(False)
    clk = clocks.stop()
    em_ms, em_launches = P.projection_trace_read("em_tc")
    hash_ms, _ = P.projection_trace_read("hash")
    hc_ms, hc_launches = P.projection_trace_read("hash_count")
    _, all_launches = P.projection_trace_read("")
    phases = {name: P.projection_trace_read(name)[0] / args.steps
              for name in ("hash_partition", "hash_count", "hash_scan", "hash_fill", "select",
                           "theta0", "em_tc", "em_reduce", "finalize")}
    hist_peak = P.projection_hist_peak(k)
    hc_rate = m * x * hc_launches / (hc_ms / 1e3) if hc_ms > 0 else None
    T = float(np.mean(ms)) / 1e3
    fp32_t0 = time.perf_counter()
    res32 = step(P.PROJ_EM_FP32)
    T32 = time.perf_counter() - fp32_t0
    R = res["n_refined"]
    scores = x * R * (iters + 1)

    errs, n_err = em_error_report(P, inst, packed, k, s, seed, iters, beta, dev,
                                  n_sample=args.err_sample, trials=1,
                                  site_prob=args.zoops or None)
    pk, pk_kind = peaks()
    flops = args.steps * x * R * (iters * 16 * inst.l + 8 * inst.l)
    achieved = flops / (em_ms / 1e3) / 1e12 if em_ms > 0 else None
    peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    line = {
        "metric": METRIC, "value": scores / T, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": T * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16-split", "data": "synthetic",
        "config": {"workload": f"markov-gc40 zoops(20,5) t=2000 n=500 k=10 s=4 m={m} top=1024 "
                               "em_iters=10 pseudocount=0.25"
                               + (f" em_model=zoops(site_prob={args.zoops})" if args.zoops
                                  else " em_model=oops"), "config_index": 5,
                   "x_lmers": x, "l2": "flushed between steps (512 MB write)"},
        "hashes_per_s": m * x / T, "hash_ms_per_step": hash_ms / args.steps,
        "ms_per_step_by_phase": phases,
        "n_candidates": res["n_candidates"], "n_refined": R,
        "fp32_ms_per_step": T32 * 1e3, "motif_found": res["consensus"],
        "motif_found_fp32": res32["consensus"], "motif_planted": inst.motif,
        "errors_vs_fp64_oracle": errs,
        "error_sample": f"{n_err} largest buckets of trial 0 (oracle hash + theta0), {iters} EM iters",
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if achieved else None, "traffic": None,
                     "kernel": "em_tc_kernel", "launches": em_launches,
                     "avg_launch_ms": em_ms / max(1, em_launches),
                     "peak_source": f"bf16_tflops_sustained ({pk_kind})"},
        "hash_roofline": {"kernel": "hash_kernel<count>", "bound": "smem_atomic",
                          "achieved": hc_rate, "peak": hist_peak, "unit": "updates/s",
                          "frac": hc_rate / hist_peak if hc_rate else None,
                          "avg_launch_ms": hc_ms / max(1, hc_launches),
                          "peak_source": f"projection_hist_peak({k}) measured in this run"},
        "clocks": clk, "gpu_launches": all_launches / max(1, args.steps), "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------

def exp_bound(P, flops, exps, tensor_peak_tflops, em_ms):
    """The EM kernel's two ceilings side by side: tensor time (algorithmic FLOPs
    at the tensor peak) and exponential time (one exp2 per score at the exp2
    rate measured now), and which of them binds."""
    rate = P.projection_ex2_peak()
    t_tensor = flops / (tensor_peak_tflops * 1e12) * 1e3
    t_exp = exps / rate * 1e3
    return {"ex2_per_s": rate, "tensor_ms": t_tensor, "exp_ms": t_exp,
            "binding": "tensor" if t_tensor >= t_exp else "exp",
            "frac_of_binding": max(t_tensor, t_exp) / em_ms if em_ms > 0 else None,
            "peak_source": "projection_ex2_peak() measured in this run"}


def protein_measure(P, stream, flush, reps=5):
    """The 20-letter search on a planted protein (15,4) input: t=20 sequences of
    600 residues, k=4 (base-20 keys), s=3, m=40 trials, 5 EM iterations.  Device
    time per search (host copies included, small) and its phases."""
    import torch
    from synth import planted_protein
    inst = planted_protein(2024, 0, 20, 600, 15, 4)
    k, s, m, iters, beta = 4, 3, 40, 5, 0.25
    ascii, off = inst.ascii, inst.seq_off
    for _ in range(2):
        r = P.projection_find_protein(ascii, off, inst.l, k, s, m, seed=1, em_iters=iters,
                                      pseudocount=beta)
    times = []
    P.projection_trace_enable(True)
    for i in range(reps):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = P.projection_find_protein(ascii, off, inst.l, k, s, m, seed=1, em_iters=iters,
                                      pseudocount=beta)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    P.projection_trace_enable(False)
    x = int(np.sum(inst.lens - inst.l + 1))
    ms = float(np.median(times))
    phases = {name: P.projection_trace_read(name)[0] / reps
              for name in ("pack", "allpairs", "enrich_sort", "theta0", "em_fp32", "em_reduce",
                           "finalize")}
    return {"workload": "planted protein (15,4) t=20 n=600, k=4 s=3 m=40, 5 EM iters",
            "ms_per_search": ms, "n_candidates": r["n_candidates"],
            "scores_per_s": r["n_candidates"] * x * (iters + 1) / (ms / 1e3),
            "enrichment": "per-trial shared-memory sort of (key, l-mer) pairs (x <= 16384)",
            "ms_by_phase": phases, "motif_found": r["consensus"], "motif_planted": inst.motif}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--precision", choices=["fp32", "bf16split"], default="bf16split")
    ap.add_argument("--ref-sample", type=int, default=6000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-inst", type=int, default=256)
    ap.add_argument("--err-sample", type=int, default=16)
    ap.add_argument("--zoops", type=float, default=0.0,
                    help="config 5 only: refine with the ZOOPS EM at this site probability")
    ap.add_argument("--trials", type=int, default=0,
                    help="config 5 only: hash this many trials instead of 500 (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.config == 4:
        return run_batched(args)
    if args.config == 5:
        return run_top(args)

    import torch
    import torch.distributed as dist

    import paper_1605_06904_gb300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    inst = rank_instance(args.config, rank)  # weak scaling: one instance per GPU
    p = dict(inst.params)
    k, s, m = resolve(inst, p)
    iters, beta, seed = p["em_iters"], p["beta"], 1000 + args.config
    prec = P.PROJ_EM_FP32 if args.precision == "fp32" else P.PROJ_EM_BF16_SPLIT
    off = inst.seq_off
    x = inst.n_lmers

    ascii_host = torch.from_numpy(inst.ascii).pin_memory()
    packed = P.projection_pack(ascii_host.to(dev))  # resident input for the device leg
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        return P.projection_find_packed(packed, off, inst.l, inst.d, k, s, m, seed=seed,
                                        em_iters=iters, pseudocount=beta, precision=prec)

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()
    C = res["n_candidates"]

    # ---- timed region: K steps, L2 flushed between steps, per-step events
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    evf = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    P.projection_trace_enable(True)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        evf[i][0].record(stream)
        flush.fill_(i & 0xFF)
        evf[i][1].record(stream)
        ev[i][0].record(stream)
        res = step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    P.projection_trace_enable(False)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    flush_ms = [a.elapsed_time(b) for a, b in evf]
    T = float(np.sum(step_ms)) / 1e3

    scores_step = x * C * (iters + 1)
    em_name = "em_fp32" if prec == P.PROJ_EM_FP32 else "em_tc"
    em_ms, em_launches = P.projection_trace_read(em_name)
    hc_ms, hc_launches = P.projection_trace_read("hash_count")
    _, all_launches = P.projection_trace_read("")
    phases = {name: P.projection_trace_read(name)[0] / args.steps
              for name in ("background", "positions", "hash_count", "hash_scan", "hash_fill",
                           "theta0", "em_tc", "em_fp32", "em_reduce", "finalize")}
    phases["all_kernels"] = P.projection_trace_read("")[0] / args.steps

    (job_scores, job_hashes, job_steps), T_job = reduce_over_ranks(
        [scores_step * args.steps, m * x * args.steps, args.steps], T, dev, world)
    value = job_scores / T_job
    hashes = job_hashes / T_job
    inst_rate = job_steps / T_job

    # ---- roofline of the dominant kernel (EM)
    pk, pk_kind = peaks()
    if prec == P.PROJ_EM_FP32:
        # algorithmic FP32 operations: per score l gather-adds (E) + exp and sum
        # (2) + l weighted adds (M-step launches only)
        ops = args.steps * x * C * (iters * (2 * inst.l + 2) + (inst.l + 2))
        achieved = ops / (em_ms / 1e3) / 1e12 if em_ms > 0 else None
        peak = SMS * FP32_LANES_PER_SM * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": None,
                "kernel": "em_fp32_kernel", "launches": em_launches,
                "avg_launch_ms": em_ms / max(1, em_launches),
                "peak_source": "152 SMs x 128 FP32 lanes x 2070 MHz (derived)"}
    else:
        # algorithmic FLOPs of the two one-hot contractions at K = 4l: 2*4l for the
        # scores (every launch) + 2*4l for the counts (M-step launches); the hi + lo
        # duplication and the K padding the kernel executes are not credited
        flops = args.steps * x * C * (iters * 16 * inst.l + 8 * inst.l)
        achieved = flops / (em_ms / 1e3) / 1e12 if em_ms > 0 else None
        peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
        traffic = (recorded_traffic("em_tc_kernel_planted15_4.md",
                                    ["em_tc.cu", "tc.cuh", "em_batch.cuh"])
                   if args.config == 2 else None)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "kernel": "em_tc_kernel", "launches": em_launches,
                "avg_launch_ms": em_ms / max(1, em_launches),
                "peak_source": f"bf16_tflops_sustained ({pk_kind})",
                "exp_bound": exp_bound(P, flops, args.steps * x * C * (iters + 1), peak, em_ms)}

    # ---- the bucket-counting kernel against the shared-memory histogram rate
    hist_peak = P.projection_hist_peak(k)
    hc_rate = m * x * hc_launches / (hc_ms / 1e3) if hc_ms > 0 else None
    hash_roof = {"kernel": "hash_kernel<count>", "bound": "smem_atomic", "achieved": hc_rate,
                 "peak": hist_peak, "unit": "updates/s",
                 "frac": hc_rate / hist_peak if hc_rate else None,
                 "avg_launch_ms": hc_ms / max(1, hc_launches),
                 "peak_source": f"projection_hist_peak({k}) measured in this run"}

    # ---- the low-memory all-pairs enrichment on the same trials (no 4^k table):
    # x^2 key comparisons per trial, against the histogram path's count + fill
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    ap = P.trial_hash_allpairs(packed, off, inst.l, k, s, seed, 0, m, cap_cand=max(1, C),
                               cap_members=max(1, res["n_members"]) if "n_members" in res else None)
    a1.record(stream)
    torch.cuda.synchronize()
    ap_ms = a0.elapsed_time(a1)
    allpairs = {"ms_for_all_trials": ap_ms, "compares_per_s": m * x * x / (ap_ms / 1e3),
                "same_candidates": ap["n_candidates"] == C,
                "hash_ms_histogram_path": P.projection_trace_read("hash")[0] / args.steps}
    protein = protein_measure(P, stream, flush) if args.config == 2 else None

    # ---- end to end through the public API: host ASCII in, result out
    e2e_times = []
    for i in range(max(3, min(args.steps, 10))):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r2 = P.projection_find(ascii_host, off, inst.l, inst.d, k, s, m, seed=seed,
                               em_iters=iters, pseudocount=beta, precision=prec)
        e2e_times.append(time.perf_counter() - t0)
    assert r2["consensus"] == res["consensus"]
    e2e_T = float(np.mean(e2e_times))
    h2d = int(inst.ascii.size) + 2 * 4 * (inst.t + 1)
    d2h = 8 + 16 + 8 + 4 * inst.t + inst.l + 4 + 16 * inst.l + 8 + 4 + 4
    e2e = {"value": scores_step / e2e_T, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": e2e_T * 1e3}

    # the other precision through the same call (one step, after the timed region)
    other = P.PROJ_EM_FP32 if prec == P.PROJ_EM_BF16_SPLIT else P.PROJ_EM_BF16_SPLIT
    flush.fill_(0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r_other = P.projection_find_packed(packed, off, inst.l, inst.d, k, s, m, seed=seed,
                                       em_iters=iters, pseudocount=beta, precision=other)
    e1.record(stream)
    torch.cuda.synchronize()
    other_ms = e0.elapsed_time(e1)
    errs = None
    if rank == 0 and not args.no_cpu_baseline:
        errs, n_err = em_error_report(P, inst, packed, k, s, seed, iters, beta, dev,
                                      n_sample=args.err_sample)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": T_job * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == P.PROJ_EM_FP32 else "bf16-split",
        "data": "synthetic", "config": config_dict(args, inst, k, s, m, iters, beta),
        "hashes_per_s": hashes, "instances_per_s": inst_rate,
        "n_candidates": C, "scores_per_step": scores_step,
        "motif_found": res["consensus"], "motif_planted": inst.motif,
        ("fp32" if other == P.PROJ_EM_FP32 else "bf16_split") + "_ms_per_step": other_ms,
        ("motif_found_fp32" if other == P.PROJ_EM_FP32 else "motif_found_bf16_split"):
            r_other["consensus"],
        "errors_vs_fp64_oracle": errs,
        "error_sample": (f"{args.err_sample} largest buckets of trials 0-1 (oracle hash + "
                         f"theta0), {iters} EM iters") if errs else None,
        "ms_per_step_by_phase": phases,
        "wall_ms_per_step": wall * 1e3 / args.steps,
        "flush_ms_per_step": float(np.mean(flush_ms)),
        "roofline": roof, "hash_roofline": hash_roof, "allpairs_enrichment": allpairs,
        "protein_search": protein, "clocks": clk, "e2e": e2e,
        "gpu_launches": all_launches / max(1, args.steps),
        "cpu_baseline": None,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        tt, det = oracle_step(inst, k, s, m, seed, iters, beta, max_sample=args.ref_sample)
        line["cpu_baseline"] = {"value": scores_step / tt, "unit": UNIT, "cores": det["threads"],
                                "kind": "oracle", "sample": sample_text(det, m),
                                "seconds_per_step_extrapolated": tt}
        # the same oracle on one core (a smaller EM sample, same extrapolation)
        tt1, det1 = oracle_step(inst, k, s, m, seed, iters, beta,
                                max_sample=max(1, args.ref_sample // 16), nthreads=1)
        line["cpu_baseline"]["single_thread"] = {
            "value": scores_step / tt1, "unit": UNIT, "cores": 1, "sample": sample_text(det1, m),
            "seconds_per_step_extrapolated": tt1}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
