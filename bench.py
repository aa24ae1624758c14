#!/usr/bin/env python
"""Throughput of the whole PROJECTION hot path (Algorithm 2 + Section 5.1 EM)
on one GB300, on seeded synthetic planted-motif inputs.

A step is one motif search over one instance: resident 2-bit input -> Philox
positions, projection, hashing and bucket counts for all m trials ->
enriched buckets -> theta^0 -> EM -> FP64 ranking, consensus, sites.

Default workload (the largest that runs on one GPU): a first-order Markov
background with 40% GC, t = 2000 sequences x n = 500 bp, a (20,5) motif
planted in 60% of them, k = 10, s = 4, m = 500 trials, the 1024 largest
enriched buckets refined by 10 EM iterations on the tensor cores (BF16 hi + lo
split, FP32 accumulation).  The same line carries, nested under
"sub_workloads", the planted (15,4) t=20 n=600 search (m = 172, every enriched
bucket refined) and the planted (18,6) t=20 n=1000 challenge search
(m = 2000), each with its own roofline.  --config 2|3 makes one of those the
main line; --config 4 runs the batched serving mix.

Prints one JSON line.  `value` is EM l-mer x PWM scores per second over the
whole step (scores per step = x * R * (em_iters + 1), R = refined buckets);
hashes/s and instances/s are reported beside it.

--impl reference times the CPU oracle (the FP64 statement of the method) on
the same workload: a sample of the trials hashed and a sample of the refined
candidates run through EM, each time scaled linearly to the whole step.
"""
from __future__ import annotations

import argparse
import hashlib
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
# stated fallbacks when no measured peaks are present (one earlier GB300 measurement)
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
FLUSH_BYTES = 512 << 20  # > 2x the 129 MB L2

# what the EM kernel executes per algorithmic FLOP is derived from its tile
# shapes: M = 128 candidate rows, N = 64 l-mers per tile, K padded to 16
EM_ROWS, EM_TILE = 128, 64

CFG_LABEL = {2: "planted(15,4) t=20 n=600", 3: "planted(18,6) t=20 n=1000",
             5: "markov-gc40 zoops(20,5) t=2000 n=500"}


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
        time.sleep(0.3)

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


def recorded_profile(profile: str, sources) -> dict:
    """Figures of a committed ncu summary (`key: value` lines), if the kernel
    sources still hash to what the capture was taken with (else {})."""
    try:
        text = open(os.path.join(ROOT, "profiles", profile)).read()
        h = hashlib.sha256()
        for s in sources:
            h.update(open(os.path.join(ROOT, "paper_1605_06904_gb300", "csrc", s), "rb").read())
        vals = dict(ln.strip().split(": ", 1) for ln in text.splitlines()
                    if ln.startswith("    ") and ": " in ln and not ln.strip().startswith("#"))
        if vals.get("source_sha256_16") != h.hexdigest()[:16]:
            return {}
        return {k: float(v) for k, v in vals.items() if k != "source_sha256_16"}
    except (OSError, ValueError):
        return {}


EM_SOURCES = ["em_tc.cu", "tc.cuh", "em_batch.cuh"]
EM_PROFILE = {2: "em_tc_kernel_planted15_4.md", 3: "em_tc_kernel_planted18_6.md",
              5: "em_tc_kernel_config5_top1024.md"}


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return dict(FALLBACK_PEAKS), "fallback"


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
                     "ll_max_rel": float((np.abs(g_ll - w_ll) / np.abs(w_ll)).max()),
                     "consensus_equal_frac": float(np.mean(
                         [O.consensus(g_pwm[q]) == O.consensus(w_pwm[q])
                          for q in range(len(sel))]))}
    out["sample"] = (f"{len(sel)} largest buckets of trials 0-{trials - 1} (oracle hash + "
                     f"theta0), {iters} EM iters; LL error relative to |LL|")
    return out


# ---------------------------------------------------------------------------
# CPU oracle leg (bounded samples, scaled linearly to the whole step)
# ---------------------------------------------------------------------------

def oracle_step(inst, k, s, m, seed, iters, beta, top=0, hash_trials=None, em_sample=6000,
                nthreads=None):
    """One oracle step on a bounded sample; returns (seconds for the whole step,
    extrapolated; details).  hash_trials: trials hashed (None = all m; their
    time is scaled by m / hash_trials).  EM runs on at most em_sample candidates
    (evenly spaced over the refined set) and its time is scaled by R / sample."""
    import oracle as O
    nthreads = nthreads or os.cpu_count() or 1
    codes = O.encode(inst.ascii)
    off = inst.seq_off
    ht = m if not hash_trials else min(m, hash_trials)
    t0 = time.perf_counter()
    h = O.hash_trials(codes, off, inst.l, k, s, seed, 0, ht)
    t_hash = time.perf_counter() - t0
    C_s = int(h["cand_key"].size)
    if top:
        pool = O.top_candidates(h["cand_cnt"], top)
        R = top
    else:
        pool = np.arange(C_s)
        R = None  # every enriched bucket of all m trials; scaled below
    stride = max(1, math.ceil(pool.size / max(1, em_sample)))
    idx = pool[::stride]
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
    if R is None:
        R = C_s * m / ht  # candidates of all m trials (exact when every trial is hashed)
    total = t_hash * (m / ht) + (t_th0 + t_em) * (R / max(1, idx.size))
    return total, {"R": R, "sample": int(idx.size), "hash_trials": ht, "m": m,
                   "t_hash": t_hash, "t_theta0": t_th0, "t_em": t_em, "threads": nthreads}


def sample_text(det):
    return (f"{det['hash_trials']} of {det['m']} trials hashed (1 thread, time x "
            f"{det['m'] / det['hash_trials']:.4g}); theta0 + EM on {det['sample']} of "
            f"{det['R']:.0f} refined candidates on {det['threads']} threads (time x "
            f"{det['R'] / max(1, det['sample']):.4g})")


def rank_instance(cfg: int, rank: int):
    """Weak scaling: rank r searches instance r of the workload."""
    return instance_for_config(cfg, rank)


def workload(cfg, rank=0, oracle_side=False):
    """(instance, k, s, m, em_iters, beta, top, seed) of a named workload; k, s
    and m left at 0 are resolved by the library (GPU leg) or by the oracle
    (CPU leg) with the same Section 5 formulas."""
    inst = rank_instance(cfg, rank)
    p = dict(inst.params)
    if oracle_side:
        import oracle as O
        k, s, m = O.default_params(inst.lens, inst.l, inst.d, p.get("k", 0), p.get("s", 0),
                                   p.get("m", 0))
    else:
        k, s, m = resolve(inst, p)
    return inst, k, s, m, p["em_iters"], p["beta"], p.get("top", 0), 1000 + cfg


def config_dict(cfg, inst, k, s, m, iters, beta, top, extra=None):
    d = {"workload": (f"{CFG_LABEL[cfg]} l={inst.l} d={inst.d} k={k} s={s} m={m} "
                      f"em_iters={iters} pseudocount={beta}"
                      + (f" top={top} buckets refined" if top else " all enriched buckets refined")),
         "config_index": cfg, "t": inst.t, "n": int(inst.lens[0]), "l": inst.l, "d": inst.d,
         "k": k, "s": s, "m": m, "em_iters": iters, "x_lmers": inst.n_lmers,
         "l2": "flushed between steps (512 MB write)",
         "parallelism": "independent instances, one per GPU (weak scaling)"}
    if extra:
        d.update(extra)
    return d


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.config == 4:
        print(json.dumps({"impl": "reference", "unavailable":
                          "the batched mix has no oracle leg of its own; the oracle arm runs "
                          "--config 2, 3 or 5"}), flush=True)
        return 0
    inst, k, s, m, iters, beta, top, seed = workload(args.config, oracle_side=True)
    ht, es = (args.ref_trials, args.ref_cands) if args.config == 5 else (None, args.ref_sample)
    for _ in range(args.warmup):
        oracle_step(inst, k, s, m, seed, iters, beta, top, ht, es)
    # a step is the bounded sample: ms_per_step is its measured time; the value
    # is the whole search's rate, from the sample's times scaled to the search
    times, walls, det = [], [], None
    for _ in range(args.steps):
        w0 = time.perf_counter()
        tt, det = oracle_step(inst, k, s, m, seed, iters, beta, top, ht, es)
        walls.append(time.perf_counter() - w0)
        times.append(tt)
    T = float(np.mean(times))
    x = inst.n_lmers
    scores = x * det["R"] * (iters + 1)
    value = scores / T
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(walls)) * 1e3,
        "ms_per_search_extrapolated": T * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": config_dict(args.config, inst, k, s, m, iters, beta, top,
                              {"em_model": f"zoops(site_prob={args.zoops})" if args.zoops
                               else "oops", "precision": args.precision}),
        "hashes_per_s": m * x / T, "instances_per_s": 1.0 / T,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": det["threads"], "kind": "oracle",
                         "sample": sample_text(det)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU measurements
# ---------------------------------------------------------------------------

PHASES = ("pack", "background", "positions", "hash_partition", "hash_count", "hash_scan",
          "hash_fill", "hash_table", "select", "hash_gather", "theta0", "em_xtiles", "em_tc",
          "em_fp32", "em_reduce", "finalize")


def em_executed_flops(inst, R, iters):
    """FLOPs the tensor-core EM executes for R candidates: per (128-candidate
    tile, 64-l-mer tile) the score MMA (hi + lo, K padded to 16) and, in M-step
    launches, the count MMA (P hi + lo)."""
    kp = 16 * math.ceil(4 * inst.l / 16)
    ns = np.maximum(inst.lens - inst.l + 1, 0)
    xt = int(np.sum((ns + EM_TILE - 1) // EM_TILE))
    ct = math.ceil(R / EM_ROWS)
    per = 2 * EM_ROWS * EM_TILE * kp * 2
    return ct * xt * per * (2 * iters + 1)


def fp32_roofline(inst, R, iters, em_ms, em_launches, sm_mhz=2070.0):
    """The FP32 EM kernel against its binding resource, the shared-memory pipe:
    per score l reads of the log-odds (E-step) and, in M-step launches, a read
    and a write of each of the l count entries and their compensation terms
    (4l more); 32 four-byte accesses per clock per SM on 152 SMs."""
    if not em_launches or em_ms <= 0:
        return None
    steps = em_launches / (iters + 1)
    acc = steps * inst.n_lmers * R * (iters * 5 * inst.l + inst.l)
    achieved = acc / (em_ms * 1e-3)
    peak = 152 * 32 * sm_mhz * 1e6
    return {"bound": "smem", "kernel": "em_fp32_kernel", "launches": em_launches,
            "avg_launch_ms": em_ms / em_launches, "achieved": achieved, "peak": peak,
            "unit": "shared-memory accesses/s", "frac": achieved / peak,
            "peak_source": "152 SMs x 32 accesses/clock x %g MHz" % sm_mhz}


def em_roofline(P, cfg, inst, R, iters, steps, em_ms, em_launches, pk, pk_kind):
    """Roofline of the tensor-core EM kernel: algorithmic FLOPs (the one-hot
    contractions at K = 4l: 8l per score for the E-step, 8l more in M-step
    launches) per launch over its CUDA-event launch time."""
    x = inst.n_lmers
    flops = steps * x * R * (iters * 16 * inst.l + 8 * inst.l)
    exe = steps * em_executed_flops(inst, R, iters)
    achieved = flops / (em_ms / 1e3) / 1e12 if em_ms > 0 else None
    burst = pk.get("bf16_tflops")
    sust = pk.get("bf16_tflops_sustained", burst)
    prof = recorded_profile(EM_PROFILE.get(cfg, ""), EM_SOURCES)
    scores_launch = x * R  # scores of one launch
    ins = prof.get("inst_executed_per_launch")
    rate = P.projection_ex2_peak()
    t_tensor = flops / (burst * 1e12) * 1e3
    t_exp = steps * x * R * (iters + 1) / rate * 1e3
    return {"bound": "tensor", "achieved": achieved, "peak": burst, "unit": "TFLOP/s",
            "frac": achieved / burst if achieved else None,
            "traffic": prof.get("traffic_bytes_per_launch"),
            "kernel": "em_tc_kernel", "launches": em_launches,
            "avg_launch_ms": em_ms / max(1, em_launches),
            "peak_source": f"bf16_tflops ({pk_kind}; burst: the kernel runs in a short step)",
            "frac_of_sustained": achieved / sust if achieved else None,
            "executed_flop_ratio": exe / flops,
            "executed_frac": (exe / (em_ms / 1e3) / 1e12) / burst if em_ms > 0 else None,
            "inst_per_score": (ins * 32 / scores_launch) if ins else None,
            "exp_bound": {"ex2_per_s": rate, "tensor_ms": t_tensor, "exp_ms": t_exp,
                          "binding": "tensor" if t_tensor >= t_exp else "exp",
                          "frac_of_binding": max(t_tensor, t_exp) / em_ms if em_ms > 0 else None,
                          "peak_source": "projection_ex2_peak() measured in this run"}}


def hash_roofline(P, k, m, x, steps, phases, pk=None, pk_kind=None):
    """The bucket-counting pass against the shared-memory histogram rate, and
    the whole hashing phase's time.  With a key-range partition (phase
    `hash_partition` present), also the partition and counting passes' HBM
    bytes as implemented (4 B per (trial, l-mer) written by the partition, the
    2-byte keys read back by the counting pass) against the measured HBM
    bandwidth: the hashing phase's memory roofline."""
    hc_ms, hc_launches = P.projection_trace_read("hash_count")
    hist_peak = P.projection_hist_peak(k)
    rate = m * x * steps / (hc_ms / 1e3) if hc_ms > 0 else None
    out = {"kernel": "hash_kernel<count>", "bound": "smem_atomic", "achieved": rate,
           "peak": hist_peak, "unit": "updates/s", "frac": rate / hist_peak if rate else None,
           "avg_launch_ms": hc_ms / max(1, hc_launches),
           "hash_phase_ms_per_step": sum(phases.get(n, 0.0) for n in
                                         ("hash_partition", "hash_count", "hash_scan",
                                          "hash_fill", "hash_table", "select", "hash_gather",
                                          "positions")),
           "peak_source": f"projection_hist_peak({k}) measured in this run"}
    part_ms = phases.get("hash_partition", 0.0) + phases.get("hash_count", 0.0)
    if phases.get("hash_partition") and pk:
        nbytes = m * x * (4 + 2)
        gbs = nbytes / (part_ms / 1e3) / 1e9
        out["partition_hbm"] = {"bound": "hbm", "bytes_per_step": nbytes,
                                "ms_per_step": part_ms, "achieved": gbs,
                                "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                                "frac": gbs / pk["hbm_gbs"] if pk.get("hbm_gbs") else None,
                                "peak_source": f"hbm_gbs ({pk_kind})",
                                "note": "partition writes + counting-pass reads, as implemented"}
    return out


def measure_search(P, cfg, inst, packed, k, s, m, seed, iters, beta, top, steps, warmup, flush,
                   stream, prec, zoops=0.0, clocks=None):
    """Times `steps` searches of one workload (L2 flushed before each, CUDA
    events on the launching stream), then the same number again with every
    library kernel traced for the per-kernel times."""
    import torch
    off = inst.seq_off

    def step():
        if zoops:
            return P.projection_find_packed_zoops(packed, off, inst.l, inst.d, k, s, m, seed=seed,
                                                  em_iters=iters, pseudocount=beta,
                                                  precision=prec, site_prob=zoops, top=top)
        if top:
            return P.projection_find_packed_top(packed, off, inst.l, inst.d, k, s, m, seed=seed,
                                                em_iters=iters, pseudocount=beta, precision=prec,
                                                top=top)
        return P.projection_find_packed(packed, off, inst.l, inst.d, k, s, m, seed=seed,
                                        em_iters=iters, pseudocount=beta, precision=prec)

    for _ in range(warmup):
        res = step()
    torch.cuda.synchronize()

    def timed(trace):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        P.projection_trace_enable(trace)
        w0 = time.perf_counter()
        for i in range(steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            out = step()  # synchronises on the result
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        w = time.perf_counter() - w0
        P.projection_trace_enable(False)
        return out, [a.elapsed_time(b) for a, b in ev], w

    # the timed steps run without the library's per-launch event trace (its
    # event records sit between the launches); a second pass over the same
    # number of steps, traced, gives the per-kernel times
    if clocks:
        clocks.start()
    res, step_ms, wall = timed(False)
    clk = clocks.stop() if clocks else None
    _, _, _ = timed(True)
    phases = {n: P.projection_trace_read(n)[0] / steps for n in PHASES}
    phases = {n: v for n, v in phases.items() if v > 0}
    all_ms, all_launches = P.projection_trace_read("")
    phases["all_kernels"] = all_ms / steps
    return {"res": res, "step_ms": step_ms, "wall_ms": wall * 1e3 / steps, "phases": phases,
            "launches": all_launches / steps, "clocks": clk}


def sub_workload(P, cfg, dev, stream, flush, steps, pk, pk_kind, with_extras=False):
    """A nested line for another workload: its own value, roofline and errors."""
    import torch
    inst, k, s, m, iters, beta, top, seed = workload(cfg)
    packed = P.projection_pack(torch.from_numpy(inst.ascii).to(dev))
    r = measure_search(P, cfg, inst, packed, k, s, m, seed, iters, beta, top, steps, 3, flush,
                       stream, P.PROJ_EM_BF16_SPLIT)
    res = r["res"]
    R = res["n_refined"]
    T = float(np.mean(r["step_ms"])) / 1e3
    em_ms, em_launches = P.projection_trace_read("em_tc")
    out = {"config": config_dict(cfg, inst, k, s, m, iters, beta, top),
           "value": inst.n_lmers * R * (iters + 1) / T, "unit": UNIT, "ms_per_step": T * 1e3,
           "steps": steps, "hashes_per_s": m * inst.n_lmers / T, "n_candidates":
               res["n_candidates"], "n_refined": R, "ms_per_step_by_phase": r["phases"],
           "gpu_launches": r["launches"],
           "roofline": em_roofline(P, cfg, inst, R, iters, steps, em_ms, em_launches, pk, pk_kind),
           "hash_roofline": hash_roofline(P, k, m, inst.n_lmers, steps, r["phases"], pk, pk_kind),
           "motif_found": res["consensus"], "motif_planted": inst.motif,
           "planted_recovered": res["consensus"] == inst.motif,
           "errors_vs_fp64_oracle": em_error_report(P, inst, packed, k, s, seed, iters, beta, dev,
                                                    n_sample=16, trials=2)}
    if with_extras:
        # the plain FP32 EM through the same call, one step
        flush.fill_(0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        P.projection_trace_enable(True)
        e0.record(stream)
        r32 = P.projection_find_packed(packed, inst.seq_off, inst.l, inst.d, k, s, m, seed=seed,
                                       em_iters=iters, pseudocount=beta, precision=P.PROJ_EM_FP32)
        e1.record(stream)
        torch.cuda.synchronize()
        P.projection_trace_enable(False)
        out["fp32_ms_per_step"] = e0.elapsed_time(e1)
        f_ms, f_launches = P.projection_trace_read("em_fp32")
        out["fp32_roofline"] = fp32_roofline(inst, r32["n_refined"], iters, f_ms, f_launches)
        out["motif_found_fp32"] = r32["consensus"]
        out["allpairs_enrichment"] = allpairs_measure(P, inst, packed, k, s, seed, m, res, stream)
        out["protein_search"] = protein_measure(P, stream, flush)
    return out


def allpairs_measure(P, inst, packed, k, s, seed, m, res, stream):
    """The low-memory all-pairs enrichment on the same trials (no 4^k table):
    x^2 key comparisons per trial."""
    import torch
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    ap = P.trial_hash_allpairs(packed, inst.seq_off, inst.l, k, s, seed, 0, m,
                               cap_cand=max(1, res["n_candidates"]),
                               cap_members=max(1, res.get("n_members", 1)))
    a1.record(stream)
    torch.cuda.synchronize()
    ms = a0.elapsed_time(a1)
    x = inst.n_lmers
    return {"ms_for_all_trials": ms, "compares_per_s": m * x * x / (ms / 1e3),
            "same_candidates": ap["n_candidates"] == res["n_candidates"]}


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
            "ms_by_phase": phases, "motif_found": r["consensus"], "motif_planted": inst.motif,
            "planted_recovered": r["consensus"] == inst.motif}


# ---------------------------------------------------------------------------
# Batched serving mix (config 4)
# ---------------------------------------------------------------------------

def run_batched(args):
    """256 planted instances of uneven t, n, (l,d): one batched call
    (tensor-core EM) per step vs the same searches as per-instance calls, with
    the tensor-core EM (what batching alone buys) and with the plain FP32 EM."""
    import torch

    import oracle as O
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
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    P.projection_trace_enable(True)
    times = []
    for q in range(args.steps):
        flush.fill_(q & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = step()  # synchronises
        times.append(time.perf_counter() - t0)
    P.projection_trace_enable(False)
    clk = clocks.stop()
    del flush
    em_ms, em_launches = P.projection_trace_read("em_tc")
    _, all_launches = P.projection_trace_read("")
    T = float(np.mean(times))
    C = sum(r["n_candidates"] for r in res)
    x = [i.n_lmers for i in insts]
    scores = sum(r["n_candidates"] * xi for r, xi in zip(res, x)) * 6

    def per_instance(prec):
        t0 = time.perf_counter()
        out = []
        for q, inst in enumerate(insts):
            out.append(P.projection_find(inst.ascii, inst.seq_off, inst.l, inst.d, K[q], S[q],
                                         M[q], seed=seeds[q], em_iters=5, pseudocount=0.25,
                                         precision=prec))
        return out, time.perf_counter() - t0

    per_instance(P.PROJ_EM_BF16_SPLIT)  # warm-up (schedules tuned per shape)
    plain_bf16, bf16_T = per_instance(P.PROJ_EM_BF16_SPLIT)
    plain_fp32, fp32_T = per_instance(P.PROJ_EM_FP32)

    def same(other):
        return float(np.mean([a["consensus"] == b["consensus"] for a, b in zip(res, other)]))

    planted = float(np.mean([r["consensus"] == i.motif for r, i in zip(res, insts)]))
    pk, pk_kind = peaks()
    flops = sum(r["n_candidates"] * xi * (5 * 16 * i.l + 8 * i.l)
                for r, xi, i in zip(res, x, insts)) * args.steps
    achieved = flops / (em_ms / 1e3) / 1e12 if em_ms > 0 else None
    peak = pk.get("bf16_tflops")

    # the oracle on a bounded sample of the mix: every 32nd instance searched
    # in full (all trials hashed, EM on every enriched bucket), time scaled by
    # the mix's total of EM scores
    cpu = None
    if not args.no_cpu_baseline:
        pick = list(range(0, len(insts), 32))
        nthreads = os.cpu_count() or 1
        t0 = time.perf_counter()
        sc = 0
        for q in pick:
            i = insts[q]
            w = O.find([z.decode() for z in i.seqs], i.l, i.d, K[q], S[q], M[q], seed=seeds[q],
                       em_iters=5, beta=0.25, nthreads=nthreads)
            sc += w["n_candidates"] * i.n_lmers * 6
        tc = time.perf_counter() - t0
        secs = tc * scores / max(1, sc)
        cpu = {"value": len(insts) / secs, "unit": "instances/s", "cores": nthreads,
               "kind": "oracle",
               "sample": f"{len(pick)} of {len(insts)} instances (every 32nd) searched in full "
                         f"({tc:.1f} s); time scaled by the whole mix's EM scores / the sample's"}
    line = {
        "metric": METRIC, "value": len(insts) / T, "unit": "instances/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": T * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16-split",
        "data": "synthetic",
        "config": {"workload": f"batched mix of {len(insts)} planted instances, t~U[10,40], "
                               "n~U[300,1200], (l,d) in {(11,2),(13,3),(15,4),(17,5),(19,6)}, "
                               "k=min(l-d,ceil(log4(t*n))), s=4, m=bound(q=0.95), 5 EM iters",
                   "config_index": 4, "instances": len(insts), "trials": int(sum(M)),
                   "candidates": int(C),
                   "l2": "flushed between steps (512 MB write); inputs copied from host each step"},
        "scores_per_s": scores / T, "hashes_per_s": sum(m * xi for m, xi in zip(M, x)) / T,
        "per_instance_bf16_split_instances_per_s": len(insts) / bf16_T,
        "batched_vs_per_instance_bf16_split": bf16_T / T,
        "equal_motif_frac_vs_per_instance_bf16_split": same(plain_bf16),
        "plain_fp32_instances_per_s": len(insts) / fp32_T,
        "batched_vs_plain": fp32_T / T, "equal_motif_frac": same(plain_fp32),
        "planted_motif_recovered_frac": planted,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if achieved else None, "traffic": None,
                     "kernel": "em_tc_kernel", "launches": em_launches,
                     "avg_launch_ms": em_ms / max(1, em_launches),
                     "peak_source": f"bf16_tflops ({pk_kind})"},
        "clocks": clk,
        "e2e": {"value": len(insts) / T, "unit": "instances/s",
                "h2d_bytes_per_step": int(sum(i.ascii.size for i in insts)),
                "d2h_bytes_per_step": int(sum(16 * i.l + 4 * i.t + i.l + 32 for i in insts)),
                "note": "the batched call takes host sequences and returns host results, so "
                        "`value` is already end to end"},
        "gpu_launches": all_launches / max(1, args.steps), "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Main line: one search workload (default: the serving-scale config 5)
# ---------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--config", type=int, default=5, choices=[2, 3, 4, 5])
    ap.add_argument("--precision", choices=["fp32", "bf16split"], default="bf16split")
    ap.add_argument("--ref-sample", type=int, default=6000,
                    help="configs 2/3: EM candidates per oracle step")
    ap.add_argument("--ref-trials", type=int, default=3,
                    help="config 5, reference arm: trials hashed per oracle step")
    ap.add_argument("--ref-cands", type=int, default=8,
                    help="config 5, reference arm: refined candidates run through EM per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="skip the nested workloads")
    ap.add_argument("--n-inst", type=int, default=256)
    ap.add_argument("--err-sample", type=int, default=16)
    ap.add_argument("--zoops", type=float, default=0.0,
                    help="config 5 only: refine with the ZOOPS EM at this site probability")
    ap.add_argument("--trials", type=int, default=0,
                    help="hash this many trials instead of the workload's m (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.config == 4:
        return run_batched(args)

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
    cfg = args.config

    inst, k, s, m, iters, beta, top, seed = workload(cfg, rank)  # weak scaling: instance = rank
    if args.trials:
        m = args.trials
    prec = P.PROJ_EM_FP32 if args.precision == "fp32" else P.PROJ_EM_BF16_SPLIT
    off = inst.seq_off
    x = inst.n_lmers

    ascii_host = torch.from_numpy(inst.ascii).pin_memory()
    packed = P.projection_pack(ascii_host.to(dev))  # resident input for the device leg
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    pk, pk_kind = peaks()

    if world > 1:
        dist.barrier()
    r = measure_search(P, cfg, inst, packed, k, s, m, seed, iters, beta, top, args.steps,
                       args.warmup, flush, stream, prec, zoops=args.zoops,
                       clocks=ClockSampler(local))
    if world > 1:
        dist.barrier()
    res = r["res"]
    R = res["n_refined"]
    T = float(np.sum(r["step_ms"])) / 1e3
    scores_step = x * R * (iters + 1)
    em_name = "em_fp32" if prec == P.PROJ_EM_FP32 else "em_tc"
    em_ms, em_launches = P.projection_trace_read(em_name)
    (job_scores, job_hashes, job_steps), T_job = reduce_over_ranks(
        [scores_step * args.steps, m * x * args.steps, args.steps], T, dev, world)

    # ---- rooflines: the EM kernel (tensor pipe) and the hashing phase
    if prec == P.PROJ_EM_FP32:
        roof = fp32_roofline(inst, R, iters, em_ms, em_launches)
    else:
        roof = em_roofline(P, cfg, inst, R, iters, args.steps, em_ms, em_launches, pk, pk_kind)
    hroof = hash_roofline(P, k, m, x, args.steps, r["phases"], pk, pk_kind)
    dominant = max((v, n) for n, v in r["phases"].items() if n != "all_kernels")[1]

    # ---- end to end through the public API: host ASCII in, result out
    e2e_times = []
    for i in range(max(3, min(args.steps, 10))):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if top:
            r2 = P.projection_find_top(ascii_host, off, inst.l, inst.d, k, s, m, seed=seed,
                                       em_iters=iters, pseudocount=beta, precision=prec, top=top)
        else:
            r2 = P.projection_find(ascii_host, off, inst.l, inst.d, k, s, m, seed=seed,
                                   em_iters=iters, pseudocount=beta, precision=prec)
        e2e_times.append(time.perf_counter() - t0)
    e2e_T = float(np.mean(e2e_times))
    h2d = int(inst.ascii.size) + 8 * (inst.t + 1)
    d2h = 96 + 4 * inst.t + inst.l + 16 * inst.l
    e2e = {"value": scores_step / e2e_T, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": e2e_T * 1e3,
           "same_motif_as_device_leg": r2["consensus"] == res["consensus"]}

    line = {
        "metric": METRIC, "value": job_scores / T_job, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": T_job * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == P.PROJ_EM_FP32 else "bf16-split",
        "data": "synthetic",
        "config": config_dict(cfg, inst, k, s, m, iters, beta, top,
                              {"em_model": f"zoops(site_prob={args.zoops})" if args.zoops
                               else "oops", "precision": args.precision}),
        "hashes_per_s": job_hashes / T_job, "instances_per_s": job_steps / T_job,
        "n_candidates": res["n_candidates"], "n_refined": R, "scores_per_step": scores_step,
        "motif_found": res["consensus"], "motif_planted": inst.motif,
        "planted_recovered": res["consensus"] == inst.motif,
        "ms_per_step_by_phase": r["phases"], "dominant_kernel_phase": dominant,
        "wall_ms_per_step": r["wall_ms"],
        "roofline": roof, "hash_roofline": hroof, "clocks": r["clocks"], "e2e": e2e,
        "gpu_launches": r["launches"], "cpu_baseline": None,
    }
    if rank == 0 and world == 1:
        # the other precision through the same call (one step, after the timed region)
        other = P.PROJ_EM_FP32 if prec == P.PROJ_EM_BF16_SPLIT else P.PROJ_EM_BF16_SPLIT
        flush.fill_(0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if top:
            r_other = P.projection_find_packed_top(packed, off, inst.l, inst.d, k, s, m, seed=seed,
                                                   em_iters=iters, pseudocount=beta,
                                                   precision=other, top=top)
        else:
            r_other = P.projection_find_packed(packed, off, inst.l, inst.d, k, s, m, seed=seed,
                                               em_iters=iters, pseudocount=beta, precision=other)
        e1.record(stream)
        torch.cuda.synchronize()
        oname = "fp32" if other == P.PROJ_EM_FP32 else "bf16_split"
        line[f"{oname}_ms_per_step"] = e0.elapsed_time(e1)
        line[f"motif_found_{oname}"] = r_other["consensus"]
        if not args.no_cpu_baseline:
            line["errors_vs_fp64_oracle"] = em_error_report(
                P, inst, packed, k, s, seed, iters, beta, dev, n_sample=args.err_sample,
                trials=1 if cfg == 5 else 2, site_prob=args.zoops or None)
        if not args.no_sub and cfg == 5:
            line["sub_workloads"] = {
                CFG_LABEL[c]: sub_workload(P, c, dev, stream, flush, st, pk, pk_kind,
                                           with_extras=(c == 2))
                for c, st in ((2, 20), (3, 5))}
        if not args.no_cpu_baseline:
            ht = 16 if cfg == 5 else None
            es = 48 if cfg == 5 else args.ref_sample
            tt, det = oracle_step(inst, k, s, m, seed, iters, beta, top, ht, es)
            line["cpu_baseline"] = {"value": scores_step / tt, "unit": UNIT,
                                    "cores": det["threads"], "kind": "oracle",
                                    "sample": sample_text(det),
                                    "seconds_per_step_extrapolated": tt}
            # the same oracle on one core (smaller samples, same scaling)
            tt1, det1 = oracle_step(inst, k, s, m, seed, iters, beta, top,
                                    4 if cfg == 5 else None, 4 if cfg == 5 else
                                    max(1, args.ref_sample // 16), nthreads=1)
            line["cpu_baseline"]["single_thread"] = {
                "value": scores_step / tt1, "unit": UNIT, "cores": 1, "sample": sample_text(det1),
                "seconds_per_step_extrapolated": tt1}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
