"""Benchmark: lnL + gradient evaluations per second of the epoch-model tree
likelihood on one B300, with the partials pass against the HBM roofline.

Workload (default): GTR nucleotide model, 3 epochs at 1/3 and 2/3 of the
root height, 500-taxon coalescent tree, 10,000 patterns with weights
U{1..20}, 4 discrete-gamma categories (alpha = 0.5), FP32 partials with
per-pattern power-of-two scaling; FP64 eigendecomposition, segment
exponentials and epoch products.  Synthetic seeded data.

A step is one pass of the whole path: branch segmentation, normalisation and
eigendecomposition of every Q_k, segment exponentials and epoch products,
pruning with rescaling, root log-sum, pre-order adjoint, per-branch adjoints
and the chain rule to node heights, boundaries, model parameters and branch
rates.  `value` is measured with all inputs resident on the device (CUDA
graph replays, CUDA events on the library's stream); `e2e` goes through the
C ABI from host arrays every step (uploads of Q, dQ, tree, tip codes and
weights; lnL and gradient read back), wall clock with the device drained.

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload (the reference arm of this comparison).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "lnL+gradient evals/sec & partials GB/s (%HBM roofline) vs plain FP64 GPU path at <=1e-5 rel"
UNIT = "evals/s"


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def make_workload(name):
    import synth

    if name == "gtr":
        w = synth.gtr_500taxa()
        return w, {"workload": "GTR 3-epoch, 500-taxon coalescent, 10,000 patterns, 4 gamma categories",
                   "taxa": 500, "patterns": 10000, "categories": 4, "states": 4, "epochs": 3,
                   "params": int(w.n_params)}
    if name == "gy94":
        w = synth.gy94_128taxa()
        return w, {"workload": "GY94 61-state 4-epoch, 128-taxon coalescent, 5,000 codon sites",
                   "taxa": 128, "patterns": int(w.n_patterns), "categories": 4, "states": 61,
                   "epochs": 4, "params": int(w.n_params)}
    if name == "seasonal":
        w = synth.flu_seasonal()
        return w, {"workload": "seasonal phylogeography: 522 dated taxa, 7 locations, 13 epochs "
                               "alternating two processes, one trait",
                   "taxa": 522, "patterns": 1, "categories": 1, "states": 7, "epochs": 13,
                   "params": int(w.n_params)}
    if name == "aa":
        w = synth.amino_acid()
        return w, {"workload": "amino acid 20-state 3-epoch, 200-taxon coalescent, 2,000 sites",
                   "taxa": 200, "patterns": int(w.n_patterns), "categories": 4, "states": 20,
                   "epochs": 3, "params": int(w.n_params)}
    raise SystemExit(f"unknown workload {name}")


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:  # sampler running before timing
                time.sleep(0.02)
            self.lines.clear()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic bytes of one partials pass (pruning over all internal nodes,
# K = 4 FP32 layout: 16 B per (category, pattern) vector, 1 B tip codes,
# 2 B scale exponents) plus the root log-sum
# ---------------------------------------------------------------------------
# DRAM bytes of one partials pass (the k4_post levels and k4_walk_post of one
# evaluation) on the GTR 500-taxon workload, from one ncu capture of those
# launches with warm L2 (dram__bytes_read.sum + dram__bytes_write.sum).
# Reported only while the kernel source is the one that was measured.
PARTIALS_TRAFFIC = {"source": "paper_1309_3075_b300/csrc/k_k4.cu",
                    "sha1": "a983f79822a0cca755b9c88c626c75824b98a782", "bytes": 216046848}


def measured_traffic(workload):
    import hashlib
    if workload != "gtr":
        return None
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), PARTIALS_TRAFFIC["source"])
    try:
        with open(path, "rb") as f:
            digest = hashlib.sha1(f.read()).hexdigest()
    except OSError:
        return None
    return PARTIALS_TRAFFIC["bytes"] if digest == PARTIALS_TRAFFIC["sha1"] else None


def partials_bytes(w):
    """Bytes the partials pass (pruning, rescaling, root log-sum) must move in
    this design: every stored partial written once and read once by its
    parent, one-byte tip codes, int16 exponents written and summed, the root's
    per-pattern outputs.  At K = 4, cherries (non-root nodes whose children
    are both tips) are not stored; their parents read the two tip codes
    instead.  Other K store every internal node (rows of 4 * Kp bytes)."""
    N, P, C = w.n_taxa, w.n_patterns, w.n_categories
    if w.K != 4:
        kp = 64 if w.K > 32 else (w.K + 3) // 4 * 4
        vec = 4 * kp * C * P
        return (N - 1) * (2 * vec + 4 * P) + N * P + 40 * P
    nn = 2 * N - 1
    parent = np.asarray(w.parent)
    kids = [[] for _ in range(nn)]
    for v in range(nn):
        if parent[v] >= 0:
            kids[parent[v]].append(v)
    root = int(np.where(parent < 0)[0][0])
    cherry = [u >= N and u != root and all(k < N for k in kids[u]) for u in range(nn)]
    vec = 16 * C * P
    total = 0
    for u in range(N, nn):
        if cherry[u]:
            continue
        total += vec + 2 * P                     # write the partial and its exponents
        for k in kids[u]:
            total += P if k < N else (2 * P if cherry[k] else vec)
    total += (N - 1) * 2 * P                     # exponents summed per pattern
    total += 8 * P + 8 * P + 8 * P + 16 * P      # site log, weights, site lnL; root outputs
    return total


def adjoint_bytes(w):
    """Bytes the gradient pass must move in this design: the outside partial
    U of every internal non-root node written once (by its parent's level)
    and read once (by its own), every stored partial read once more, tip
    codes, exponents and pattern weights once per internal node; the G tile
    sums and the chain rule are small.  At K = 4 the cherries' partials are
    not stored (recomputed from their tips' codes)."""
    N, P, C = w.n_taxa, w.n_patterns, w.n_categories
    nn = 2 * N - 1
    kp = 4 if w.K <= 4 else (64 if w.K > 32 else (w.K + 3) // 4 * 4)
    vec = 4 * kp * C * P
    parent = np.asarray(w.parent)
    kids = [[] for _ in range(nn)]
    for v in range(nn):
        if parent[v] >= 0:
            kids[parent[v]].append(v)
    root = int(np.where(parent < 0)[0][0])
    cherry = [u >= N and u != root and all(k < N for k in kids[u]) for u in range(nn)]
    stored = sum(1 for u in range(N, nn) if not (w.K == 4 and cherry[u]))
    return (N - 2) * 2 * vec + stored * vec + N * P + (N - 1) * 6 * P


def survey_bytes(w):
    """The same pass counted with every internal node stored (no cherry
    tables): the reference figure for this pass."""
    N, P, C = w.n_taxa, w.n_patterns, w.n_categories
    vec = 16 * C * P
    return (N - 1) * (2 * vec + 4 * P) + N * P + 40 * P


def l2_note(w):
    """Whether the step's partials (forward and adjoint, FP32) exceed the
    126 MB L2, so that successive steps cannot reuse them from cache."""
    mb = 2 * (w.n_taxa - 1) * w.n_categories * w.n_patterns * (4 if w.K <= 4 else 4 * w.K) * 4 / 1e6
    if mb > 126:
        return f"working set > L2 (forward + adjoint partials {mb:.0f} MB per step)"
    return f"working set {mb:.1f} MB fits in L2 (latency-bound shape)"


def max_over_ranks(x, world):
    """Largest x over the ranks of the default process group (the slowest rank's
    time is the job's time); x itself when there is one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, seconds, world):
    """Whole-job throughput: the units all replicas processed over the slowest
    replica's time."""
    return world * units_per_rank / seconds


def run_ours(args, w, cfg, rank, world):
    import torch

    from paper_1309_3075_b300 import binding
    from paper_1309_3075_b300.binding import EPOCH_FP32, EPOCH_FP32_TC, EPOCH_FP64, EpochLikelihood

    dev = rank % max(torch.cuda.device_count(), 1)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    # above 8 states the contractions run on the tensor cores (TF32 x 3 split,
    # tiles 16, 32 or 64 states wide): faster than the SIMT kernels at every
    # measured K from 9 to 64
    prec = EPOCH_FP32_TC if w.K > 8 else EPOCH_FP32
    lik = EpochLikelihood(w, precision=prec, cuda_stream=stream.cuda_stream)
    nn = 2 * w.n_taxa - 1

    # ---- device-resident timing: K graph replays --------------------------
    clocks = ClockSampler(dev)
    clocks.start()
    for _ in range(args.warmup):
        binding.epoch_evaluate_async(lik.ctx, True)
    torch.cuda.synchronize()
    l0, _ = lik.counters()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        binding.epoch_evaluate_async(lik.ctx, True)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    clk = clocks.stop()
    l1, _ = lik.counters()
    launches = l1 - l0
    lnl32, g32 = binding.epoch_read_results(lik.ctx, nn, w.n_epochs, lik.n_params, True)
    ms_step = ms / args.steps

    # ---- the partials pass alone (dominant kernel), same stream ------------
    for _ in range(3):
        binding.epoch_update_partials(lik.ctx)
    torch.cuda.synchronize()
    reps = max(args.steps, 10)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        binding.epoch_update_partials(lik.ctx)
    e1.record(stream)
    torch.cuda.synchronize()
    part_ms = e0.elapsed_time(e1) / reps
    pbytes = partials_bytes(w)

    # ---- the gradient pass alone (pre-order adjoint, G, chain rule) --------
    # epoch_gradient after the partials of the same inputs; its enqueued
    # kernels sit between the events (it reads the gradient back at the end)
    gr = max(5, min(args.steps, 50))
    grad_ms = 0.0
    for _ in range(gr + 2):
        binding.epoch_update_partials(lik.ctx)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        binding.epoch_gradient(lik.ctx, nn, w.n_epochs, lik.n_params)
        g1.record(stream)
        torch.cuda.synchronize()
        if _ >= 2:
            grad_ms += g0.elapsed_time(g1) / gr
    abytes = adjoint_bytes(w)
    achieved = pbytes / (part_ms * 1e-3) / 1e9
    peak, peak_kind = hbm_peak()

    # ---- e2e through the C ABI from host arrays ----------------------------
    # An inference loop changes the model parameters and node heights between
    # evaluations; the alignment is uploaded once.  Every step uploads all of
    # them (from pinned host memory), evaluates, and reads back lnL and the
    # whole gradient.  A second loop also re-uploads the alignment each step.
    def pinned(a, dtype=np.float64):
        t = torch.empty(np.asarray(a).shape, dtype=torch.float64 if dtype == np.float64
                        else torch.int32, pin_memory=True)
        v = t.numpy()
        v[...] = a
        return t, v
    keep = []
    host = {}
    for name, arr in (("Q", w.Q), ("dQ", w.dQ), ("pi", w.pi), ("b", w.boundaries),
                      ("cr", w.cat_rates), ("cw", w.cat_weights), ("h", w.heights),
                      ("pw", w.pattern_weights)):
        t, v = pinned(arr)
        keep.append(t)
        host[name] = v
    tt, tips = pinned(np.asarray(w.tips, dtype=np.int32), np.int32)
    keep.append(tt)
    for _ in range(2):
        lik.load(w)
        binding.epoch_evaluate_async(lik.ctx, True)
        binding.epoch_read_results(lik.ctx, nn, w.n_epochs, lik.n_params, True)
    torch.cuda.synchronize()
    e_steps = max(5, min(args.steps, 50))

    def e2e_loop(with_alignment):
        t0 = time.perf_counter()
        for _ in range(e_steps):
            binding.epoch_set_rate_matrices(lik.ctx, host["Q"], host["pi"], 1, 1)
            binding.epoch_set_rate_derivatives(lik.ctx, host["dQ"])
            binding.epoch_set_boundaries(lik.ctx, host["b"])
            binding.epoch_set_categories(lik.ctx, host["cr"], host["cw"])
            binding.epoch_set_heights(lik.ctx, host["h"])
            if with_alignment:
                binding.epoch_set_tip_data(lik.ctx, tips, host["pw"])
            binding.epoch_evaluate_async(lik.ctx, True)
            binding.epoch_read_results(lik.ctx, nn, w.n_epochs, lik.n_params, True)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / e_steps

    e2e_s = max_over_ranks(e2e_loop(False), world)
    e2e_aln_s = max_over_ranks(e2e_loop(True), world)
    h2d = (host["Q"].nbytes + host["dQ"].nbytes + host["pi"].nbytes + host["b"].nbytes
           + host["cr"].nbytes + host["cw"].nbytes + host["h"].nbytes)
    h2d_aln = h2d + w.n_taxa * w.n_patterns + host["pw"].nbytes
    d2h = 8 + 8 * (2 * nn + w.n_epochs - 1 + lik.n_params)

    # ---- plain FP64 GPU path on the same workload --------------------------
    lik64 = EpochLikelihood(w, precision=EPOCH_FP64, cuda_stream=stream.cuda_stream)
    for _ in range(2):
        binding.epoch_evaluate_async(lik64.ctx, True)
    torch.cuda.synchronize()
    f_steps = max(3, min(args.steps, 10))
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(f_steps):
        binding.epoch_evaluate_async(lik64.ctx, True)
    f1.record(stream)
    torch.cuda.synchronize()
    fp64_ms = f0.elapsed_time(f1) / f_steps
    lnl64, g64 = binding.epoch_read_results(lik64.ctx, nn, w.n_epochs, lik64.n_params, True)
    lik64.close()
    lik.close()
    forest = run_forest(args, stream) if not args.no_forest else None
    rel_err = abs(lnl32 - lnl64) / abs(lnl64)
    grad_err = float(np.abs(g32["heights"] - g64["heights"]).max() / np.abs(g64["heights"]).max())

    out = {
        "metric": METRIC,
        "value": job_rate(1.0, ms_step * 1e-3, world),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == EPOCH_FP32 else "f32 (tf32x3 tensor-core contractions)",
        "data": "synthetic (seeded coalescent tree, simulated alignment)",
        "config": {**cfg, "parallelism": f"replicas{world}", "l2": l2_note(w)},
        "e2e": {"value": job_rate(1.0, e2e_s, world), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "per_step_inputs": "Q, dQ, pi, boundaries, categories, node heights (pinned); "
                                   "alignment uploaded once",
                "with_alignment_each_step": {"value": job_rate(1.0, e2e_aln_s, world), "unit": UNIT,
                                             "h2d_bytes_per_step": int(h2d_aln)}},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": measured_traffic(args.workload),
                     "peak_source": peak_kind,
                     "kernel": "partials pass (post-order pruning + rescaling + root)",
                     "effective_gbs_all_nodes_stored": survey_bytes(w) / (part_ms * 1e-3) / 1e9,
                     "ms_per_launch": part_ms, "algorithmic_bytes": int(pbytes)},
        "roofline_gradient_pass": {
            "bound": "hbm", "achieved": abytes / (grad_ms * 1e-3) / 1e9, "peak": peak,
            "unit": "GB/s", "frac": abytes / (grad_ms * 1e-3) / 1e9 / peak,
            "peak_source": peak_kind, "ms_per_launch": grad_ms, "algorithmic_bytes": int(abytes),
            "kernel": "gradient pass (pre-order adjoint + G + chain rule; includes the "
                      "read-back of the gradient)"},
        "fp64_gpu": {"value": 1e3 / fp64_ms, "unit": UNIT, "ms_per_step": fp64_ms,
                     "lnL_rel_err_fp32_vs_fp64": rel_err, "grad_rel_err_fp32_vs_fp64": grad_err,
                     "speedup": fp64_ms / ms_step},
        "lnL": lnl32,
        "clocks": clk,
    }
    if forest:
        out["forest"] = forest
    return out


def run_forest(args, stream):
    """The batched trait workload: 256 coalescent trees (50-1000 taxa, 1-8
    epochs, K = 50 asymmetric rates, 1-4 patterns) in one persistent launch
    replayed from a CUDA graph (epoch_batch_*)."""
    import torch

    import synth
    from paper_1309_3075_b300.binding import EpochBatch

    bw = synth.asym50_forest()
    fb = EpochBatch(bw.trees, cuda_stream=stream.cuda_stream)
    try:
        for _ in range(max(3, args.warmup)):  # the first call tunes the launch shape
            fb.evaluate()
        reps = max(10, min(args.steps, 50))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        from paper_1309_3075_b300 import binding
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            binding.epoch_batch_evaluate_async(fb.b)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        lnl = fb.evaluate()
        warps, ctas = fb.launch_shape()
    finally:
        fb.close()
    n_tax = sum(t.n_taxa for t in bw.trees)
    return {"workload": f"{len(bw.trees)} trees, {n_tax} taxa in all, K=50 asymmetric, "
                        "1-8 epochs, 1-4 patterns, one launch per evaluation",
            "batch_evals_per_s": 1e3 / ms, "tree_evals_per_s": len(bw.trees) * 1e3 / ms,
            "ms_per_batch": ms, "launch_shape": {"warps_per_cta": warps, "ctas_per_sm": ctas},
            "lnL_sum": float(np.sum(lnl))}


def oracle_sample_rate(w, budget_s):
    """Oracle lnL + gradient on pattern slices of the workload; returns
    (evals/s scaled to the full workload, description, cores)."""
    import oracle

    P = w.n_patterns
    sl = min(P, 1000)
    sub = w.slice_patterns(0, sl)
    oracle.build()
    n = 0
    t0 = time.perf_counter()
    while True:
        oracle.gradient(sub)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    per_full = dt / n * (P / sl)
    return 1.0 / per_full, f"{n} lnL+gradient evaluations on the first {sl} of {P} patterns " \
                           f"(oracle, single thread), scaled by {P}/{sl}", 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gtr", choices=["gtr", "gy94", "seasonal", "aa"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-forest", action="store_true",
                    help="skip the batched 256-tree measurement")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    w, cfg = make_workload(args.workload)

    if args.impl == "reference":
        if rank != 0:
            return
        rate, sample, cores = oracle_sample_rate(w, args.cpu_seconds * max(args.steps, 1) / 50)
        out = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": 0,
               "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {**cfg, "parallelism": "cpu"},
               "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": sample},
               "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    out = run_ours(args, w, cfg, rank, world)
    if rank == 0:
        rate, sample, cores = oracle_sample_rate(w, args.cpu_seconds)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": sample}
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
