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

PATH_NAMES = {1: "EPOCH_FP32", 2: "EPOCH_FP32_TC", 4: "EPOCH_FP32_TC_BF16"}
DTYPES = {1: "f32", 2: "f32 (tf32x3 tensor-core contractions)",
          4: "f32 (bf16x3 tensor-core contractions)"}
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
# clocks sampled during the timed regions (read-only NVML queries)
# ---------------------------------------------------------------------------
class _Nvml:
    """The few read-only NVML queries the sampler needs, through ctypes on the
    driver's libnvidia-ml (no Python NVML package needed)."""

    CLOCK_SM = 1
    # clock-event reason bits (nvml.h)
    REASONS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
               "hw_thermal_slowdown": 0x40}

    def __init__(self):
        import ctypes
        self.C = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        rc = self.lib.nvmlInit_v2()
        if rc != 0:
            raise RuntimeError(f"nvmlInit_v2 returned {rc}")

    def handle(self, bus=None, index=0):
        h = self.C.c_void_p()
        rc = 1
        if bus:
            rc = self.lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), self.C.byref(h))
        if rc != 0:
            rc = self.lib.nvmlDeviceGetHandleByIndex_v2(self.C.c_uint(index), self.C.byref(h))
        if rc != 0:
            raise RuntimeError(f"no NVML handle ({rc})")
        return h

    def sm_clock(self, h):
        v = self.C.c_uint()
        rc = self.lib.nvmlDeviceGetClockInfo(h, self.CLOCK_SM, self.C.byref(v))
        return float(v.value) if rc == 0 else None

    def sm_max_clock(self, h):
        v = self.C.c_uint()
        rc = self.lib.nvmlDeviceGetMaxClockInfo(h, self.CLOCK_SM, self.C.byref(v))
        return float(v.value) if rc == 0 else None

    def reasons(self, h):
        v = self.C.c_ulonglong()
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        return int(v.value) if fn(h, self.C.byref(v)) == 0 else 0

    def close(self):
        self.lib.nvmlShutdown()


class ClockSampler:
    """Polls the SM clock and the clock-event reasons of one GPU through NVML
    from a host thread (about one sample per millisecond), with host
    timestamps, so that samples can be matched to timed regions as short as a
    few milliseconds.  Only reads: no clock or other setting is changed."""

    def __init__(self, device=0):
        self.device = device
        self.samples = []          # (t, sm_mhz, reasons bit mask)
        self.windows = {}          # name -> [(t0, t1)]
        self.sm_max = None
        self._stop = threading.Event()
        self._paused = threading.Event()  # set: no polling (host-bound sections)
        self._thread = None
        self._nv = None
        self.error = None

    def start(self):
        try:
            nv = _Nvml()
            bus = None
            try:
                import torch
                pr = torch.cuda.get_device_properties(self.device)
                bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
            except Exception:
                pass
            h = nv.handle(bus, self.device)
            self.sm_max = nv.sm_max_clock(h)
            self._nv = nv
        except Exception as e:  # no NVML: the line says so
            self.error = repr(e)[:200]
            return self

        def run():
            while not self._stop.is_set():
                if self._paused.is_set():
                    time.sleep(0.005)
                    continue
                mhz = nv.sm_clock(h)
                if mhz is not None:
                    self.samples.append((time.perf_counter(), mhz, nv.reasons(h)))
                time.sleep(0.001)

        self._thread = threading.Thread(target=run, daemon=True)
        self._thread.start()
        t0 = time.time()
        while not self.samples and time.time() - t0 < 2.0:
            time.sleep(0.005)
        return self

    def pause(self):
        self._paused.set()

    def resume(self):
        self._paused.clear()

    def window(self, name, t0, t1):
        self.windows.setdefault(name, []).append((t0, t1))

    def stop(self):
        self._stop.set()
        if self._thread:
            self._thread.join(timeout=2.0)
        if self._nv:
            try:
                self._nv.close()
            except Exception:
                pass

    def summary(self, names):
        """Median SM clock and the reasons seen over the samples inside the
        named windows."""
        if self._nv is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0,
                    "error": self.error}
        spans = [w for n in names for w in self.windows.get(n, [])]
        inside = [smp for smp in self.samples if any(a <= smp[0] <= b for a, b in spans)]
        sm = [x[1] for x in inside]
        reasons = sorted({k for _, _, r in inside for k, f in _Nvml.REASONS.items() if r & f})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": self.sm_max,
                "reasons": reasons, "samples": len(sm), "windows": list(names),
                "source": "NVML (libnvidia-ml), about 1 ms period"}


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
                    "sha1": "bcf7f4e922551e9f72bdd7c21de636fe88fc997c", "bytes": 201416960}


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


def timed_replays(stream, fn, reps):
    """ms per call of fn() over reps calls, CUDA events on the launching
    stream, synchronized on both sides; also the host span for the clock
    windows."""
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, (t0, time.perf_counter())


def run_ours(args, w, cfg, rank, world):
    import torch

    from paper_1309_3075_b300 import binding
    from paper_1309_3075_b300.binding import (EPOCH_FP32, EPOCH_FP32_AUTO, EPOCH_FP32_TC,
                                              EPOCH_FP32_TC_BF16, EpochLikelihood)

    dev = rank % max(torch.cuda.device_count(), 1)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    # K = 4 has its own FP32 path; other K take whichever FP32 path (SIMT or
    # tensor-core tile products) the library's probe measures faster, unless
    # --precision names one
    chosen = {"simt": EPOCH_FP32, "tf32x3": EPOCH_FP32_TC, "bf16x3": EPOCH_FP32_TC_BF16}
    want = chosen.get(args.precision, EPOCH_FP32 if w.K == 4 else EPOCH_FP32_AUTO)
    lik = EpochLikelihood(w, precision=want, cuda_stream=stream.cuda_stream)
    prec, probe_simt, probe_tc, probe_bf = binding.epoch_path_info(lik.ctx)
    nn = 2 * w.n_taxa - 1
    clocks = ClockSampler(dev).start()

    # ---- device-resident timing: K graph replays --------------------------
    for _ in range(args.warmup):
        binding.epoch_evaluate_async(lik.ctx, True)
    torch.cuda.synchronize()
    l0, _ = lik.counters()
    if world > 1:
        torch.distributed.barrier()
    ms_raw, span = timed_replays(stream, lambda: binding.epoch_evaluate_async(lik.ctx, True),
                                 args.steps)
    clocks.window("step", *span)
    ms = max_over_ranks(ms_raw * args.steps, world)
    l1, _ = lik.counters()
    launches = l1 - l0
    lnl32, g32 = binding.epoch_read_results(lik.ctx, nn, w.n_epochs, lik.n_params, True)
    ms_step = ms / args.steps

    # ---- the partials pass alone (dominant kernel of the forward), same stream
    for _ in range(3):
        binding.epoch_update_partials(lik.ctx)
    part_ms, span = timed_replays(stream, lambda: binding.epoch_update_partials(lik.ctx),
                                  max(args.steps, 10))
    clocks.window("passes", *span)
    pbytes = partials_bytes(w)

    # ---- the gradient pass alone (pre-order adjoint, G, chain rule) --------
    # epoch_gradient after the partials of the same inputs; its enqueued
    # kernels sit between the events (it reads the gradient back at the end)
    gr = max(5, min(args.steps, 50))
    grad_ms = 0.0
    t0 = time.perf_counter()
    for i in range(gr + 2):
        binding.epoch_update_partials(lik.ctx)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        binding.epoch_gradient(lik.ctx, nn, w.n_epochs, lik.n_params)
        g1.record(stream)
        torch.cuda.synchronize()
        if i >= 2:
            grad_ms += g0.elapsed_time(g1) / gr
    clocks.window("passes", t0, time.perf_counter())
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
    # host-bound loops of ~0.5 ms steps: 100 steps each, the three variants
    # alternated three times, the median kept
    e_steps = 100

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
        t1 = time.perf_counter()
        return (t1 - t0) / e_steps

    # the same step as one call (epoch_evaluate_step): inputs from the pinned
    # host arrays, outputs into pinned host arrays, no copies in Python
    outs = {}
    for name, n in (("heights", nn), ("boundaries", max(w.n_epochs - 1, 1)),
                    ("params", max(lik.n_params, 1)), ("branch_rates", nn)):
        t, v = pinned(np.zeros(n))
        keep.append(t)
        outs[name] = v

    step = binding.epoch_step_function(lik.ctx, host["Q"], host["pi"], host["dQ"], host["b"],
                                       host["cr"], host["cw"], host["h"], True, outs)

    def e2e_one_call():
        t0 = time.perf_counter()
        for _ in range(e_steps):
            step()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        return (t1 - t0) / e_steps

    # the e2e loops are bound by host work: the clock poller (a Python thread)
    # is paused so that it does not compete with them for the interpreter
    clocks.pause()
    e2e_one_call()  # warm
    runs = {"one": [], "sep": [], "aln": []}
    for _ in range(3):
        runs["one"].append(e2e_one_call())
        runs["sep"].append(e2e_loop(False))
        runs["aln"].append(e2e_loop(True))
    clocks.resume()
    e2e_step_s = max_over_ranks(float(np.median(runs["one"])), world)
    e2e_s = max_over_ranks(float(np.median(runs["sep"])), world)
    e2e_aln_s = max_over_ranks(float(np.median(runs["aln"])), world)
    h2d = (host["Q"].nbytes + host["dQ"].nbytes + host["pi"].nbytes + host["b"].nbytes
           + host["cr"].nbytes + host["cw"].nbytes + host["h"].nbytes)
    h2d_aln = h2d + w.n_taxa * w.n_patterns + host["pw"].nbytes
    d2h = 8 + 8 * (2 * nn + w.n_epochs - 1 + lik.n_params)

    # ---- plain FP64 GPU path on the same workload --------------------------
    fp64_ms, lnl64, g64 = time_fp64(w, stream, args, clocks)
    lik.close()
    rel_err = abs(lnl32 - lnl64) / abs(lnl64)
    grad_err = float(np.abs(g32["heights"] - g64["heights"]).max() / np.abs(g64["heights"]).max())

    forest = run_forest(args, stream, clocks) if not args.no_forest else None
    codon = run_codon(args, stream, clocks) if (args.workload == "gtr" and not args.no_codon) else None
    clocks.stop()
    clk = clocks.summary(["step"])
    if clk["samples"] < 3:  # a short timed region: all timed GPU sections
        clk = clocks.summary(["step", "passes", "fp64", "forest", "codon"])
    norm = None
    if clk.get("sm_mhz") and clk.get("sm_max_mhz"):
        norm = {"ms_per_step_x_sm_mhz": ms_step * clk["sm_mhz"],
                "ms_per_step_at_max_clock": ms_step * clk["sm_mhz"] / clk["sm_max_mhz"]}

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
        "dtype": DTYPES.get(prec, "f32"),
        "data": "synthetic (seeded coalescent tree, simulated alignment)",
        "config": {**cfg, "parallelism": f"replicas{world}", "l2": l2_note(w)},
        "e2e": {"value": job_rate(1.0, e2e_step_s, world), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "api": "epoch_evaluate_step (one call per step, bound to the pinned buffers "
                       "with epoch_step_function)",
                "steps": e_steps, "repeats": "median of 3",
                "per_step_inputs": "Q, dQ, pi, boundaries, categories, node heights (pinned); "
                                   "alignment uploaded once",
                "separate_calls": {"value": job_rate(1.0, e2e_s, world), "unit": UNIT,
                                   "api": "five setters, epoch_evaluate_async, "
                                          "epoch_read_results"},
                "with_alignment_each_step": {"value": job_rate(1.0, e2e_aln_s, world), "unit": UNIT,
                                             "h2d_bytes_per_step": int(h2d_aln),
                                             "api": "separate calls"}},
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
        "path": {"precision_in_use": PATH_NAMES.get(prec, str(prec)),
                 "probe_ms_simt": probe_simt, "probe_ms_tc_tf32x3": probe_tc,
                 "probe_ms_tc_bf16x3": probe_bf},
        "clocks": clk,
    }
    if norm:
        out["clock_normalised"] = norm
    if forest:
        out["forest"] = forest
    if codon:
        out["gy94"] = codon
    return out


def time_fp64(w, stream, args, clocks):
    """The plain FP64 GPU path (EPOCH_FP64) on the same workload: ms per
    lnL + gradient evaluation (graph replays), lnL and gradient."""
    from paper_1309_3075_b300 import binding
    from paper_1309_3075_b300.binding import EPOCH_FP64, EpochLikelihood

    nn = 2 * w.n_taxa - 1
    lik64 = EpochLikelihood(w, precision=EPOCH_FP64, cuda_stream=stream.cuda_stream)
    try:
        for _ in range(2):
            binding.epoch_evaluate_async(lik64.ctx, True)
        ms, span = timed_replays(stream, lambda: binding.epoch_evaluate_async(lik64.ctx, True),
                                 max(3, min(args.steps, 10)))
        clocks.window("fp64", *span)
        lnl64, g64 = binding.epoch_read_results(lik64.ctx, nn, w.n_epochs, lik64.n_params, True)
    finally:
        lik64.close()
    return ms, lnl64, g64


# Tensor-pipe activity of the codon path's tcgen05 kernels, from one ncu
# capture (sm__pipe_tensor_cycles_active over elapsed cycles, cycle-weighted
# over the captured k_tc_* launches).  Reported only while the kernel source
# is the one that was measured.
# time-weighted sm__pipe_tensor_cycles_active of the BF16 x 3 tile-product
# launches of one codon evaluation (ncu hardware counters), valid while the
# tensor-core source is the one it was measured on
CODON_TENSOR = {"source": "paper_1309_3075_b300/csrc/k_tc.cu",
                "sha1": "64aeb387c566d565e01d2f1d4ab0ce96eccf18d2", "frac": 0.063,
                "arm": "EPOCH_FP32_TC_BF16", "profile": "profiles/tc_codon_gy94.md"}


def codon_tensor_frac():
    import hashlib
    if not CODON_TENSOR["sha1"]:
        return None
    try:
        with open(os.path.join(ROOT, CODON_TENSOR["source"]), "rb") as f:
            digest = hashlib.sha1(f.read()).hexdigest()
    except OSError:
        return None
    return CODON_TENSOR["frac"] if digest == CODON_TENSOR["sha1"] else None


def run_codon(args, stream, clocks):
    """The codon workload (GY94, K = 61, 4 epochs, 128 taxa, 5,000 codon
    sites, 4 categories): lnL + gradient on the tensor-core path (TF32x3
    tile products) against the plain FP64 GPU path."""
    from paper_1309_3075_b300 import binding
    from paper_1309_3075_b300.binding import (EPOCH_FP32, EPOCH_FP32_AUTO, EPOCH_FP32_TC,
                                              EPOCH_FP32_TC_BF16, EpochLikelihood)

    w, cfg = make_workload("gy94")
    nn = 2 * w.n_taxa - 1
    lik = EpochLikelihood(w, precision=EPOCH_FP32_AUTO, cuda_stream=stream.cuda_stream)
    prec, probe_simt, probe_tc, probe_bf = binding.epoch_path_info(lik.ctx)
    try:
        for _ in range(3):
            binding.epoch_evaluate_async(lik.ctx, True)
        ms, span = timed_replays(stream, lambda: binding.epoch_evaluate_async(lik.ctx, True),
                                 max(10, min(args.steps, 50)))
        clocks.window("codon", *span)
        lnl, g = binding.epoch_read_results(lik.ctx, nn, w.n_epochs, lik.n_params, True)
    finally:
        lik.close()
    fp64_ms, lnl64, g64 = time_fp64(w, stream, args, clocks)
    flops = codon_flops(w)
    # every FP32 arm on the same workload: SIMT contractions, TF32 x 3 and
    # BF16 x 3 tile products (lnL + gradient, graph replays)
    arms = {}
    for name, p in (("EPOCH_FP32", EPOCH_FP32), ("EPOCH_FP32_TC", EPOCH_FP32_TC),
                    ("EPOCH_FP32_TC_BF16", EPOCH_FP32_TC_BF16)):
        la = EpochLikelihood(w, precision=p, cuda_stream=stream.cuda_stream)
        try:
            for _ in range(2):
                binding.epoch_evaluate_async(la.ctx, True)
            ams, span = timed_replays(stream, lambda: binding.epoch_evaluate_async(la.ctx, True),
                                      max(3, min(args.steps, 10)))
            clocks.window("codon", *span)
            lnl_a, g_a = binding.epoch_read_results(la.ctx, nn, w.n_epochs, la.n_params, True)
        finally:
            la.close()
        arms[name] = {"ms_per_step": ams, "tile_product_tflops": flops / (ams * 1e-3) / 1e12
                      if p != EPOCH_FP32 else None,
                      "lnL_rel_err_vs_fp64": abs(lnl_a - lnl64) / abs(lnl64),
                      "grad_rel_err_vs_fp64": float(np.abs(g_a["params"] - g64["params"]).max()
                                                    / np.abs(g64["params"]).max())}
    return {"workload": cfg["workload"], "patterns": cfg["patterns"], "evals_per_s": 1e3 / ms,
            "ms_per_step": ms,
            "dtype": DTYPES.get(prec, "f32"),
            "path": {"precision_in_use": PATH_NAMES.get(prec, str(prec)),
                     "probe_ms_simt": probe_simt, "probe_ms_tc_tf32x3": probe_tc,
                     "probe_ms_tc_bf16x3": probe_bf},
            "fp64_gpu_ms_per_step": fp64_ms, "speedup_vs_fp64": fp64_ms / ms,
            "lnL_rel_err_vs_fp64": abs(lnl - lnl64) / abs(lnl64),
            "grad_rel_err_vs_fp64": float(np.abs(g["params"] - g64["params"]).max()
                                          / np.abs(g64["params"]).max()),
            "tile_product_tflops": flops / (ms * 1e-3) / 1e12,
            "arms": arms,
            "tensor_pipe_active_frac": codon_tensor_frac(),
            "tensor_pipe_arm": CODON_TENSOR["arm"],
            "tensor_profile": CODON_TENSOR["profile"]}


def codon_flops(w):
    """Useful FLOPs of the tensor-core tile products of one lnL + gradient
    evaluation at K states (unpadded): for every internal non-root node v,
    S_v = P_v L_v in pruning, S_v again and U_v = P_v^T X_v in the adjoint,
    2 K^2 per (category, pattern) each.  Tips take table rows instead."""
    K, C, P, N = w.K, w.n_categories, w.n_patterns, w.n_taxa
    stored = N - 2
    return 2.0 * K * K * C * P * 3 * stored


def forest_flops(bw):
    """Useful FP32 FLOPs of one evaluation of the batched trees: every
    uniformisation term is a K x K matrix applied to the tree's P_t pattern
    vectors (2 K^2 P_t), with the kernel's own truncation (Poisson tail below
    1e-9, pieces of mu dt <= 30) counted term by term on the host."""
    total = 0.0
    for w in bw.trees:
        K, P = w.K, w.n_patterns
        mus = []
        for e in range(w.n_epochs):
            q = np.asarray(w.Q)[np.asarray(w.epoch_to_matrix)[e]]
            c = -(np.asarray(w.pi) * np.diag(q)).sum() if getattr(w, "normalise", 1) else 1.0
            c = c if c > 0 else 1.0
            mus.append(np.max(-np.diag(q)) / c)
        mus = np.array(mus)
        parent = np.asarray(w.parent)
        h = np.asarray(w.heights)
        v = np.where(parent >= 0)[0]
        lo, hi = h[v], h[parent[v]]
        edges = np.r_[-np.inf, np.asarray(w.boundaries), np.inf]
        seg = np.clip(np.minimum(hi[:, None], edges[None, 1:])
                      - np.maximum(lo[:, None], edges[None, :-1]), 0.0, None)
        mt = (seg * mus[None, :]).ravel()
        mt = mt[mt > 0]
        pieces = np.where(mt > 30.0, np.ceil(mt / 30.0), 1.0)
        mp = mt / pieces
        wgt = np.exp(-mp)
        terms = np.zeros_like(mp)
        live = np.ones(mp.shape, bool)
        m = 0
        while live.any() and m < 4096:
            r = (m + 1) - mp
            done = live & (r > 0) & (wgt * (m + 1) <= 1e-9 * r)
            live &= ~done
            m += 1
            terms[live] += 1
            wgt = wgt * mp / m
        total += float((terms * pieces).sum()) * 2.0 * K * K * P
    return total


def fp32_simt_peak(sm_mhz):
    """FP32 FMA peak of the part: 148 SMs x 128 FP32 lanes x 2 FLOP per clock."""
    return 148 * 128 * 2 * sm_mhz * 1e6 / 1e12


def run_forest(args, stream, clocks):
    """The batched trait workload: 256 coalescent trees (50-1000 taxa, 1-8
    epochs, K = 50 asymmetric rates, 1-4 patterns) in one persistent launch
    replayed from a CUDA graph (epoch_batch_*).  Its partials (about 67 MB)
    fit in L2, so it is bound by the FP32 uniformisation arithmetic, reported
    against the FP32 FMA peak at the sampled SM clock."""
    import synth
    from paper_1309_3075_b300 import binding
    from paper_1309_3075_b300.binding import EpochBatch

    bw = synth.asym50_forest()
    fb = EpochBatch(bw.trees, cuda_stream=stream.cuda_stream)
    try:
        for _ in range(max(3, args.warmup)):  # the first call tunes the launch shape
            fb.evaluate()
        ms, span = timed_replays(stream, lambda: binding.epoch_batch_evaluate_async(fb.b),
                                 max(10, min(args.steps, 50)))
        clocks.window("forest", *span)
        lnl = fb.evaluate()
        warps, ctas = fb.launch_shape()
        # lnL + gradient (heights, boundaries) of every tree in one launch
        for _ in range(3):  # the first call tunes this launch's shape
            fb.evaluate_gradient()
        gms, span = timed_replays(stream, lambda: binding.epoch_batch_evaluate_gradient_async(fb.b),
                                  max(10, min(args.steps, 50)))
        clocks.window("forest", *span)
    finally:
        fb.close()
    n_tax = sum(t.n_taxa for t in bw.trees)
    flops = forest_flops(bw)
    clk = clocks.summary(["forest"]).get("sm_mhz") or clocks.sm_max or 2032.0
    peak = fp32_simt_peak(clk)
    achieved = flops / (ms * 1e-3) / 1e12
    return {"workload": f"{len(bw.trees)} trees, {n_tax} taxa in all, K=50 asymmetric, "
                        "1-8 epochs, 1-4 patterns, one launch per evaluation",
            "batch_evals_per_s": 1e3 / ms, "tree_evals_per_s": len(bw.trees) * 1e3 / ms,
            "ms_per_batch": ms, "launch_shape": {"warps_per_cta": warps, "ctas_per_sm": ctas},
            "with_gradient": {"ms_per_batch": gms, "batch_evals_per_s": 1e3 / gms,
                              "tree_evals_per_s": len(bw.trees) * 1e3 / gms,
                              "outputs": "lnL, d lnL/d heights and d lnL/d boundaries per tree"},
            "lnL_sum": float(np.sum(lnl)),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "peak_source": f"derived: 148 SMs x 128 FP32 lanes x 2 FLOP x {clk:.0f} MHz",
                         "algorithmic_flops": flops,
                         "kernel": "k_forest (uniformisation terms, K x K matrix on the "
                                   "pattern vectors)"}}


def _oracle_slice(w):
    """One oracle lnL + gradient on a pattern slice (a process-pool worker)."""
    import oracle

    return oracle.gradient(w)["lnL"]


def oracle_rates(w, budget_s, cores=None):
    """The FP64 CPU oracle, as it stands, on the host cores.

    * all cores: the full workload's patterns split into one slice per core,
      each an independent oracle lnL + gradient in a spawned worker process
      (patterns are independent, so lnL and the gradient are the sums over
      slices); one evaluation of the whole workload per round;
    * one core: the oracle on the first 1,000 patterns in this process,
      scaled to the full pattern count.
    Returns {"multi": (rate, description, cores), "single": (rate,
    description)}; rates in evaluations of the full workload per second."""
    import multiprocessing as mp

    import oracle

    oracle.build()
    P = w.n_patterns
    cores = cores or len(os.sched_getaffinity(0))
    cuts = np.linspace(0, P, cores + 1).astype(int)
    slices = [w.slice_patterns(int(a), int(b)) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
    with mp.get_context("spawn").Pool(len(slices)) as pool:
        pool.map(_oracle_slice, slices)  # workers load the oracle
        n = 0
        t0 = time.perf_counter()
        while True:
            pool.map(_oracle_slice, slices)
            n += 1
            if time.perf_counter() - t0 > budget_s:
                break
        dt = (time.perf_counter() - t0) / n
    multi = (1.0 / dt, f"{n} lnL+gradient evaluations of all {P} patterns, split into "
                       f"{len(slices)} slices on {len(slices)} spawned worker processes",
             len(slices))
    sl = min(P, 1000)
    sub = w.slice_patterns(0, sl)
    m = 0
    t0 = time.perf_counter()
    while True:
        oracle.gradient(sub)
        m += 1
        if time.perf_counter() - t0 > budget_s:
            break
    per_full = (time.perf_counter() - t0) / m * (P / sl)
    single = (1.0 / per_full, f"{m} lnL+gradient evaluations on the first {sl} of {P} "
                              f"patterns (one thread), scaled by {P}/{sl}")
    return {"multi": multi, "single": single}


def cpu_baseline(w, budget_s):
    r = oracle_rates(w, budget_s)
    rate, sample, cores = r["multi"]
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "nproc": os.cpu_count(),
            "single_thread": {"value": r["single"][0], "unit": UNIT, "cores": 1,
                              "sample": r["single"][1]}}


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
    ap.add_argument("--no-codon", action="store_true",
                    help="skip the codon (GY94) measurement beside the default workload")
    ap.add_argument("--precision", default="auto", choices=["auto", "simt", "tf32x3", "bf16x3"],
                    help="FP32 arm of the timed workload (auto: the library's probe)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    w, cfg = make_workload(args.workload)

    if args.impl == "reference":
        if rank != 0:
            return
        # the oracle on all host cores; each timed step is one evaluation of
        # the whole workload, the run bounded to about a minute
        base = cpu_baseline(w, min(60.0, args.cpu_seconds * max(args.steps, 1) / 50))
        rate = base["value"]
        out = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": 0,
               "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {**cfg, "parallelism": "cpu"},
               "cpu_baseline": base,
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
        out["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
