#!/usr/bin/env python
"""Benchmark of the DPM scoring hot path (correlation, distance transform, shift-and-sum, threshold).

Workload (default): a 20-class bank of DPM-shaped class models (120 components: roots 5x11, 7x7, 11x5 and their
mirrors, 8 parts of 6x6 each; 1080 filters) on one 1280x720 image as a 45-level HOG-shaped pyramid (10 levels per
octave, sbin 8; 440,714 cells, uniform [0, 0.2)). A step is one whole pass of the path over that image: correlation
(decomposed per filter, split-BF16 tensor cores for the channel stage, FP32 passes), distance transform, assembly,
per-class thresholds and the copy of the detections to the host. The rank is found first: the cheapest of Sec. 5's
(S, T) root / part rank pairs on a ladder whose detections agree >= 99.5% with the full FP32 form (the metric's
condition); the line reports that agreement, the pair, the full FP32 form's images/s and the speed-up.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--form decomposed|full] [--precision bf16x3|bf16|fp8|fp32]
                  [--rank R | --ranks S,T] [--mode per_filter|joint]
  python bench.py --impl reference    # the FP64 CPU oracle on the same workload and metric
  python bench.py --workload c2|c4|c5 # the other configurations (one JSON line each, same keys):
      c2  one 500x375 image scored by one 6-component class model (54 filters), with rank sweeps, NMS, the
          convolution-shortening cascade and the HOG pyramid
      c4  the bank on a batch of 64 images, W ~ U{320..1280}, H ~ U{240..720}, one batch call per step
      c5  serving: Poisson arrivals (200 requests/s), sizes 640x480 / 1280x720 / 1920x1080, each request asking
          for 1..20 classes of the bank; p50/p99 latency from submission to results

Reported beside the headline: the full form in FP32 (the GPU baseline the decomposed form must beat) and in the
tensor-core precisions, the rank ladder, the per-stage device times and rooflines, detection parity with the FP64
oracle on the same factors for a bounded sample of components (`cpu_baseline`), and the end-to-end leg (`e2e`), which
copies each image's pyramid from pinned host memory on a copy stream, overlapping the previous image's scoring.

Under torchrun every rank scores its own replica of the image (images are independent: no data-path collective); the
barrier and the max-over-ranks timing use the process group.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1707_03268_gb300 import synth  # noqa: E402

METRIC = "images/sec and p50/p99 latency, decomposed BF16 vs full FP32, at >=99.5% agreement"
L2_BYTES = 129 * 1024 * 1024
AUTO_RANK_E = (0.25, 0.5, 1.0, 2.0, 4.0)  # the rank criterion's constant (Sec. 4 leaves it open)
RANK_SWEEP = {"per_filter": (4, 8, 16, 24, 32, 36), "joint": (16, 32, 64, 128, 256)}
PRECISIONS = {"fp32": 0, "bf16": 1, "fp8": 2, "bf16x3": 3}


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest x over the ranks (one all-reduce; x itself for one rank). The timed region's length is the slowest
    rank's, so whole-job rates divide by this."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: the units every rank processed (replicas: the same count on each) over the slowest
    rank's time."""
    return units_per_rank * world / (max_ms / 1e3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default: 20 at c3, 2000 at c2)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="tdpm", choices=["tdpm", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c2", "c3", "c4", "c5"])
    ap.add_argument("--form", default=None, choices=["decomposed", "full"])
    ap.add_argument("--precision", default=None, choices=sorted(PRECISIONS))
    ap.add_argument("--rank", type=int, default=None,
                    help="one CP rank for every filter (per_filter) or per shape group (joint); default: the rank "
                         "ladder (the cheapest root/part rank pair whose detections agree >= 99.5%% with full FP32)")
    ap.add_argument("--ranks", default=None, help="per_filter: root and part ranks S,T (Sec. 5's (S, T) pairs)")
    ap.add_argument("--mode", default=None, choices=["per_filter", "joint"])
    ap.add_argument("--als-iters", type=int, default=300, help="ALS cycles per decomposition")
    ap.add_argument("--variants", default=None,
                    help="c4: comma-separated subset of the variants to run, e.g. full_bf16,full_fp8")
    ap.add_argument("--serve-seconds", type=float, default=20.0, help="c5: length of the arrival stream")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="c5: mean arrival rate (requests/s)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fuse", action="store_true",
                    help="decomposed per-filter form: channel stage and separable passes as two launches")
    ap.add_argument("--no-compare", action="store_true", help="skip the full-form comparison runs")
    ap.add_argument("--no-sweep", action="store_true", help="skip the rank sweeps and the post-processing steps")
    args = ap.parse_args()
    # per-workload defaults: the per-filter decomposition in split BF16 (the precision that keeps >= 99.5% agreement)
    dflt = {"c2": ("decomposed", "bf16x3", None, "per_filter"), "c3": ("decomposed", "bf16x3", None, "per_filter"),
            "c4": ("decomposed", "bf16x3", None, "per_filter"), "c5": ("decomposed", "bf16x3", None, "per_filter")}
    for k, v in zip(("form", "precision", "rank", "mode"), dflt[args.workload]):
        if getattr(args, k) is None:
            setattr(args, k, v)
    if args.steps is None:
        args.steps = {"c2": 2000, "c3": 20, "c4": 5, "c5": 0}[args.workload]
    if args.mode == "joint" and args.rank is None:
        args.rank = 32
    return args


def load_taus(workload: str, n_comp: int) -> np.ndarray:
    """Per-component detection thresholds from tests/golden/thresholds.json (written from the FP64 oracle's full-form
    scores): one threshold for the one-class model (c2), one per class of six components for the bank (c3)."""
    with open(os.path.join(ROOT, "tests", "golden", "thresholds.json")) as f:
        g = json.load(f)
    if workload == "c2":
        return np.full(n_comp, float(g["c2"]["tau"]), dtype=np.float32)
    per = int(g["c3"]["components_per_class"])
    return np.repeat(np.asarray(g["c3"]["tau_per_class"], dtype=np.float32), per)[:n_comp]


def load_tau():
    with open(os.path.join(ROOT, "tests", "golden", "thresholds.json")) as f:
        return float(json.load(f)["c2"]["tau"])


# Sec. 5's (S, T) pairs: root rank S, part rank T; the ladder runs from the cheapest (the parts dominate the cost) and
# stops at the first pair whose detections agree >= 99.5% with the full FP32 form. S = 64 is the exact slice form of
# every root shape here (h*w <= 55).
RANK_LADDER = ((16, 16), (24, 24), (64, 24), (32, 32), (64, 32), (64, 36))
AGREEMENT_BAR = 0.995
DEFAULT_PAIR = (64, 32)  # the batch and serving workloads: the (S, T) pair the bank's ladder reaches the bar with


def filter_ranks(model, S: int, T: int) -> np.ndarray:
    """Per-filter ranks in model order (root, then parts, per component), capped at the exact rank h*w."""
    out = []
    for c in model.components:
        out.append(min(S, c.root.shape[0] * c.root.shape[1]))
        out.extend(min(T, p.filt.shape[0] * p.filt.shape[1]) for p in c.parts)
    return np.asarray(out, dtype=np.int32)


# ------------------------------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def pinned_records(torch, tdpm, n):
    """A host array of n detection records in page-locked memory (the read-back lands there directly, without page
    faults or a staging copy)."""
    raw = torch.empty(n * tdpm.DETECTION_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
    buf = raw.numpy().view(tdpm.DETECTION_DTYPE)
    _PINNED.append(raw)  # keeps the page-locked allocation alive with the view
    return buf


_PINNED = []


# ------------------------------------------------------------------------------------------------ roofline model
FUSED_SHAPES = {(6, 6), (5, 11), (7, 7), (11, 5)}  # filter shapes with a compiled fused decomposed kernel


def stage_bytes(wl, pyr, form: str, precision: str, rank: int, joint: bool, fused: bool = True):
    """Algorithmic DRAM bytes and flops per stage for one image: every input read once, every output written once.
    The fused decomposed kernel ("zsep_tc") reads the features and writes the filter maps; its flops are those of the
    separable passes and the recombination (FP32 ALU work; its channel-stage MMAs are a small tensor-core load)."""
    sizes = pyr.sizes
    lam = pyr.lam
    L = len(sizes)
    # rank: one rank for every filter (or the joint rank), or per-filter ranks in model order
    per_rank = None if np.isscalar(rank) or rank is None else [int(r) for r in rank]
    groups = {}
    fid = 0
    for comp in wl.model.components:
        for f in [comp.root] + [p.filt for p in comp.parts]:
            role = 0 if f is comp.root else 1
            r_f = per_rank[fid] if per_rank is not None else (rank or 0)
            groups.setdefault((role,) + f.shape[:2], []).append(min(r_f, f.shape[0] * f.shape[1]))
            fid += 1
    tc = precision in ("bf16", "bf16x3", "fp8")
    fb = {"fp32": 4, "bf16": 2, "bf16x3": 4, "fp8": 1}[precision]  # feature bytes per channel read by the correlation
    corr = "corr_tc" if tc else "corr_f32"
    zproj = "zproj_tc" if tc else "zproj_f32"
    out = {corr: [0, 0], zproj: [0, 0], "sep": [0, 0], "recomb_tc": [0, 0], "dt": [0, 0], "assemble": [0, 0],
           "to_bf16": [0, 0], "zsep_tc": [0, 0]}
    ub = 4 if precision == "bf16x3" else 2  # bytes per U_r value on the joint tensor-core path (hi + lo parts)
    if tc:
        out["to_fp8" if precision == "fp8" else "to_bf16"] = [sum(H * W * 32 * (4 + fb) for (H, W) in sizes), 0]
    for (role, h, w), fl in groups.items():
        K = len(fl)
        if joint:
            R = min(rank, h * w * 32)       # the joint form is exact from h*w*32 shared terms on
        else:
            R = sum(fl)                     # per filter: exact from h*w terms (the slices) on
        js = range(lam, L) if role == 0 else range(0, L - lam)
        for j in js:
            H, W = sizes[j]
            Ho, Wo = H - h + 1, W - w + 1
            if Ho <= 0 or Wo <= 0:
                continue
            # a per-filter group at its exact rank (every filter h*w terms) is scored by the full form's kernel
            if form == "full" or (not joint and min(fl) >= h * w):
                out[corr][0] += H * W * 32 * fb + K * Ho * Wo * 4
                out[corr][1] += 2 * h * w * 32 * K * Ho * Wo
            elif (fused and not joint and precision in ("bf16", "bf16x3") and (h, w) in FUSED_SHAPES
                  and max(fl) <= 64):
                out["zsep_tc"][0] += H * W * 32 * fb + K * Ho * Wo * 4
                out["zsep_tc"][1] += 2 * Ho * Wo * R * (h + w + 1)
            else:
                out[zproj][0] += H * W * 32 * fb + R * H * W * 4
                out[zproj][1] += 2 * 32 * R * H * W
                if joint and tc:
                    # separable passes write U_r; Lambda U runs on tensor cores
                    out["sep"][0] += R * H * W * 4 + R * Ho * Wo * ub
                    out["sep"][1] += 2 * R * Ho * Wo * (h + w)
                    out["recomb_tc"][0] += R * Ho * Wo * ub + K * Ho * Wo * 4
                    out["recomb_tc"][1] += 2 * K * R * Ho * Wo
                else:
                    out["sep"][0] += R * H * W * 4 + K * Ho * Wo * 4
                    terms = K * R if joint else R  # (filter, term) pairs
                    out["sep"][1] += 2 * Ho * Wo * terms * (h + w + 1)
    for comp in wl.model.components:
        h0, w0 = comp.root.shape[:2]
        for j in range(lam, L):
            l = j - lam
            H, W = sizes[j]
            Hp, Wp = sizes[l]
            Y, X = H - h0 + 1, W - w0 + 1
            for p in comp.parts:
                hp, wp = p.filt.shape[:2]
                Hs, Ws = Hp - hp + 1, Wp - wp + 1
                if Hs <= 0 or Ws <= 0:
                    Y = X = 0
                    break
                Y = min(Y, (Hs - 1 - p.anchor[0]) // 2 + 1)
                X = min(X, (Ws - 1 - p.anchor[1]) // 2 + 1)
            if Y <= 0 or X <= 0:
                continue
            n = len(comp.parts)
            for p in comp.parts:
                hp, wp = p.filt.shape[:2]
                Hs, Ws = Hp - hp + 1, Wp - wp + 1
                # fused passes: read the part map once, write values + argmax at the Y x X anchored positions (the
                # x-pass intermediate stays in shared memory)
                out["dt"][0] += Hs * Ws * 4 + Y * X * 8
            out["assemble"][0] += Y * X * 4 * (n + 2)
    return {k: {"bytes": v[0], "flops": v[1]} for k, v in out.items()}


def measured_traffic(workload: str, form: str, precision: str, mode: str, stage: str):
    """DRAM bytes per image of a stage from the committed ncu capture of the same configuration
    (profiles/roofline_traffic.json), or None when there is none or when a kernel source it was measured on has changed
    since (its SHA-256 no longer matches)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            table = json.load(f)
    except Exception:
        return None
    cfg = table.get("configs", {}).get(f"{workload}:{form}:{precision}:{mode}", {})
    e = cfg.get(stage)
    if not e:
        return None
    for path, sha in e.get("sources", {}).items():
        try:
            with open(os.path.join(ROOT, path), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != sha:
                    return None
        except OSError:
            return None
    return e.get("dram_bytes_per_image")


def sm_count() -> int:
    """Streaming multiprocessors of device 0, read from the device (152 on a GB300)."""
    import torch
    return int(torch.cuda.get_device_properties(0).multi_processor_count)


def fp32_alu_peak_tflops(sm_mhz: float, sms: int) -> float:
    """FP32 FMA roofline: SMs x 128 FP32 lanes x 2 flops per FMA x SM clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


TENSOR_STAGES = ("corr_tc", "zproj_tc", "recomb_tc")
ALU_STAGES = ("corr_f32", "zproj_f32", "sep", "zsep_tc")


def stage_roofline(name, ms_per_image, launches_per_image, model, peaks, sm_mhz):
    """Roofline of one stage: achieved algorithmic throughput against the peak of whichever resource binds it
    (the one whose peak would take longest for the stage's algorithmic bytes or flops)."""
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    src_hbm = "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"
    b, f = model[name]["bytes"], model[name]["flops"]
    s = ms_per_image / 1e3
    cand = [("hbm", b / (hbm * 1e9))]
    tp = float(peaks.get("bf16_tflops", 1900.0))
    if name in TENSOR_STAGES:
        cand.append(("tensor", f / (tp * 1e12)))
    elif name in ALU_STAGES:
        cand.append(("alu", f / (fp32_alu_peak_tflops(sm_mhz, sm_count()) * 1e12)))
    bound = max(cand, key=lambda c: c[1])[0]
    out = {"kernel": name, "bound": bound, "launches_per_image": launches_per_image, "ms_per_image": ms_per_image,
           "traffic": None, "algorithmic_bytes_per_image": b, "algorithmic_flops_per_image": f}
    if bound == "hbm":
        out.update(achieved=b / s / 1e9, peak=hbm, unit="GB/s", peak_source=src_hbm)
    elif bound == "tensor":
        out.update(achieved=f / s / 1e12, peak=tp, unit="TFLOP/s",
                   peak_source="MEASURED_PEAKS.json bf16_tflops burst (of measured)" if "bf16_tflops" in peaks
                   else "fallback 1900 TFLOP/s")
    else:
        sms = sm_count()
        pk = fp32_alu_peak_tflops(sm_mhz, sms)
        out.update(achieved=f / s / 1e12, peak=pk, unit="TFLOP/s",
                   peak_source=f"derived: {sms} SMs (read from the device) x 128 FP32 lanes x 2 flop x median SM "
                               f"clock under load ({sm_mhz:.0f} MHz)")
    out["frac"] = out["achieved"] / out["peak"]
    return out


# ------------------------------------------------------------------------------------------------ oracle legs
def workload_of(name: str):
    return {"c2": synth.config_c2, "c3": synth.config_c3, "c4": synth.config_c3, "c5": synth.config_c3}[name]()


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, same workload and metric (rank 0 of N only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as orc

    wl = workload_of(args.workload)
    pyr = wl.pyramids[0]
    n_comp = len(wl.model.components)
    taus = load_taus("c2" if args.workload == "c2" else "c3", n_comp)

    def one_step(i):
        # one component of the model over the whole pyramid: 1/n_comp of an image
        c = i % n_comp
        sub = synth.Model([wl.model.components[c]])
        orc.detect(orc.score_pyramid(sub, pyr), float(taus[c]))

    for i in range(args.warmup):
        one_step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        one_step(i)
    dt = time.perf_counter() - t0
    v = (args.steps / n_comp) / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "images/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "form": "full (FP64 oracle)", "levels": len(pyr.levels),
                       "components": n_comp, "filters": len(wl.model.filters())},
            "cpu_baseline": {"value": v, "unit": "images/s", "cores": orc.num_threads(), "kind": "oracle",
                             "sample": f"each step scores one of the {n_comp} components over the whole "
                                       f"{len(pyr.levels)}-level pyramid (1/{n_comp} of an image)"},
            "e2e": {"value": v, "unit": "images/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_oracle(wl, filters, gpu_dets, taus, budget_s: float = 15.0):
    """The FP64 oracle as it stands, on this host's cores: the model's components one after another over the whole
    pyramid (with the GPU run's filters, rebuilt from the library's FP64 factors for the decomposed form) until the
    time budget is spent. Rate = the share of an image scored / time. Its detections give the parity agreement of
    the GPU's detections of the same components."""
    from oracle import oracle as orc
    pyr = wl.pyramids[0]
    comps = wl.model.components
    fid0, starts = 0, []
    for c in comps:
        starts.append(fid0)
        fid0 += 1 + len(c.parts)
    n = 0
    ok = set()
    t0 = time.perf_counter()
    while n < len(comps):
        c = comps[n]
        sub = synth.Model([c])
        fs = None if filters is None else filters[starts[n]:starts[n] + 1 + len(c.parts)]
        for d in orc.detect(orc.score_pyramid(sub, pyr, filters=fs), float(taus[n])):
            ok.add((n,) + tuple(d[1:4]))
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    gk = set(k for k in gpu_dets if k[0] < n)
    return {"value": (n / len(comps)) / dt, "unit": "images/s", "cores": orc.num_threads(), "kind": "oracle",
            "sample": f"{n} of the {len(comps)} components over the whole {len(pyr.levels)}-level pyramid "
                      f"({n}/{len(comps)} of an image), FP64, the GPU run's filters",
            "parity_agreement_with_gpu": len(ok & gk) / max(1, len(ok | gk)), "oracle_detections": len(ok),
            "components_compared": n}


def factor_filters(tdpm, ctx, mid):
    """Filters rebuilt in FP64 from the library's exported factors, model order (for the oracle leg)."""
    from oracle import oracle as orc
    n_f, n_g = tdpm.tdpm_model_info(ctx, mid)
    out = [None] * n_f
    for g in range(n_g):
        info = tdpm.tdpm_group_info(ctx, mid, g)
        A, B, C, Lam = tdpm.tdpm_get_factors(ctx, mid, g)
        F = orc.joint_reconstruct(Lam, A, B, C)
        for k, fid in enumerate(info["filter_ids"]):
            out[fid] = F[k]
    return out


# ------------------------------------------------------------------------------------------------ class banks (c3, c4)
def _timed_steps(torch, step, steps, warmup, flush, stream):
    """Device time of each step (CUDA events on the launching stream), L2 flushed between steps outside the events."""
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    out = None
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        out = step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sorted(a.elapsed_time(b) for a, b in ev)
    return {"ms_sum": sum(ms), "p50": ms[len(ms) // 2], "p99": ms[min(len(ms) - 1, int(math.ceil(0.99 * len(ms))) - 1)],
            "last": out}


def _class_taus(dets, n_comp, comps_per_class=6, q=99.0):
    """Per-class threshold: the q-th percentile of the class's scores over every scored position (from the full FP32
    form, which matches the FP64 oracle to 1e-5 of the largest score)."""
    taus = np.full(n_comp, np.inf, dtype=np.float64)
    cls = dets["component"] // comps_per_class
    for c in range(n_comp // comps_per_class):
        sc = dets["score"][cls == c]
        if len(sc):
            taus[c * comps_per_class:(c + 1) * comps_per_class] = np.percentile(sc, q)
    return taus


def run_bank(args):
    """c4: the 20-class bank on a batch of 64 images. Every variant is timed (one batch call + detection readback per
    step); agreement of each with the full FP32 form under per-class thresholds; error of sampled filter maps against
    the full FP32 form's and against the FP64 oracle (the filters rebuilt from the library's factors for the decomposed
    forms)."""
    import torch
    from oracle import oracle as orc
    from paper_1707_03268_gb300 import tdpm

    torch.cuda.set_device(0)
    wl = synth.config_c4()
    n_comp = len(wl.model.components)
    ctx = tdpm.tdpm_create(0)
    tdpm.tdpm_set_fusion(ctx, not args.no_fuse)
    mid = tdpm.tdpm_load_model(ctx, wl.model)
    dps = [tdpm.DevicePyramid([torch.from_numpy(l).cuda() for l in p.levels], p.lam) for p in wl.pyramids]
    cells = sum(l.shape[0] * l.shape[1] for p in wl.pyramids for l in p.levels)
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    cap = 1 << 22
    det_buf = pinned_records(torch, tdpm, cap)
    steps = max(3, min(args.steps, 20 if args.workload == "c3" else 5))
    warmup = max(3, min(args.warmup, 3))

    def detections(form, prec, taus):
        sid = tdpm.tdpm_build_batch_scores(ctx, mid, dps, form, prec, stream)
        d = tdpm.tdpm_detect_thresholds(ctx, sid, np.broadcast_to(taus, (len(dps), n_comp)), capacity=cap,
                                        stream=stream, out=det_buf)
        tdpm.tdpm_release(ctx, sid)
        return d

    def keys(d):
        return set(zip(d["image"].tolist(), d["component"].tolist(), d["level"].tolist(), d["y"].tolist(),
                       d["x"].tolist()))

    # thresholds from the full FP32 form
    sid = tdpm.tdpm_build_batch_scores(ctx, mid, dps[:1], tdpm.FORM_FULL, tdpm.PREC_FP32, stream)
    allp = tdpm.tdpm_detect(ctx, sid, -np.inf, capacity=1 << 24, stream=stream,
                            out=np.zeros(1 << 24, dtype=tdpm.DETECTION_DTYPE)).copy()
    tdpm.tdpm_release(ctx, sid)
    taus = _class_taus(allp, n_comp)
    del allp

    S, Tr = (int(v) for v in args.ranks.split(",")) if args.ranks else DEFAULT_PAIR
    pair = f"{S}/{Tr}"
    variants = [("full", "fp32", None, None), ("full", "bf16", None, None), ("full", "bf16x3", None, None),
                ("full", "fp8", None, None), ("decomposed", "bf16x3", pair, "per_filter"),
                ("decomposed", "bf16", pair, "per_filter"), ("decomposed", "bf16", 8, "joint")]
    head = ("decomposed", "bf16x3", pair, "per_filter") if args.form == "decomposed" and args.mode == "per_filter" \
        else (args.form, args.precision, args.rank if args.form == "decomposed" else None,
              args.mode if args.form == "decomposed" else None)
    if head not in variants:
        variants.append(head)

    def vlabel(v):
        return f"{v[0]}_{v[1]}" + (f"_{v[3]}_r{str(v[2]).replace('/', '_')}" if v[2] else "")
    if args.variants:
        keep = set(args.variants.split(","))
        variants = [v for v in variants if vlabel(v) in keep]
        if variants and head not in variants:
            head = variants[0]
    rng = np.random.default_rng(0)
    filters = wl.model.filters()
    # sampled filter maps of image 0 in the full FP32 form (itself checked against the FP64 oracle by the tests): the
    # reference of each variant's map error
    pyr0 = wl.pyramids[0]
    sample_maps = []
    sid = tdpm.tdpm_build_batch_scores(ctx, mid, dps[:1], tdpm.FORM_FULL, tdpm.PREC_FP32, stream)
    for _ in range(12):
        fid = int(rng.integers(0, len(filters)))
        f = filters[fid]
        js = [j for j in range(len(pyr0.levels)) if pyr0.levels[j].shape[0] >= f.shape[0] and
              pyr0.levels[j].shape[1] >= f.shape[1]]
        j = js[len(js) // 3]
        try:
            ref = tdpm.tdpm_get_maps(ctx, sid, tdpm.MAP_FILTER_SCORE, fid, j, image=0).astype(np.float64)
        except tdpm.TdpmError:
            continue  # this filter's role does not score this level
        if ref.size:
            # the FP64 oracle's map of the exact filter (what every form's error is measured against)
            ref64 = orc.correlate(pyr0.levels[j], f.astype(np.float64))
            sample_maps.append((fid, j, ref, ref64))
    tdpm.tdpm_release(ctx, sid)
    results = {}
    ref_keys = None
    head_clocks = None
    for form_s, prec_s, r, mode in variants:
        form = tdpm.FORM_FULL if form_s == "full" else tdpm.FORM_DECOMPOSED
        prec = PRECISIONS[prec_s]
        rep = None
        if form == tdpm.FORM_DECOMPOSED:
            t0 = time.perf_counter()
            if mode == "joint":
                rep = tdpm.tdpm_decompose(ctx, mid, r, tdpm.DECOMP_JOINT, max_iters=30, seed=1)
            else:
                rs, rt = (int(v) for v in str(r).split("/"))
                rep = tdpm.tdpm_decompose_ranks(ctx, mid, filter_ranks(wl.model, rs, rt), max_iters=args.als_iters,
                                                seed=1)
            rep["seconds"] = time.perf_counter() - t0
        is_head = (form_s, prec_s, r, mode) == head
        if is_head:
            sampler = ClockSampler(0)
            sampler.start()
        run = _timed_steps(torch, lambda: detections(form, prec, taus), steps, warmup, flush, stream)
        if is_head:
            head_clocks = sampler.stop()
        k = keys(run["last"])
        # one more step with every stage bracketed by events (shape groups serial on the stream)
        tdpm.tdpm_profile_reset(ctx)
        tdpm.tdpm_profile_enable(ctx, True)
        detections(form, prec, taus)
        tdpm.tdpm_profile_enable(ctx, False)
        stages = {n: ms for n, (ms, _) in tdpm.tdpm_profile_read(ctx).items()}
        if ref_keys is None:
            ref_keys = k
        label = vlabel((form_s, prec_s, r, mode))
        # error of the sampled filter maps (image 0) against the full FP32 form's: what the precision and, for the
        # decomposed forms, the decomposition give up
        sid = tdpm.tdpm_build_batch_scores(ctx, mid, dps[:1], form, prec, stream)
        rebuilt = factor_filters(tdpm, ctx, mid) if form == tdpm.FORM_DECOMPOSED else None
        err_full = err64 = err64_same = 0.0
        for fid, j, ref, ref64 in sample_maps:
            got = tdpm.tdpm_get_maps(ctx, sid, tdpm.MAP_FILTER_SCORE, fid, j, image=0).astype(np.float64)
            scale = max(np.max(np.abs(ref64)), 1e-30)
            err_full = max(err_full, float(np.max(np.abs(got - ref)) / scale))
            err64 = max(err64, float(np.max(np.abs(got - ref64)) / scale))
            if rebuilt is not None:
                same = orc.correlate(pyr0.levels[j], rebuilt[fid])
                err64_same = max(err64_same, float(np.max(np.abs(got - same)) / scale))
        tdpm.tdpm_release(ctx, sid)
        n_img = len(dps)
        results[label] = {"images_per_s": steps * n_img / (run["ms_sum"] / 1e3), "p50_ms_per_step": run["p50"],
                          "p99_ms_per_step": run["p99"], "detections": len(k),
                          "agreement_with_full_fp32": len(k & ref_keys) / max(1, len(k | ref_keys)),
                          "max_rel_error_vs_full_fp32_maps": err_full,
                          "max_rel_error_vs_fp64_oracle_exact_filters": err64,
                          "max_rel_error_vs_fp64_oracle_same_factors": err64_same if rebuilt is not None else None,
                          "stages_ms_per_step": stages, "decomposition_report": rep}
    hl = vlabel(head)
    h = results[hl]
    line = {"metric": METRIC, "value": h["images_per_s"], "unit": "images/s", "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": None, "p50_ms": h["p50_ms_per_step"], "p99_ms": h["p99_ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision if args.precision != "fp32" else "f32", "data": "synthetic",
            "config": {"workload": wl.name, "images": len(dps), "cells": cells, "components": n_comp,
                       "filters": len(filters), "form": head[0], "precision": head[1], "rank": head[2],
                       "decomposition": head[3], "thresholds": "99th percentile of each class's scores (full FP32)",
                       "l2": "flushed between timed steps (256 MB write outside the events)"},
            "clocks": head_clocks, "variants": results, "autotune": tdpm.tdpm_autotune_read(ctx)}
    print(json.dumps(line), flush=True)
    tdpm.tdpm_destroy(ctx)


# ------------------------------------------------------------------------------------------------ serving (c5)
def run_serve(args):
    """c5: an open-loop Poisson stream of requests into the library's server; each request is one image (one of three
    sizes, its pyramid already on the device) and a set of classes of the 20-class bank (a component subset of the
    bank model). Latency = results ready - submission; throughput = requests completed / stream length."""
    import threading
    import torch
    from paper_1707_03268_gb300 import tdpm

    torch.cuda.set_device(0)
    rng = np.random.default_rng(4)
    comps = []
    for _ in range(20):
        comps.extend(synth.make_dpm_class(rng))
    ctx = tdpm.tdpm_create(0)
    tdpm.tdpm_set_fusion(ctx, not args.no_fuse)
    bank = tdpm.tdpm_load_model(ctx, synth.Model(comps))
    form = tdpm.FORM_FULL if args.form == "full" else tdpm.FORM_DECOMPOSED
    prec = PRECISIONS[args.precision]
    ranks_used = None
    if form == tdpm.FORM_DECOMPOSED:
        if args.mode == "joint":
            tdpm.tdpm_decompose(ctx, bank, args.rank, tdpm.DECOMP_JOINT, max_iters=30, seed=1)
        else:
            ranks_used = (tuple(int(v) for v in args.ranks.split(",")) if args.ranks
                          else (args.rank, args.rank) if args.rank else DEFAULT_PAIR)
            tdpm.tdpm_decompose_ranks(ctx, bank, filter_ranks(synth.Model(comps), *ranks_used),
                                      max_iters=args.als_iters, seed=1)
    sizes = ((480, 640), (720, 1280), (1080, 1920))
    pyrs = {hw: tdpm.DevicePyramid([torch.from_numpy(l).cuda()
                                    for l in synth.make_pyramid(rng, synth.pyramid_sizes(*hw), synth.LAMBDA).levels],
                                   synth.LAMBDA) for hw in sizes}
    n_req = int(args.serve_seconds * args.serve_rate)
    reqs = synth.serving_requests(seed=4, n=n_req, rate_hz=args.serve_rate, sizes=sizes)
    n_warm = min(len(reqs) // 6, int(2000 * args.serve_rate / 200.0))
    # one threshold for every class: the 99th percentile of the bank's scores on the 1280x720 image (full FP32)
    sid = tdpm.tdpm_build_pyramid_scores(ctx, bank, pyrs[(720, 1280)], tdpm.FORM_FULL, tdpm.PREC_FP32)
    tau = float(np.percentile(tdpm.tdpm_detect(ctx, sid, -np.inf, capacity=1 << 24)["score"], 99))
    tdpm.tdpm_release(ctx, sid)
    tdpm.tdpm_server_start(ctx, max_batch_images=16, max_inflight=3, max_wait_us=500, mem_budget_bytes=96 << 30)
    # warm the plans and the tuner for each size with one request alone
    for hw in sizes:
        t = tdpm.tdpm_submit(ctx, pyrs[hw], [bank], form, prec, tau, list(range(6)))
        tdpm.tdpm_poll(ctx, t)
    tickets = [None] * len(reqs)
    t0 = time.perf_counter()

    def submitter():
        for i, r in enumerate(reqs):
            delay = r["t_arrival"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            cs = [6 * c + k for c in r["classes"] for k in range(6)]
            tickets[i] = tdpm.tdpm_submit(ctx, pyrs[r["img_hw"]], [bank], form, prec, tau, cs)

    th = threading.Thread(target=submitter)
    clocks = ClockSampler(0)
    clocks.start()
    th.start()
    lat, n_det, done_t = [], 0, []
    for i in range(len(reqs)):
        while tickets[i] is None:
            time.sleep(0.0002)
        d, info = tdpm.tdpm_poll(ctx, tickets[i])
        n_det += len(d)
        lat.append((info["t_done_ns"] - info["t_submit_ns"]) / 1e6)
        done_t.append(time.perf_counter() - t0)
    th.join()
    clk = clocks.stop()
    wall = time.perf_counter() - t0
    tdpm.tdpm_server_stop(ctx)
    meas = sorted(lat[n_warm:])
    span = done_t[-1] - done_t[n_warm - 1] if n_warm > 0 else done_t[-1]
    thr = (len(reqs) - n_warm) / span
    line = {"metric": "requests/s and p50/p99 latency under a Poisson stream (continuous batching)",
            "value": thr, "unit": "images/s", "n_gpus": 1, "steps": len(reqs) - n_warm, "warmup": n_warm,
            "ms_per_step": None, "p50_ms": meas[len(meas) // 2],
            "p99_ms": meas[min(len(meas) - 1, int(math.ceil(0.99 * len(meas))) - 1)],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision if args.precision != "fp32" else "f32", "data": "synthetic",
            "config": {"workload": f"c5_serving_{args.serve_rate:g}rps", "offered_rate": args.serve_rate,
                       "requests": len(reqs), "warmup_requests_excluded": n_warm, "sizes": [f"{w}x{h}" for h, w in sizes],
                       "classes_per_request": "U{1..20} distinct of a 20-class bank (component subsets of one model)",
                       "form": args.form, "precision": args.precision,
                       "rank": (args.rank if args.mode == "joint" else None) if form == tdpm.FORM_DECOMPOSED else None,
                       "rank_root_S": ranks_used[0] if ranks_used else None,
                       "rank_part_T": ranks_used[1] if ranks_used else None,
                       "decomposition": args.mode if form == tdpm.FORM_DECOMPOSED else None,
                       "server": {"max_batch_images": 16, "max_inflight": 3, "max_wait_us": 500},
                       "tau": tau},
            "latency_ms_mean": float(np.mean(meas)), "detections": n_det, "wall_s": wall, "clocks": clk,
            "autotune": tdpm.tdpm_autotune_read(ctx)}
    print(json.dumps(line), flush=True)
    tdpm.tdpm_destroy(ctx)


# ------------------------------------------------------------------------------------------------ main arm
def _host_ms(fn, reps=20):
    fn()
    t0 = time.perf_counter()
    for _ in range(reps):
        fn()
    return (time.perf_counter() - t0) * 1e3 / reps


def nms_measure(tdpm, ctx, mid, dp, form, prec, tau, stream):
    """Greedy NMS of the headline detections, with every component in one class and with one class per component."""
    sid = tdpm.tdpm_build_pyramid_scores(ctx, mid, dp, form, prec, stream)
    dets = tdpm.tdpm_detect(ctx, sid, tau, stream=stream)
    out = {"detections": len(dets)}
    for name, cls in (("one_class", None), ("per_component", list(range(6)))):
        kept = tdpm.tdpm_detect_nms(ctx, sid, tau, cls, 0.5, 4.0, stream=stream)
        out[name] = {"kept": len(kept), "ms_per_call_host": _host_ms(
            lambda: tdpm.tdpm_detect_nms(ctx, sid, tau, cls, 0.5, 4.0, stream=stream))}
    out["detect_ms_per_call_host"] = _host_ms(lambda: tdpm.tdpm_detect(ctx, sid, tau, stream=stream))
    tdpm.tdpm_release(ctx, sid)
    return out


def hog_measure(torch, tdpm, ctx, mid, form, prec, stream, score_ms, peaks, h=375, w=500, steps=200):
    """The feature extraction block on a 500x375 8-bit image: HOG pyramid time on the device (inputs resident, CUDA
    events), its share of the scoring time (the paper puts scoring at about 20x extraction), and image -> detections
    end to end (image H2D from pinned memory, HOG pyramid, scoring, detection read-back)."""
    img = synth.make_image(np.random.default_rng(21), h, w)
    host = torch.from_numpy(img).pin_memory()
    d_img = host.cuda()
    shapes, nbytes = tdpm.tdpm_hog_pyramid_shape(h, w)
    out = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    pyr = None
    pyr = tdpm.HogPyramid(h, w, out=out)
    for _ in range(5):
        pyr.compute(ctx, d_img, stream)
    torch.cuda.synchronize()
    l0 = tdpm.tdpm_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        pyr.compute(ctx, d_img, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    hog_ms = e0.elapsed_time(e1) / steps
    launches = (tdpm.tdpm_kernel_launches() - l0) / steps
    # detections from the device pyramid, end to end
    tau = None

    def e2e():
        d_img.copy_(host, non_blocking=True)
        pyr.compute(ctx, d_img, stream)
        sid = tdpm.tdpm_build_pyramid_scores(ctx, mid, pyr, form, prec, stream)
        d = tdpm.tdpm_detect(ctx, sid, tau, stream=stream)
        tdpm.tdpm_release(ctx, sid)
        return d

    sid = tdpm.tdpm_build_pyramid_scores(ctx, mid, pyr, form, prec, stream)
    tau = float(np.percentile(tdpm.tdpm_detect(ctx, sid, -np.inf, stream=stream)["score"], 99.5))
    tdpm.tdpm_release(ctx, sid)
    for _ in range(5):
        e2e()
    torch.cuda.synchronize()
    e0.record(stream)
    n_e2e = 100
    for _ in range(n_e2e):
        n_det = len(e2e())
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / n_e2e
    alg_bytes = h * w * 3 + nbytes  # the image read once, the features written once
    hbm = (peaks or {}).get("hbm_gbs")
    return {"image": f"{w}x{h}", "levels": len(shapes), "feature_bytes": nbytes, "hog_ms_per_image": hog_ms,
            "launches_per_image": launches, "scoring_ms_over_hog_ms": score_ms / hog_ms,
            "roofline": {"bound": "hbm", "algorithmic_bytes": alg_bytes, "achieved_gbs": alg_bytes / hog_ms / 1e6,
                         "peak_gbs": hbm, "frac": (alg_bytes / hog_ms / 1e6 / hbm) if hbm else None},
            "image_to_detections_images_per_s": 1e3 / e2e_ms, "image_to_detections_ms": e2e_ms,
            "detections": n_det, "tau": tau, "h2d_bytes_per_step": h * w * 3}


def cascade_measure(torch, tdpm, ctx, mid, wl, form, prec, tau, stream, n_train=4, per_comp=5):
    """Thresholds of Sec. 4 from planted positives on n_train training images of the workload's size (per_comp
    instances of every component each), then the cascade on the workload image with two planted instances per
    component: pruned share of all root hypotheses, CP terms evaluated, recall of the planted instances, and the
    detections kept at the headline threshold."""
    pyr = wl.pyramids[0]
    rng = np.random.default_rng(11)

    def dev(p):
        return tdpm.DevicePyramid([torch.from_numpy(np.ascontiguousarray(l)).cuda() for l in p.levels], p.lam)

    def places(base, k):
        sid = tdpm.tdpm_build_pyramid_scores(ctx, mid, dev(base), form, prec, stream)
        allr = tdpm.tdpm_detect(ctx, sid, -np.inf, stream=stream)
        tdpm.tdpm_release(ctx, sid)
        out = []
        for c in range(len(wl.model.components)):
            idx = np.nonzero(allr["component"] == c)[0]
            for i in sorted(rng.choice(idx, size=k, replace=False)):
                out.append((c, int(allr["level"][i]), int(allr["y"][i]), int(allr["x"][i])))
        return out

    def records(pl):
        r = np.zeros(len(pl), dtype=tdpm.DETECTION_DTYPE)
        for i, (im, c, j, y, x) in enumerate(pl):
            r[i]["image"], r[i]["component"], r[i]["level"], r[i]["y"], r[i]["x"] = im, c, j, y, x
        return r

    train, pos = [], []
    for im in range(n_train):
        base = synth.make_pyramid(rng, pyr.sizes, pyr.lam)
        pl = places(base, per_comp)
        train.append(dev(synth.plant_objects(rng, base, wl.model, pl)))
        pos += [(im,) + p for p in pl]
    s_train = tdpm.tdpm_build_batch_scores(ctx, mid, train, form, prec, stream)
    t = tdpm.tdpm_cascade_thresholds(ctx, s_train, train, records(pos), mid, stream)
    tdpm.tdpm_release(ctx, s_train)
    pl_test = places(pyr, 2)
    d_test = dev(synth.plant_objects(rng, pyr, wl.model, pl_test))
    s_test = tdpm.tdpm_build_pyramid_scores(ctx, mid, d_test, form, prec, stream)
    kept, st = tdpm.tdpm_detect_cascade(ctx, s_test, [d_test], t, -np.inf, stream=stream)
    kkeys = set(zip(kept["component"].tolist(), kept["level"].tolist(), kept["y"].tolist(), kept["x"].tolist()))
    dense = tdpm.tdpm_detect(ctx, s_test, tau, stream=stream)
    kept_tau, _ = tdpm.tdpm_detect_cascade(ctx, s_test, [d_test], t, tau, stream=stream)
    out = {"positives": len(pos), "training_images": n_train, "hypotheses": st["candidates"],
           "pruned_fraction": st["pruned"] / max(1, st["candidates"]),
           "terms_evaluated_fraction": st["terms_evaluated"] / max(1, st["terms_total"]),
           "recall_planted": sum(1 for p in pl_test if p in kkeys) / len(pl_test),
           "dense_detections_at_tau": len(dense), "cascade_detections_at_tau": len(kept_tau),
           "ms_per_call_host_all_hypotheses": _host_ms(
               lambda: tdpm.tdpm_detect_cascade(ctx, s_test, [d_test], t, -np.inf, stream=stream), 10),
           "detect_ms_per_call_host_all_hypotheses": _host_ms(
               lambda: tdpm.tdpm_detect(ctx, s_test, -np.inf, stream=stream), 10)}
    tdpm.tdpm_release(ctx, s_test)
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "c4":
        run_bank(args)
        return
    if args.workload == "c5":
        run_serve(args)
        return
    import torch
    import torch.distributed as dist
    from paper_1707_03268_gb300 import tdpm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    form = tdpm.FORM_DECOMPOSED if args.form == "decomposed" else tdpm.FORM_FULL
    prec = PRECISIONS[args.precision]
    joint = args.mode == "joint"
    dmode = tdpm.DECOMP_JOINT if joint else tdpm.DECOMP_PER_FILTER
    wl = workload_of(args.workload)
    pyr = wl.pyramids[0]
    n_comp = len(wl.model.components)
    taus = load_taus(args.workload, n_comp)
    ctx = tdpm.tdpm_create(local)
    tdpm.tdpm_set_fusion(ctx, not args.no_fuse)
    mid = tdpm.tdpm_load_model(ctx, wl.model)
    # the pyramid in one flat device buffer (levels are views), so that a host copy is one transfer
    host_flat = torch.from_numpy(np.concatenate([l.reshape(-1) for l in pyr.levels])).pin_memory()
    dev_flat = host_flat.cuda()
    levels, off = [], 0
    for l in pyr.levels:
        levels.append(dev_flat[off:off + l.size].view(l.shape))
        off += l.size
    dp = tdpm.DevicePyramid(levels, pyr.lam)
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    cap = 1 << 20
    det_buf = pinned_records(torch, tdpm, cap)
    tau_rows = np.ascontiguousarray(taus[None, :])

    def step(f, p, pyramid=None):
        sid = tdpm.tdpm_build_pyramid_scores(ctx, mid, pyramid or dp, f, p, stream)
        dets = tdpm.tdpm_detect_thresholds(ctx, sid, tau_rows, capacity=cap, stream=stream, out=det_buf)
        tdpm.tdpm_release(ctx, sid)
        return dets

    def keys(d):
        return set(zip(d["component"].tolist(), d["level"].tolist(), d["y"].tolist(), d["x"].tolist()))

    def agree(a, b):
        return len(a & b) / max(1, len(a | b))

    def timed(f, p, steps, warmup, prof=False, label=None):
        for _ in range(warmup):
            step(f, p)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        if label:
            torch.cuda.nvtx.range_push(label)  # the timed steps only, for profilers (ncu --nvtx-include "label/")
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if prof:
            tdpm.tdpm_profile_reset(ctx)
            tdpm.tdpm_profile_enable(ctx, True)
        launches0 = tdpm.tdpm_kernel_launches()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for i in range(steps):
            flush.zero_()  # evict the pyramid and the arena from L2 between steps (outside the events)
            ev[i][0].record(stream)
            step(f, p)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        if label:
            torch.cuda.nvtx.range_pop()
        if world > 1:
            dist.barrier()
        wall = time.perf_counter() - t0
        launches = tdpm.tdpm_kernel_launches() - launches0
        stages = None
        if prof:
            tdpm.tdpm_profile_enable(ctx, False)
            stages = tdpm.tdpm_profile_read(ctx)
        ms = [a.elapsed_time(b) for a, b in ev]
        total_ms = max_over_ranks(sum(ms), world)
        return {"ms": ms, "total_ms": total_ms, "wall_s": wall, "launches": launches, "stages": stages}

    def rate(run):
        return job_rate(len(run["ms"]), world, run["total_ms"])

    n_cmp = max(5, min(50, args.steps // 4))
    # ---- the reference of the agreement: the full form in FP32 (the plain FP32 GPU baseline)
    full32 = timed(tdpm.FORM_FULL, tdpm.PREC_FP32, n_cmp, 2)
    full_keys = keys(step(tdpm.FORM_FULL, tdpm.PREC_FP32))

    # ---- decomposition: a fixed rank, a fixed (S, T) pair, or the rank ladder
    rep, ladder, ranks_used = None, None, None
    if form == tdpm.FORM_DECOMPOSED:
        if joint:
            rep = tdpm.tdpm_decompose(ctx, mid, args.rank, dmode, max_iters=args.als_iters, seed=1)
        elif args.rank is not None or args.ranks is not None:
            S, T = (args.rank, args.rank) if args.rank is not None else tuple(int(v) for v in args.ranks.split(","))
            ranks_used = (S, T)
            rep = tdpm.tdpm_decompose_ranks(ctx, mid, filter_ranks(wl.model, S, T), max_iters=args.als_iters, seed=1)
        else:
            ladder = []
            for S, T in RANK_LADDER:
                t0 = time.perf_counter()
                rep = tdpm.tdpm_decompose_ranks(ctx, mid, filter_ranks(wl.model, S, T), max_iters=args.als_iters,
                                                seed=1)
                secs = time.perf_counter() - t0
                a = agree(keys(step(form, prec)), full_keys)
                run = timed(form, prec, 3, 1)
                ladder.append({"S_root": S, "T_part": T, "agreement_with_full_fp32": a, "images_per_s": rate(run),
                               "max_rel_error": rep["max_rel_error"], "mean_rel_error": rep["mean_rel_error"],
                               "gain_formula_1": rep["gain"], "decompose_seconds": secs})
                ranks_used = (S, T)
                if a >= AGREEMENT_BAR:
                    break

    # ---- headline run (an NVTX range marks its timed steps for profilers: ncu --nvtx --nvtx-include "headline/")
    clocks = ClockSampler(local)
    clocks.start()
    main_run = timed(form, prec, args.steps, args.warmup, label="headline")
    clk = clocks.stop()
    value = rate(main_run)
    ms_sorted = sorted(main_run["ms"])
    p50 = ms_sorted[len(ms_sorted) // 2]
    p99 = ms_sorted[min(len(ms_sorted) - 1, int(math.ceil(0.99 * len(ms_sorted))) - 1)]
    head_dets = step(form, prec).copy()
    head_keys = keys(head_dets)
    agreement = agree(head_keys, full_keys)

    # ---- per-stage device time (same workload, CUDA events around each stage on its stream)
    prof_run = timed(form, prec, max(5, min(20, args.steps // 4)), 1, prof=True)
    stages = prof_run["stages"]
    n_prof = len(prof_run["ms"])
    rank_model = (filter_ranks(wl.model, *ranks_used) if ranks_used else args.rank) if form == tdpm.FORM_DECOMPOSED \
        else None
    model = stage_bytes(wl, pyr, args.form, args.precision, rank_model, joint, fused=not args.no_fuse)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    sm_mhz = (clk or {}).get("sm_mhz") or 1920.0
    rooflines = {name: stage_roofline(name, ms / n_prof, n / n_prof, model, peaks, sm_mhz)
                 for name, (ms, n) in stages.items() if name in model}
    for name, r in rooflines.items():
        r["traffic"] = measured_traffic(args.workload, args.form, args.precision, args.mode, name)
    dom_name = max(stages.items(), key=lambda kv: kv[1][0])[0]
    roofline = rooflines.get(dom_name)

    # ---- end to end through the public API: pyramid H2D from pinned host memory, detections D2H. Two device copies
    # of the pyramid: the next image's transfer (on a copy stream) overlaps this image's scoring; a buffer is written
    # again only after the detection read-back of the step that scored it has returned.
    h2d = host_flat.numel() * 4
    dev_flat2 = torch.empty_like(dev_flat)
    levels2, off = [], 0
    for l in pyr.levels:
        levels2.append(dev_flat2[off:off + l.size].view(l.shape))
        off += l.size
    bufs = [dev_flat, dev_flat2]
    pyrs = [dp, tdpm.DevicePyramid(levels2, pyr.lam)]
    copy_stream = torch.cuda.Stream()
    ready = [torch.cuda.Event(), torch.cuda.Event()]

    def prefetch(k):
        with torch.cuda.stream(copy_stream):
            bufs[k].copy_(host_flat, non_blocking=True)  # every level of the image, one transfer from pinned memory
            ready[k].record(copy_stream)

    def e2e_step(i):
        cur = i % 2
        stream.wait_event(ready[cur])
        sid = tdpm.tdpm_build_pyramid_scores(ctx, mid, pyrs[cur], form, prec, stream)
        prefetch(1 - cur)  # queued after this step's job-table upload, so that upload does not wait behind it
        dets = tdpm.tdpm_detect_thresholds(ctx, sid, tau_rows, capacity=cap, stream=stream, out=det_buf)
        tdpm.tdpm_release(ctx, sid)
        return dets

    prefetch(0)
    for i in range(args.warmup):
        e2e_step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    n_det = 0
    for i in range(args.steps):
        n_det = len(e2e_step(args.warmup + i))
    ev1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    e2e = {"value": job_rate(args.steps, world, e2e_ms), "unit": "images/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": n_det * tdpm.DETECTION_DTYPE.itemsize + 8,
           "note": "the next image's pyramid transfer overlaps the current image's scoring (two device buffers)"}

    # ---- the full form in the tensor-core precisions on the same image: speed and agreement with full FP32
    compare = {"full_fp32_images_per_s": rate(full32), "full_fp32_p50_ms": sorted(full32["ms"])[len(full32["ms"]) // 2],
               "speedup_vs_full_fp32": value / rate(full32), "agreement_with_full_fp32": agreement,
               "detections": len(head_keys), "detections_full_fp32": len(full_keys)}
    if not args.no_compare:
        for pname in ("bf16x3", "bf16", "fp8"):
            run = timed(tdpm.FORM_FULL, PRECISIONS[pname], n_cmp, 2)
            k = keys(step(tdpm.FORM_FULL, PRECISIONS[pname]))
            compare[f"full_{pname}_images_per_s"] = rate(run)
            compare[f"full_{pname}_agreement_with_full_fp32"] = agree(k, full_keys)
        if form == tdpm.FORM_DECOMPOSED:
            compare["speedup_vs_full_bf16x3"] = value / compare["full_bf16x3_images_per_s"]

    # ---- oracle leg: CPU baseline and parity of the headline detections (same filters)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        filters = factor_filters(tdpm, ctx, mid) if form == tdpm.FORM_DECOMPOSED else None
        cpu = cpu_baseline_oracle(wl, filters, head_keys, taus)

    # ---- accuracy given up by the decomposition: agreement with the full FP32 form per uniform rank
    sweep = None
    if form == tdpm.FORM_DECOMPOSED and not joint and not args.no_sweep and args.workload == "c2":
        sweep = {}
        for r in RANK_SWEEP["per_filter"]:
            rr = tdpm.tdpm_decompose(ctx, mid, r, dmode, max_iters=500, seed=1)
            a = keys(step(form, prec))
            run = timed(form, prec, 50, 2)
            sweep[r] = {"agreement_with_full_fp32": agree(a, full_keys), "images_per_s": rate(run),
                        "max_rel_error": rr["max_rel_error"], "mean_rel_error": rr["mean_rel_error"],
                        "gain_formula_1": rr["gain"]}

    # ---- rank detection (Sec. 4): per filter the smallest rank meeting the error criterion with constant e
    auto_sweep = None
    if form == tdpm.FORM_DECOMPOSED and not joint and not args.no_sweep and args.workload == "c2":
        auto_sweep = {}
        for e in AUTO_RANK_E:
            t0 = time.perf_counter()
            rr, ranks = tdpm.tdpm_decompose_auto(ctx, mid, e, 36, max_iters=500, seed=1)
            secs = time.perf_counter() - t0
            a = keys(step(form, prec))
            run = timed(form, prec, 50, 2)
            auto_sweep[e] = {"ranks_mean": float(np.mean(ranks)), "ranks_min": int(ranks.min()),
                             "ranks_max": int(ranks.max()), "gain_formula_1": rr["gain"],
                             "max_rel_error": rr["max_rel_error"], "mean_rel_error": rr["mean_rel_error"],
                             "agreement_with_full_fp32": agree(a, full_keys), "images_per_s": rate(run),
                             "decompose_seconds": secs}

    # ---- post-processing on the one-class model: NMS (f4), convolution shortening (f1), HOG pyramid (f3)
    post = None
    if form == tdpm.FORM_DECOMPOSED and not joint and not args.no_sweep and rank == 0 and args.workload == "c2":
        tdpm.tdpm_decompose_ranks(ctx, mid, filter_ranks(wl.model, *ranks_used), max_iters=args.als_iters, seed=1)
        tau = float(taus[0])
        post = {"nms": nms_measure(tdpm, ctx, mid, dp, form, prec, tau, stream),
                "cascade": cascade_measure(torch, tdpm, ctx, mid, wl, form, prec, tau, stream),
                "hog": hog_measure(torch, tdpm, ctx, mid, form, prec, stream, main_run["total_ms"] / args.steps,
                                   peaks)}

    line = {"metric": METRIC, "value": value, "unit": "images/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main_run["total_ms"] / args.steps, "p50_ms": p50, "p99_ms": p99,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision if prec != tdpm.PREC_FP32 else "f32", "data": "synthetic",
            "config": {"workload": wl.name, "image": "x".join(str(v) for v in
                                                             {"c2": (500, 375), "c3": (1280, 720)}[args.workload]),
                       "levels": len(pyr.levels), "components": n_comp, "filters": len(wl.model.filters()),
                       "form": args.form, "precision": args.precision,
                       "precision_note": {"bf16x3": "BF16 tensor cores, operands split hi+lo (3 MMAs per product), "
                                                    "FP32 accumulation",
                                          "bf16": "BF16 tensor cores, FP32 accumulation",
                                          "fp8": "E4M3 tensor cores (per-tensor scales), FP32 accumulation",
                                          "fp32": "FP32 ALUs"}[args.precision],
                       "decomposition": args.mode if form == tdpm.FORM_DECOMPOSED else None,
                       "rank_root_S": ranks_used[0] if ranks_used else (args.rank if joint else None),
                       "rank_part_T": ranks_used[1] if ranks_used else (args.rank if joint else None),
                       "als_iters": args.als_iters if form == tdpm.FORM_DECOMPOSED else None,
                       "thresholds": "per class: 99th percentile of the FP64 oracle's full-form scores"
                                     if args.workload == "c3" else "99th percentile of the FP64 oracle's scores",
                       "fused": (not args.no_fuse) if form == tdpm.FORM_DECOMPOSED else None,
                       "l2": "flushed between timed steps (256 MB write outside the events)",
                       "parallelism": f"replicas x{world}"},
            "agreement_with_full_fp32": agreement, "agreement_bar": AGREEMENT_BAR,
            "agreement_met": agreement >= AGREEMENT_BAR,
            "full_fp32_images_per_s": rate(full32), "speedup_vs_full_fp32": value / rate(full32),
            "gpu_launches": main_run["launches"],
            "stages_ms_per_image": {k: v[0] / n_prof for k, v in stages.items()},
            "roofline": roofline, "rooflines": rooflines, "e2e": e2e, "cpu_baseline": cpu, "clocks": clk,
            "compare": compare, "rank_ladder": ladder, "decomposition_report": rep, "rank_sweep": sweep,
            "auto_rank_sweep": auto_sweep, "post_processing": post,
            "autotune": tdpm.tdpm_autotune_read(ctx),
            "wall_s_timed": main_run["wall_s"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    tdpm.tdpm_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
