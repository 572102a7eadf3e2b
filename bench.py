#!/usr/bin/env python
"""Benchmark of the DPM scoring hot path (correlation, distance transform, shift-and-sum, threshold).

Workload (default): one 500x375 image as a 36-level HOG-shaped pyramid (10 levels per octave, sbin 8; 88,330 cells,
uniform [0, 0.2)), scored by a 6-component DPM-shaped class model (roots 5x11, 7x7, 11x5 and their mirrors, 8 parts of
6x6 each, 54 filters). A step is one whole pass of the path over that image: correlation (decomposed, rank 8 per
filter, on BF16 tensor cores by default), both distance-transform passes, assembly, threshold and the copy of the
detections to the host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--form decomposed|full] [--precision bf16x3|bf16|fp32]
                  [--rank R] [--mode per_filter|joint]
  python bench.py --impl reference    # the FP64 CPU oracle on the same workload and metric

Reported beside the headline: the full form in FP32 (the GPU baseline the decomposed form must beat) and in the same
precision, detection agreement with the FP64 oracle on the same factors (parity), and a rank sweep of the detection
agreement of the decomposed form with the full FP32 form (the accuracy the decomposition gives up).

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
RANK_SWEEP = {"per_filter": (4, 8, 16, 24, 32, 36), "joint": (16, 32, 64, 128, 256)}
PRECISIONS = {"fp32": 0, "bf16": 1, "bf16x3": 3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="tdpm", choices=["tdpm", "reference"])
    ap.add_argument("--form", default="decomposed", choices=["decomposed", "full"])
    ap.add_argument("--precision", default="bf16x3", choices=sorted(PRECISIONS))
    ap.add_argument("--rank", type=int, default=8, help="CP rank per filter (per_filter) or per shape group (joint)")
    ap.add_argument("--mode", default="per_filter", choices=["per_filter", "joint"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the full-form comparison runs")
    ap.add_argument("--no-sweep", action="store_true", help="skip the rank sweep")
    return ap.parse_args()


def load_tau():
    with open(os.path.join(ROOT, "tests", "golden", "thresholds.json")) as f:
        return float(json.load(f)["c2"]["tau"])


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


# ------------------------------------------------------------------------------------------------ roofline model
def stage_bytes(wl, pyr, form: str, precision: str, rank: int, joint: bool):
    """Algorithmic DRAM bytes and flops per stage for one image: every input read once, every output written once."""
    sizes = pyr.sizes
    lam = pyr.lam
    L = len(sizes)
    groups = {}
    for comp in wl.model.components:
        groups.setdefault((0,) + comp.root.shape[:2], []).append(comp.root)
        for p in comp.parts:
            groups.setdefault((1,) + p.filt.shape[:2], []).append(p.filt)
    tc = precision in ("bf16", "bf16x3")
    fb = {"fp32": 4, "bf16": 2, "bf16x3": 4}[precision]  # feature bytes per channel read by the correlation
    corr = "corr_tc" if tc else "corr_f32"
    zproj = "zproj_tc" if tc else "zproj_f32"
    out = {corr: [0, 0], zproj: [0, 0], "sep": [0, 0], "recomb_tc": [0, 0], "dt": [0, 0], "assemble": [0, 0],
           "to_bf16": [0, 0]}
    ub = 4 if precision == "bf16x3" else 2  # bytes per U_r value on the joint tensor-core path (hi + lo parts)
    if tc:
        out["to_bf16"][0] = sum(H * W * 32 * (4 + fb) for (H, W) in sizes)
    for (role, h, w), fl in groups.items():
        K = len(fl)
        if joint:
            R = min(rank, h * w * 32)       # the joint form is exact from h*w*32 shared terms on
        else:
            R = K * min(rank, h * w)        # per filter: exact from h*w terms (the slices) on
        js = range(lam, L) if role == 0 else range(0, L - lam)
        for j in js:
            H, W = sizes[j]
            Ho, Wo = H - h + 1, W - w + 1
            if Ho <= 0 or Wo <= 0:
                continue
            if form == "full":
                out[corr][0] += H * W * 32 * fb + K * Ho * Wo * 4
                out[corr][1] += 2 * h * w * 32 * K * Ho * Wo
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
                    per_filter_terms = R if joint else R // K
                    out["sep"][1] += 2 * K * Ho * Wo * per_filter_terms * (h + w + 1)
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
                # x pass: read the part map, write values + argmax at X sampled columns of every row;
                # y pass: read them back, write values + argmax at the Y x X anchored positions
                out["dt"][0] += Hs * Ws * 4 + 2 * (Hs * X * 8) + Y * X * 8
            out["assemble"][0] += Y * X * 4 * (n + 2)
    return {k: {"bytes": v[0], "flops": v[1]} for k, v in out.items()}


def fp32_alu_peak_tflops(sm_mhz: float) -> float:
    """FP32 FMA roofline: 152 SMs x 128 FP32 lanes x 2 flops per FMA x SM clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


TENSOR_STAGES = ("corr_tc", "zproj_tc", "recomb_tc")
ALU_STAGES = ("corr_f32", "zproj_f32", "sep")


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
        cand.append(("alu", f / (fp32_alu_peak_tflops(sm_mhz) * 1e12)))
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
        pk = fp32_alu_peak_tflops(sm_mhz)
        out.update(achieved=f / s / 1e12, peak=pk, unit="TFLOP/s",
                   peak_source="derived: 152 SM x 128 FP32 lanes x 2 flop x median SM clock under load")
    out["frac"] = out["achieved"] / out["peak"]
    return out


# ------------------------------------------------------------------------------------------------ oracle legs
def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, same workload and metric (rank 0 of N only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as orc

    wl = synth.config_c2()
    pyr = wl.pyramids[0]
    n_comp = len(wl.model.components)

    def one_step(i):
        # one component of the model over the whole pyramid: 1/6 of an image
        sub = synth.Model([wl.model.components[i % n_comp]])
        orc.detect(orc.score_pyramid(sub, pyr), load_tau())

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
            "config": {"workload": wl.name, "form": "full (FP64 oracle)", "image": "500x375", "levels": len(pyr.levels),
                       "components": n_comp, "filters": len(wl.model.filters())},
            "cpu_baseline": {"value": v, "unit": "images/s", "cores": orc.num_threads(), "kind": "oracle",
                             "sample": "each step scores one of the 6 components over the whole 36-level pyramid "
                                       "(1/6 of an image)"},
            "e2e": {"value": v, "unit": "images/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_oracle(wl, filters, gpu_keys, tau, budget_s: float = 15.0):
    """The FP64 oracle as it stands, on this host's cores: the same whole image with the same filters (rebuilt from
    the library's FP64 factors for the decomposed form), repeated within a time budget. Its detections also give the
    parity agreement of the GPU's detections."""
    from oracle import oracle as orc
    pyr = wl.pyramids[0]
    n = 0
    t0 = time.perf_counter()
    dets = None
    while True:
        dets = orc.detect(orc.score_pyramid(wl.model, pyr, filters=filters), tau)
        n += 1
        if time.perf_counter() - t0 >= budget_s or n >= 20:
            break
    dt = time.perf_counter() - t0
    ok = set(d[:4] for d in dets)
    return {"value": n / dt, "unit": "images/s", "cores": orc.num_threads(), "kind": "oracle",
            "sample": f"{n} whole 500x375 images (36 levels, 54 filters), FP64, same filters as the GPU run",
            "parity_agreement_with_gpu": len(ok & gpu_keys) / max(1, len(ok | gpu_keys)),
            "oracle_detections": len(ok)}


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


# ------------------------------------------------------------------------------------------------ main arm
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
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
    wl = synth.config_c2()
    pyr = wl.pyramids[0]
    tau = load_tau()
    ctx = tdpm.tdpm_create(local)
    mid = tdpm.tdpm_load_model(ctx, wl.model)
    levels = [torch.from_numpy(l).cuda() for l in pyr.levels]
    dp = tdpm.DevicePyramid(levels, pyr.lam)
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    cap = 1 << 16
    det_buf = np.zeros(cap, dtype=tdpm.DETECTION_DTYPE)

    def step(f, p):
        sid = tdpm.tdpm_build_pyramid_scores(ctx, mid, dp, f, p, stream)
        dets = tdpm.tdpm_detect(ctx, sid, tau, capacity=cap, stream=stream, out=det_buf)
        tdpm.tdpm_release(ctx, sid)
        return dets

    def keys(d):
        return set(zip(d["component"].tolist(), d["level"].tolist(), d["y"].tolist(), d["x"].tolist()))

    def timed(f, p, steps, warmup, prof=False):
        for _ in range(warmup):
            step(f, p)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
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
            flush.zero_()  # the pyramid is smaller than L2: evict it between steps (outside the events)
            ev[i][0].record(stream)
            step(f, p)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        wall = time.perf_counter() - t0
        launches = tdpm.tdpm_kernel_launches() - launches0
        stages = None
        if prof:
            tdpm.tdpm_profile_enable(ctx, False)
            stages = tdpm.tdpm_profile_read(ctx)
        ms = [a.elapsed_time(b) for a, b in ev]
        total_ms = sum(ms)
        if world > 1:
            t = torch.tensor([total_ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total_ms = float(t.item())
        return {"ms": ms, "total_ms": total_ms, "wall_s": wall, "launches": launches, "stages": stages}

    def rate(run):
        return len(run["ms"]) * world / (run["total_ms"] / 1e3)

    rep = None
    if form == tdpm.FORM_DECOMPOSED:
        rep = tdpm.tdpm_decompose(ctx, mid, args.rank, dmode, max_iters=500, seed=1)

    # ---- headline run
    clocks = ClockSampler(local)
    clocks.start()
    main_run = timed(form, prec, args.steps, args.warmup)
    clk = clocks.stop()
    value = rate(main_run)
    ms_sorted = sorted(main_run["ms"])
    p50 = ms_sorted[len(ms_sorted) // 2]
    p99 = ms_sorted[min(len(ms_sorted) - 1, int(math.ceil(0.99 * len(ms_sorted))) - 1)]
    head_keys = keys(step(form, prec))

    # ---- per-stage device time (same workload, CUDA events around each stage on its stream)
    prof_run = timed(form, prec, max(10, args.steps // 4), 1, prof=True)
    stages = prof_run["stages"]
    n_prof = len(prof_run["ms"])
    model = stage_bytes(wl, pyr, args.form, args.precision, args.rank, joint)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    sm_mhz = (clk or {}).get("sm_mhz") or 1920.0
    rooflines = {name: stage_roofline(name, ms / n_prof, n / n_prof, model, peaks, sm_mhz)
                 for name, (ms, n) in stages.items() if name in model}
    dom_name = max(stages.items(), key=lambda kv: kv[1][0])[0]
    roofline = rooflines.get(dom_name)

    # ---- end to end through the public API: pyramid H2D from pinned host memory, detections D2H
    host_levels = [torch.from_numpy(l).pin_memory() for l in pyr.levels]
    h2d = sum(l.numel() * 4 for l in host_levels)

    def e2e_step():
        for hl, dl in zip(host_levels, levels):
            dl.copy_(hl, non_blocking=True)
        return step(form, prec)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    n_det = 0
    for _ in range(args.steps):
        n_det = len(e2e_step())
    ev1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = ev0.elapsed_time(ev1)
    if world > 1:
        t = torch.tensor([e2e_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e = {"value": args.steps * world / (e2e_ms / 1e3), "unit": "images/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": n_det * tdpm.DETECTION_DTYPE.itemsize + 8}

    # ---- full-form comparison runs on the same image
    compare = None
    if not args.no_compare:
        n_cmp = max(10, args.steps // 4)
        full32 = timed(tdpm.FORM_FULL, tdpm.PREC_FP32, n_cmp, 2)
        full_keys = keys(step(tdpm.FORM_FULL, tdpm.PREC_FP32))
        compare = {"full_fp32_images_per_s": rate(full32), "full_fp32_p50_ms": sorted(full32["ms"])[n_cmp // 2],
                   "speedup_vs_full_fp32": value / rate(full32),
                   "agreement_with_full_fp32": len(head_keys & full_keys) / max(1, len(head_keys | full_keys)),
                   "detections": len(head_keys), "detections_full_fp32": len(full_keys)}
        if prec != tdpm.PREC_FP32 or form != tdpm.FORM_FULL:
            fullp = timed(tdpm.FORM_FULL, prec, n_cmp, 2)
            compare[f"full_{args.precision}_images_per_s"] = rate(fullp)

    # ---- oracle leg: CPU baseline and parity of the headline detections (same factors)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        filters = factor_filters(tdpm, ctx, mid) if form == tdpm.FORM_DECOMPOSED else None
        cpu = cpu_baseline_oracle(wl, filters, head_keys, tau)

    # ---- accuracy given up by the decomposition: agreement with the full FP32 form per rank
    sweep = None
    if form == tdpm.FORM_DECOMPOSED and not args.no_sweep and compare is not None:
        sweep = {}
        for r in RANK_SWEEP[args.mode]:
            rr = tdpm.tdpm_decompose(ctx, mid, r, dmode, max_iters=500, seed=1)
            a = keys(step(form, prec))
            run = timed(form, prec, 50, 2)
            sweep[r] = {"agreement_with_full_fp32": len(a & full_keys) / max(1, len(a | full_keys)),
                        "images_per_s": rate(run), "max_rel_error": rr["max_rel_error"],
                        "mean_rel_error": rr["mean_rel_error"], "gain_formula_1": rr["gain"]}

    line = {"metric": METRIC, "value": value, "unit": "images/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main_run["total_ms"] / args.steps, "p50_ms": p50, "p99_ms": p99,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision if prec != tdpm.PREC_FP32 else "f32", "data": "synthetic",
            "config": {"workload": wl.name, "image": "500x375", "levels": len(pyr.levels),
                       "components": len(wl.model.components), "filters": len(wl.model.filters()),
                       "form": args.form, "precision": args.precision,
                       "precision_note": {"bf16x3": "BF16 tensor cores, operands split hi+lo (3 MMAs per product), "
                                                    "FP32 accumulation",
                                          "bf16": "BF16 tensor cores, FP32 accumulation",
                                          "fp32": "FP32 ALUs"}[args.precision],
                       "rank": args.rank if form == tdpm.FORM_DECOMPOSED else None,
                       "decomposition": args.mode if form == tdpm.FORM_DECOMPOSED else None,
                       "l2": "flushed between timed steps (256 MB write outside the events)",
                       "parallelism": f"replicas x{world}"},
            "gpu_launches": main_run["launches"],
            "stages_ms_per_image": {k: v[0] / n_prof for k, v in stages.items()},
            "roofline": roofline, "rooflines": rooflines, "e2e": e2e, "cpu_baseline": cpu, "clocks": clk,
            "compare": compare, "decomposition_report": rep, "rank_sweep": sweep,
            "autotune": tdpm.tdpm_autotune_read(ctx),
            "wall_s_timed": main_run["wall_s"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    tdpm.tdpm_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
