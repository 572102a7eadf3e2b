#!/usr/bin/env python
"""Benchmark of the DPM scoring hot path (correlation, distance transform, shift-and-sum, threshold).

Workload (default): one 500x375 image as a 36-level HOG-shaped pyramid (10 levels per octave, sbin 8; 88,330 cells,
uniform [0, 0.2)), scored by a 6-component DPM-shaped class model (roots 5x11, 7x7, 11x5 and their mirrors, 8 parts of
6x6 each, 54 filters). A step is one whole pass of the path over that image: correlation (decomposed BF16 by default),
both distance-transform passes, assembly, threshold and the copy of the detections to the host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--form decomposed|full] [--precision bf16|fp32] [--rank R]
  python bench.py --impl reference    # the FP64 CPU oracle on the same workload and metric

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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1707_03268_gb300 import synth  # noqa: E402

METRIC = "images/sec and p50/p99 latency, decomposed BF16 vs full FP32, at >=99.5% agreement"
L2_BYTES = 129 * 1024 * 1024
RANK_LADDER = (4, 6, 8, 12, 16, 20, 24, 28, 32)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="tdpm", choices=["tdpm", "reference"])
    ap.add_argument("--form", default="decomposed", choices=["decomposed", "full"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--rank", type=int, default=0,
                    help="CP rank of the decomposed form; 0 = the smallest rank of RANK_LADDER whose detections agree "
                         ">= 99.5%% with the full FP32 form")
    ap.add_argument("--mode", default="per_filter", choices=["per_filter", "joint"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the full FP32 comparison run")
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
    """Algorithmic DRAM bytes (and flops) per stage for one image: every input read once, every output written once."""
    sizes = pyr.sizes
    lam = pyr.lam
    L = len(sizes)
    groups = {}
    for comp in wl.model.components:
        groups.setdefault((0,) + comp.root.shape[:2], []).append(comp.root)
        for p in comp.parts:
            groups.setdefault((1,) + p.filt.shape[:2], []).append(p.filt)
    bf = precision == "bf16"
    fb = 2 if bf else 4
    corr = "corr_tc" if bf else "corr_f32"
    zproj = "zproj_tc" if bf else "zproj_f32"
    out = {corr: [0, 0], zproj: [0, 0], "sep": [0, 0], "dt": [0, 0], "assemble": [0, 0], "to_bf16": [0, 0]}
    if bf:
        out["to_bf16"][0] = sum(H * W * 32 * (4 + 2) for (H, W) in sizes)
    for (role, h, w), fl in groups.items():
        K = len(fl)
        R = (rank * K if not joint else rank) if rank < h * w else h * w * K
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


TENSOR_STAGES = ("corr_tc", "zproj_tc")
ALU_STAGES = ("corr_f32", "zproj_f32", "sep")


def stage_roofline(name, ms_per_image, launches_per_image, model, peaks, sm_mhz):
    """Roofline of one stage: achieved algorithmic throughput against the peak of whichever resource binds it
    (the one whose peak would take longest for the stage's algorithmic bytes or flops)."""
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    src_hbm = "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"
    b, f = model[name]["bytes"], model[name]["flops"]
    s = ms_per_image / 1e3
    t_hbm = b / (hbm * 1e9)
    cand = [("hbm", t_hbm)]
    if name in TENSOR_STAGES:
        tp = float(peaks.get("bf16_tflops", 1900.0))
        cand.append(("tensor", f / (tp * 1e12)))
    elif name in ALU_STAGES:
        cand.append(("alu", f / (fp32_alu_peak_tflops(sm_mhz) * 1e12)))
    bound = max(cand, key=lambda c: c[1])[0]
    out = {"kernel": name, "bound": bound, "launches_per_image": launches_per_image, "ms_per_image": ms_per_image,
           "traffic": None, "algorithmic_bytes_per_image": b, "algorithmic_flops_per_image": f}
    if bound == "hbm":
        out.update(achieved=b / s / 1e9, peak=hbm, unit="GB/s", peak_source=src_hbm)
    elif bound == "tensor":
        tp = float(peaks.get("bf16_tflops", 1900.0))
        out.update(achieved=f / s / 1e12, peak=tp, unit="TFLOP/s",
                   peak_source="MEASURED_PEAKS.json bf16_tflops burst (of measured)" if "bf16_tflops" in peaks
                   else "fallback 1900 TFLOP/s")
    else:
        pk = fp32_alu_peak_tflops(sm_mhz)
        out.update(achieved=f / s / 1e12, peak=pk, unit="TFLOP/s",
                   peak_source="derived: 152 SM x 128 FP32 lanes x 2 flop x median SM clock under load")
    out["frac"] = out["achieved"] / out["peak"]
    return out


# ------------------------------------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as orc
    from paper_1707_03268_gb300 import synth as sy

    wl = sy.config_c2()
    pyr = wl.pyramids[0]
    n_comp = len(wl.model.components)

    def one_step(i):
        # one component of the model over the whole pyramid: 1/6 of an image
        c = i % n_comp
        sub = sy.Model([wl.model.components[c]])
        scored = orc.score_pyramid(sub, pyr)
        orc.detect(scored, load_tau())

    for i in range(args.warmup):
        one_step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        one_step(i)
    dt = time.perf_counter() - t0
    images = args.steps / n_comp
    v = images / dt
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


def cpu_baseline_oracle(wl, budget_s: float = 15.0):
    """The FP64 oracle as it stands, on this host's cores: whole-image full-form scoring, repeated within a budget."""
    from oracle import oracle as orc
    pyr = wl.pyramids[0]
    n = 0
    t0 = time.perf_counter()
    while True:
        orc.detect(orc.score_pyramid(wl.model, pyr), load_tau())
        n += 1
        if time.perf_counter() - t0 >= budget_s or n >= 20:
            break
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "images/s", "cores": orc.num_threads(), "kind": "oracle",
            "sample": f"{n} whole 500x375 images (36 levels, 54 filters), full form, FP64"}


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
    prec = tdpm.PREC_BF16 if args.precision == "bf16" else tdpm.PREC_FP32
    joint = args.mode == "joint"
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

    def step(model_id, f, p):
        sid = tdpm.tdpm_build_pyramid_scores(ctx, model_id, dp, f, p, stream)
        dets = tdpm.tdpm_detect(ctx, sid, tau, capacity=cap, stream=stream, out=det_buf)
        tdpm.tdpm_release(ctx, sid)
        return dets

    def keys(d):
        return set(zip(d["component"].tolist(), d["level"].tolist(), d["y"].tolist(), d["x"].tolist()))

    rep = None
    rank_sweep = None
    chosen_rank = args.rank
    if form == tdpm.FORM_DECOMPOSED:
        dmode = tdpm.DECOMP_JOINT if joint else tdpm.DECOMP_PER_FILTER
        if args.rank > 0:
            rep = tdpm.tdpm_decompose(ctx, mid, args.rank, dmode, max_iters=500, seed=1)
        else:
            # smallest rank whose detections agree >= 99.5% with the full FP32 form (the metric's condition)
            ref_keys = keys(step(mid, tdpm.FORM_FULL, tdpm.PREC_FP32))
            rank_sweep = {}
            for r in RANK_LADDER:
                rep = tdpm.tdpm_decompose(ctx, mid, r, dmode, max_iters=500, seed=1)
                a = keys(step(mid, form, prec))
                rank_sweep[r] = {"agreement": len(a & ref_keys) / max(1, len(a | ref_keys)),
                                 "max_rel_error": rep["max_rel_error"], "mean_rel_error": rep["mean_rel_error"],
                                 "gain_formula_1": rep["gain"]}
                chosen_rank = r
                if rank_sweep[r]["agreement"] >= 0.995:
                    break

    def timed(model_id, f, p, steps, warmup, prof=False):
        for _ in range(warmup):
            step(model_id, f, p)
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
        n_det = 0
        for i in range(steps):
            flush.zero_()  # inputs are smaller than L2: evict them between steps (outside the events)
            ev[i][0].record(stream)
            n_det = len(step(model_id, f, p))
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
        return {"ms": ms, "total_ms": total_ms, "wall_s": wall, "launches": launches, "n_det": n_det,
                "stages": stages}

    # ---- headline run (decomposed BF16 by default)
    clocks = ClockSampler(local)
    clocks.start()
    main_run = timed(mid, form, prec, args.steps, args.warmup)
    clk = clocks.stop()
    value = args.steps * world / (main_run["total_ms"] / 1e3)
    ms_sorted = sorted(main_run["ms"])
    p50 = ms_sorted[len(ms_sorted) // 2]
    p99 = ms_sorted[min(len(ms_sorted) - 1, int(math.ceil(0.99 * len(ms_sorted))) - 1)]

    # ---- per-stage device time (same workload, CUDA events around each stage on its stream)
    prof_run = timed(mid, form, prec, max(10, args.steps // 2), 1, prof=True)
    stages = prof_run["stages"]
    model = stage_bytes(wl, pyr, args.form, args.precision, chosen_rank, joint)
    dom_name, (dom_ms, dom_n) = max(stages.items(), key=lambda kv: kv[1][0])
    roofline = None
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    steps_prof = prof_run_steps(prof_run)
    sm_mhz = (clk or {}).get("sm_mhz") or 1920.0
    rooflines = {name: stage_roofline(name, ms / steps_prof, n / steps_prof, model, peaks, sm_mhz)
                 for name, (ms, n) in stages.items() if name in model}
    roofline = rooflines.get(dom_name)

    # ---- end to end through the public API: pyramid H2D from pinned host memory, detections D2H
    host_levels = [torch.from_numpy(l).pin_memory() for l in pyr.levels]
    h2d = sum(l.numel() * 4 for l in host_levels)

    def e2e_step():
        for hl, dl in zip(host_levels, levels):
            dl.copy_(hl, non_blocking=True)
        return step(mid, form, prec)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
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

    # ---- comparison: full FP32 on the same image, and detection agreement with it
    compare = None
    if not args.no_compare:
        full_run = timed(mid, tdpm.FORM_FULL, tdpm.PREC_FP32, max(10, args.steps // 2), 2)
        d_main = step(mid, form, prec).copy()
        d_full = step(mid, tdpm.FORM_FULL, tdpm.PREC_FP32).copy()
        ka = set(zip(d_main["component"], d_main["level"], d_main["y"], d_main["x"]))
        kb = set(zip(d_full["component"], d_full["level"], d_full["y"], d_full["x"]))
        agree = len(ka & kb) / max(1, len(ka | kb))
        full_ms = sorted(full_run["ms"])
        compare = {"full_fp32_images_per_s": len(full_ms) / (sum(full_ms) / 1e3),
                   "full_fp32_p50_ms": full_ms[len(full_ms) // 2],
                   "agreement_vs_full_fp32": agree, "detections": len(ka), "detections_full_fp32": len(kb)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_oracle(wl)

    line = {"metric": METRIC, "value": value, "unit": "images/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main_run["total_ms"] / args.steps, "p50_ms": p50, "p99_ms": p99,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if prec == tdpm.PREC_BF16 else "f32", "data": "synthetic",
            "config": {"workload": wl.name, "image": "500x375", "levels": len(pyr.levels),
                       "components": len(wl.model.components), "filters": len(wl.model.filters()),
                       "form": args.form, "precision": args.precision,
                       "rank": chosen_rank if form == tdpm.FORM_DECOMPOSED else None,
                       "decomposition": args.mode if form == tdpm.FORM_DECOMPOSED else None,
                       "l2": "flushed between timed steps (256 MB write outside the events)",
                       "parallelism": f"replicas x{world}"},
            "gpu_launches": main_run["launches"], "stages_ms_per_image": {k: v[0] / prof_run_steps(prof_run)
                                                                          for k, v in stages.items()},
            "roofline": roofline, "rooflines": rooflines, "e2e": e2e, "cpu_baseline": cpu, "clocks": clk,
            "compare": compare,
            "decomposition_report": rep, "rank_sweep": rank_sweep, "wall_s_timed": main_run["wall_s"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    tdpm.tdpm_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


def prof_run_steps(run) -> int:
    return len(run["ms"])


if __name__ == "__main__":
    main()
