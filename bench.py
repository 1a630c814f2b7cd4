#!/usr/bin/env python3
"""Throughput of the non-separable lifting 2-D DWT (CDF 9/7) on GB300.

One step is one forward pyramid (5 levels, CDF 9/7, FP32, the non-separable
scheme with reduced operations) over one synthetic 16384 x 16384 FP32 image
already resident in HBM.  The JSON line reports whole-job Gpixel/s (input
pixels per second), the roofline of the level-1 kernel (algorithmic bytes over
its CUDA-event time, against the measured HBM copy bandwidth), the oracle timed
on the host cores, an end-to-end figure through the public API with host
buffers, SM clocks sampled during the run, and a comparison of schemes and
coefficient precisions on the same image.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank transforms its own image (replicas, weak scaling); the
time is the maximum over ranks.  --impl reference times the CPU oracle.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2-D CDF 9/7 DWT Gpixel/s + % HBM peak: non-sep vs separable, FP32 vs FP16"
UNIT = "Gpixel/s"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=16384)
    ap.add_argument("--levels", type=int, default=5)
    ap.add_argument("--scheme", default="reduced", choices=["nonsep", "reduced", "sep", "polyconv", "conv", "nsconv"])
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--profile", action="store_true",
                    help="warm-up and K steps only (for ncu captures); prints a minimal line")
    ap.add_argument("--profile-workload", default="main", choices=["main", "batch512", "grad16x4096"],
                    help="with --profile: the single image (main), the 512-image batch (3 levels; --persistent "
                         "for the one-launch form) or the 16 x 4096^2 forward + L1 adjoint (4 levels)")
    ap.add_argument("--persistent", action="store_true", help="one persistent launch for the whole pyramid")
    ap.add_argument("--grad-images", type=int, default=16,
                    help="with --profile-workload grad16x4096: the number of 4096^2 images (a smaller case for ncu)")
    ap.add_argument("--tune-choice", type=int, default=-1,
                    help="apply this dwt2_autotune choice instead of timing the candidates (ncu captures)")
    return ap.parse_args()


def workload_name(a) -> str:
    return f"CDF 9/7 forward, {a.levels} levels, {a.size}x{a.size} FP32 image, scheme {a.scheme}"


def config_of(a, world):
    return {"workload": workload_name(a), "h": a.size, "w": a.size, "levels": a.levels, "wavelet": "cdf97",
            "scheme": a.scheme, "coef_dtype": "f32", "input": "gradient (0.5*U[0,255] + ramp), seed 2",
            "l2": "inputs larger than L2: 1 GiB read + 1 GiB written per step, no flush",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


# ------------------------------------------------------------------ helpers

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_hash() -> str:
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(ROOT, "paper_1704_08657_gb300", "csrc", "*")))
    for f in files:
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


TUNE_SEGS = (0, 2, 4, 8, 12, 16, 24, 32)  # candidate segment heights of dwt2_autotune
FWD_CFGS = ((2, 3, 3, 4, 0), (2, 2, 4, 4, 0), (2, 2, 4, 8, 0), (2, 2, 4, 8, 1), (2, 2, 4, 4, 1))  # (ql, qr, nst, nw, spec)
TUNE_BITS, TUNE_LEVELS = 6, 5


def tuned_levels(choice, levels, persistent):
    """(ql, qr, nst, nw, seg_rows) of each level from a per-level tuning choice."""
    if persistent or choice is None or choice < 0:
        return []
    out = []
    for lev in range(levels):
        f = (choice >> (TUNE_BITS * min(lev, TUNE_LEVELS - 1))) & ((1 << TUNE_BITS) - 1)
        out.append(FWD_CFGS[f // len(TUNE_SEGS)] + (TUNE_SEGS[f % len(TUNE_SEGS)],))
    return out


def profiled_traffic(h, w, cfg):
    """Per-launch DRAM bytes of the level-1 kernel in configuration cfg
    (ql, qr, nst, nw, spec) from the committed ncu summary, when it was taken
    on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "forward_level1_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("kernel_hash") != kernel_hash():
        return None
    per_px = d.get("dram_bytes_per_pixel", {}).get(",".join(str(int(v)) for v in cfg))
    return None if per_px is None else float(per_px) * h * w


class ClockSampler:
    """nvidia-smi samples (every 100 ms) of SM clock and throttle reasons."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: str):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 10:
                self.rows.append((time.time(), parts))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self, t0, t1):
        rows = [p for (t, p) in self.rows if t0 - 0.15 <= t <= t1 + 0.15]
        if not rows:
            rows = [p for (_, p) in self.rows]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        loaded = [r for r in rows if (num(r[5]) or 0) >= 50] or rows
        sm = [num(r[2]) for r in loaded if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": num(loaded[0][3]), "reasons": reasons, "samples": len(loaded),
                "power_w_max": max((num(r[4]) or 0) for r in loaded)}


def gpu_selector(dev, local: int) -> str:
    """nvidia-smi -i argument for the torch device (its UUID when known)."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(dev).uuid)
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    return vis.split(",")[local] if vis else str(local)


def max_over_ranks(v: float, pg, dev=None) -> float:
    """The largest of every rank's v (the job ends with its slowest rank);
    pg is torch.distributed (any backend) or None for one process."""
    if pg is None:
        return float(v)
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def replica_value(side: int, world: int, ms_step: float) -> float:
    """Whole-job Gpixel/s: every rank transforms its own side x side image per
    step, and a step lasts ms_step (the maximum over ranks)."""
    return side * side * world / (ms_step * 1e-3) / 1e9


def emit(line: dict, rank: int) -> bool:
    """Rank 0 prints the job's one JSON line; the other ranks print nothing."""
    if rank != 0:
        return False
    print(json.dumps(line), flush=True)
    return True


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------ CPU oracle

def time_oracle(size: int, levels: int, budget_s: float, min_runs: int = 1):
    """Oracle forward pyramid on a size x size gradient image; returns
    (pixels per second, runs, seconds, threads)."""
    import numpy as np

    import oracle
    from paper_1704_08657_gb300 import synth
    oracle.build()
    x = synth.gradient(size, size, seed=2).astype(np.float64)
    runs, t = 0, 0.0
    while runs < min_runs or t < budget_s:
        t0 = time.perf_counter()
        oracle.forward97(x, levels)
        t += time.perf_counter() - t0
        runs += 1
        if runs >= 50:
            break
    return size * size * runs / t, runs, t, oracle.threads()


def oracle_sample_side(levels: int, per_step_s: float) -> int:
    """Side of the square sample the oracle transforms in about per_step_s."""
    import numpy as np

    import oracle
    from paper_1704_08657_gb300 import synth
    oracle.build()
    x = synth.gradient(1024, 1024, seed=2).astype(np.float64)
    oracle.forward97(x, levels)
    t0 = time.perf_counter()
    oracle.forward97(x, levels)
    dt = max(time.perf_counter() - t0, 1e-4)
    side = int((per_step_s / dt) ** 0.5 * 1024)
    return max(256, min(16384, side // 64 * 64))


def run_reference(a):
    world, rank, _ = dist_env()
    if rank != 0:
        return  # only rank 0 runs the CPU oracle
    per_step = min(3.0, max(0.05, 150.0 / max(1, a.steps + a.warmup)))
    side = oracle_sample_side(a.levels, per_step)
    import numpy as np

    import oracle
    from paper_1704_08657_gb300 import synth
    x = synth.gradient(side, side, seed=2).astype(np.float64)
    for _ in range(a.warmup):
        oracle.forward97(x, a.levels)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        oracle.forward97(x, a.levels)
    dt = time.perf_counter() - t0
    value = side * side * a.steps / dt / 1e9
    sample = f"oracle (C, FP64 separable lifting) on a {side}x{side} crop-size image of the same recipe, per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(a, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- GPU arm

def run_profile_workload(a):
    """--profile on the batching or differentiation workload: warm-up steps,
    then K timed steps, one short JSON line (for ncu launch lists)."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1704_08657_gb300 import abi, synth
    from paper_1704_08657_gb300.dwt import Plan
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    flags = abi.DWT2_FLAG_PERSISTENT if a.persistent else 0
    if a.profile_workload == "batch512":
        shapes = synth.batch_shapes(512, seed=4)
        buf, descs = synth.batch_pack(shapes, seed=5)
        x = torch.from_numpy(buf).to(dev)
        c = torch.empty_like(x)
        plan = Plan(descs, 3, flags=flags, device=dev)
        px = sum(h * w for h, w in shapes)

        def step():
            plan.forward(x, c, stream)
    else:
        side, nimg = 4096, a.grad_images
        descs = [(i * side * side, side, side, side) for i in range(nimg)]
        x = torch.randint(0, 256, (nimg * side * side,), device=dev,
                          generator=torch.Generator(dev).manual_seed(6)).float()
        c = torch.empty_like(x)
        g = torch.empty_like(x)
        plan = Plan(descs, 4, scheme="reduced", flags=flags, device=dev)
        px = nimg * side * side
        scale = 1.0 / plan.n_detail()

        def step():
            plan.forward(x, c, stream)
            plan.adjoint_l1(c, scale, g, stream)
    tuned = (abi.dwt2_autotune(plan.handle, x.data_ptr(), c.data_ptr(), plan.workspace.data_ptr(),
                               stream.cuda_stream, a.tune_choice) if a.tune_choice >= 0 else plan.autotune(x, c, stream))
    for _ in range(max(3, a.warmup)):
        step()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / a.steps
    print(json.dumps({"mode": "profile", "workload": a.profile_workload, "persistent": bool(a.persistent),
                      "ms_per_step": ms, "gpx_s": px / (ms * 1e-3) / 1e9, "status": plan.status(),
                      "autotuned_choice": tuned}), flush=True)


def run_ours(a):
    import numpy as np
    import torch

    if a.profile and a.profile_workload != "main":
        return run_profile_workload(a)

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_1704_08657_gb300 import abi, synth
    from paper_1704_08657_gb300.dwt import Plan

    n = a.size
    x_host = synth.gradient(n, n, seed=2 + rank)
    x = torch.from_numpy(x_host).to(dev)
    stream = torch.cuda.current_stream(dev)

    def make(scheme, coef_dtype=torch.float32, levels=a.levels, wavelet="cdf97", flags=0):
        return Plan.single(n, n, levels, scheme=scheme, coef_dtype=coef_dtype, wavelet=wavelet, flags=flags,
                           device=dev)

    plan = make(a.scheme, flags=abi.DWT2_FLAG_PERSISTENT if a.persistent else 0)
    coef = torch.empty_like(x)
    ws = plan.workspace
    if a.tune_choice >= 0:
        tuned = abi.dwt2_autotune(plan.handle, x.data_ptr(), coef.data_ptr(), ws.data_ptr(), stream.cuda_stream,
                                  a.tune_choice)
    else:
        tuned = plan.autotune(x, coef)  # untimed: picks the kernel configuration and segment height per level

    def step():
        abi.dwt2_forward(plan.handle, x.data_ptr(), coef.data_ptr(), ws.data_ptr(), stream.cuda_stream)

    def barrier():
        torch.cuda.synchronize(dev)
        if pg is not None:
            pg.barrier()

    # warm-up and clock soak (untimed)
    for _ in range(max(3, a.warmup)):
        step()
    if a.profile:
        torch.cuda.synchronize(dev)
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(a.steps):
            step()
        p1.record(stream)
        torch.cuda.synchronize(dev)
        ms = p0.elapsed_time(p1) / a.steps
        print(json.dumps({"mode": "profile", "workload": workload_name(a), "ms_per_step": ms,
                          "gpx_s": n * n / (ms * 1e-3) / 1e9, "status": plan.status(), "autotuned_choice": tuned,
                          "launches_per_step": 1 if a.persistent else a.levels}), flush=True)
        return
    sampler = ClockSampler(gpu_selector(dev, local))
    sampler.start()
    t_soak = time.time()
    barrier()
    while time.time() - t_soak < 1.0:
        for _ in range(50):
            step()
        torch.cuda.synchronize(dev)

    # timed region: exactly K steps (no per-level events inside it)
    barrier()
    t_wall0 = time.time()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    barrier()
    t_wall1 = time.time()
    ms_total = e0.elapsed_time(e1)
    # then the per-level kernel times from the plan's event pairs (mean over
    # up to 256 further steps)
    abi.dwt2_profile(plan.handle, True)
    for _ in range(max(3, min(a.steps, 256))):
        step()
    levels_ms = abi.dwt2_profile_read(plan.handle, a.levels)
    abi.dwt2_profile(plan.handle, False)
    l1 = levels_ms[0]
    sampler.stop()
    clocks = sampler.summary(t_soak, time.time())
    assert plan.status() == 0, "device status word set during the bench"

    ms_total = max_over_ranks(ms_total, pg, dev)
    ms_step = ms_total / a.steps
    px = n * n * world
    value = replica_value(n, world, ms_step)

    # roofline of the level-1 kernel: 4 B read + 4 B written per pixel
    peak, peak_kind = measured_peaks()
    achieved = 8.0 * n * n / (l1 * 1e-3) / 1e9
    lvl_cfg = tuned_levels(tuned, a.levels, a.persistent)
    ql, qr, nst, nw, spec, seg = lvl_cfg[0] if lvl_cfg else (2, 3, 3, 4, 0, 0)
    kname = (f"pml_kernel<Fwd97<{a.scheme}>, float> (whole pyramid)" if a.persistent else
             f"fwd_tma_kernel<Fwd97<{a.scheme}, {ql}>, float, {ql}, {qr}, {nst}, {nw}, "
             f"{'true' if spec else 'false'}> (level 1)")
    roof = {"bound": "hbm", "kernel": kname,
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": f"{peak_kind} HBM copy bandwidth (burst; the kernel is timed inside the pyramid)",
            "level1_ms": l1, "levels_ms": levels_ms,
            "traffic": profiled_traffic(n, n, (ql, qr, nst, nw, spec)), "algorithmic_bytes": 8 * n * n}

    cfg = config_of(a, world)
    cfg["autotuned_choice"] = tuned
    cfg["per_level_config"] = [{"ql": c[0], "qr": c[1], "nst": c[2], "nw": c[3], "interior_loop": bool(c[4]),
                                "seg_rows": c[5] or "auto"} for c in lvl_cfg]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "roofline": roof, "gpu_launches": a.steps * a.levels, "clocks": clocks}

    # end to end through the public API with host buffers: every step copies
    # its input from pinned host memory, runs dwt2_forward and copies the
    # coefficients back to pinned host memory.  Steps are pipelined over two
    # device buffer sets and three streams (host-to-device, compute,
    # device-to-host), so one step's copies overlap its neighbours' work.
    hin = torch.from_numpy(x_host).pin_memory()
    hout = [torch.empty_like(hin).pin_memory() for _ in range(2)]
    xd = [torch.empty_like(x) for _ in range(2)]
    cd = [torch.empty_like(x) for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("in", "fwd", "out")}

    def e2e_steps(k):
        for i in range(k):
            b = i % 2
            if i >= 2:
                s_in.wait_event(ev["fwd"][b])  # xd[b] free once step i-2 has read it
            with torch.cuda.stream(s_in):
                xd[b].copy_(hin, non_blocking=True)
            ev["in"][b].record(s_in)
            stream.wait_event(ev["in"][b])
            if i >= 2:
                stream.wait_event(ev["out"][b])  # cd[b] free once step i-2 was copied out
            plan.forward(xd[b], cd[b], stream)
            ev["fwd"][b].record(stream)
            s_out.wait_event(ev["fwd"][b])
            with torch.cuda.stream(s_out):
                hout[b].copy_(cd[b], non_blocking=True)
            ev["out"][b].record(s_out)
        stream.wait_stream(s_in)
        stream.wait_stream(s_out)
    e2e_steps(2)
    barrier()
    ee0 = torch.cuda.Event(enable_timing=True)
    ee1 = torch.cuda.Event(enable_timing=True)
    ee0.record(stream)
    s_in.wait_stream(stream)
    e2e_steps(a.e2e_steps)
    ee1.record(stream)
    barrier()
    e2e_ms = ee0.elapsed_time(ee1) / a.e2e_steps
    e2e_ms = max_over_ranks(e2e_ms, pg, dev)
    ok = bool(torch.equal(hout[(a.e2e_steps - 1) % 2], coef.cpu()))

    # the host link of this machine on the same buffers (one direction at a time), for context: the
    # end-to-end figure is bounded by it and it differs between boxes
    def link_gbs(dst, src):
        with torch.cuda.stream(s_in):
            dst.copy_(src, non_blocking=True)
            l0 = torch.cuda.Event(enable_timing=True)
            l1 = torch.cuda.Event(enable_timing=True)
            l0.record(s_in)
            for _ in range(3):
                dst.copy_(src, non_blocking=True)
            l1.record(s_in)
        l1.synchronize()
        return 3 * 4 * n * n / (l0.elapsed_time(l1) * 1e-3) / 1e9
    link = {"h2d_gbs": link_gbs(xd[0], hin), "d2h_gbs": link_gbs(hout[0], cd[0])}
    line["e2e"] = {"value": px / (e2e_ms * 1e-3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": 4 * n * n,
                   "d2h_bytes_per_step": 4 * n * n, "steps": a.e2e_steps, "ms_per_step": e2e_ms,
                   "path": "pinned host -> dwt2_forward -> pinned host, pipelined over 2 buffer sets "
                           "and 3 streams", "result_matches_device_run": ok, "host_link": link}
    del hin, hout, xd, cd

    # every workload of the benchmark's configurations, each with its own
    # roofline fraction (C1 small image, C2 size sweep, C3 precision, C4
    # batching, C5 differentiation)
    if not a.no_compare and world == 1:
        comp = {}
        ctx = Ctx(dev, stream, barrier, peak)
        comp.update(c1_small(ctx))
        comp.update(c2_sweep(ctx, x_host if n == 16384 else None))
        comp.update(c3_precision(ctx))
        comp.update(c4_batch(ctx))
        comp.update(c5_grad(ctx))
        comp.update(f_schemes(ctx, x_host if n == 16384 else None))
        comp.update(inverse_adjoint(ctx, x_host if n == 16384 else None))
        line["compare"] = comp

    if rank == 0 and world == 1 and not a.no_cpu:
        line["cpu_baseline"] = oracle_baseline(a.levels)
    emit(line, rank)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()


# ------------------------------------------------------------ the configurations

class Ctx:
    """Device, stream, barrier and the roofline denominator shared by the
    configuration runners."""

    def __init__(self, dev, stream, barrier, peak):
        import torch
        self.dev, self.stream, self.barrier, self.peak = dev, stream, barrier, peak
        # a buffer of twice the L2 size: writing it evicts earlier data from L2
        self.flush_buf = torch.empty(2 * 129 * 2 ** 20 // 4, dtype=torch.float32, device=dev)

    def flush(self):
        self.flush_buf.zero_()


def alg_bytes(h: int, w: int, levels: int, coef_bytes: int = 4, in_bytes: int = 4) -> int:
    """Algorithmic bytes of a pyramid of per-level launches: every level reads
    its input once (the image, then the FP32/int32 low-low band of the level
    before) and writes its four bands once (intermediate low-low bands in the
    compute type, everything else in the coefficient type)."""
    tot = 0
    for k in range(levels):
        hq, wq = (h + 1) // 2, (w + 1) // 2
        last = k == levels - 1
        tot += h * w * (in_bytes if k == 0 else 4)
        tot += (h * w - hq * wq) * coef_bytes + hq * wq * (coef_bytes if last else 4)
        h, w = hq, wq
    return tot


def _time(fn, steps, stream, barrier):
    import torch
    for _ in range(3):
        fn()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    barrier()
    return e0.elapsed_time(e1) / steps


def _time_flushed(fn, reps, ctx):
    """Median of single calls, each after writing a buffer of twice the L2
    size (the flush is outside the events)."""
    import torch
    for _ in range(3):
        fn()
    ctx.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in ev:
        ctx.flush()
        e0.record(ctx.stream)
        fn()
        e1.record(ctx.stream)
    ctx.barrier()
    return statistics.median(e0.elapsed_time(e1) for e0, e1 in ev)


def level_ms(plan, fn, ctx, n):
    """Mean milliseconds of the first n levels of a plan's calls, from the
    plan's own event pairs (a pass of its own, after the timed loop)."""
    from paper_1704_08657_gb300 import abi
    abi.dwt2_profile(plan.handle, True)
    for _ in range(20):
        fn()
    ctx.barrier()
    ms = abi.dwt2_profile_read(plan.handle, n)
    abi.dwt2_profile(plan.handle, False)
    return ms


def _entry(ctx, px, ms, nbytes, **kw):
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"gpx_s": px / (ms * 1e-3) / 1e9, "ms": ms, "alg_bytes": nbytes, "alg_gbs": gbs,
            "frac": gbs / ctx.peak, **kw}


def c1_small(ctx):
    """512 x 512 uniform FP32 image (seed 1), one level of CDF 9/7, plain
    non-separable lifting: forward, inverse and the pair in microseconds
    (L2-resident, launch-bound), beside the oracle's seconds for the same pair."""
    import numpy as np
    import torch

    import oracle
    from paper_1704_08657_gb300 import synth
    from paper_1704_08657_gb300.dwt import Plan
    n = 512
    xh = synth.uniform(n, n, seed=1)
    x = torch.from_numpy(xh).to(ctx.dev)
    p = Plan.single(n, n, 1, scheme="nonsep", device=ctx.dev)
    c = torch.empty_like(x)
    r = torch.empty_like(x)
    ms_f = _time(lambda: p.forward(x, c, ctx.stream), 200, ctx.stream, ctx.barrier)
    ms_i = _time(lambda: p.inverse(c, r, ctx.stream), 200, ctx.stream, ctx.barrier)

    def pair():
        p.forward(x, c, ctx.stream)
        p.inverse(c, r, ctx.stream)
    ms_p = _time(pair, 200, ctx.stream, ctx.barrier)
    ms_pf = _time_flushed(pair, 50, ctx)
    assert p.status() == 0
    err = float((r - x).abs().max())
    p.close()
    oracle.build()
    x64 = xh.astype(np.float64)
    res = {"oracle_cores": oracle.threads()}
    cores = oracle.threads()
    for thr, key in ((1, "oracle_s_1thread"), (cores, "oracle_s_all_cores")):
        oracle.set_threads(thr)
        runs, t = 0, 0.0
        while runs < 5 or t < 1.0:
            t0 = time.perf_counter()
            oracle.inverse97(oracle.forward97(x64, 1), 1)
            t += time.perf_counter() - t0
            runs += 1
        res[key] = t / runs
    oracle.set_threads(cores)
    return {"C1/512x512/L1/nonsep/f32/forward+inverse": {
        "us_forward": ms_f * 1e3, "us_inverse": ms_i * 1e3, "us_pair": ms_p * 1e3, "us_pair_l2_flushed": ms_pf * 1e3,
        "gpx_s_pair": n * n / (ms_p * 1e-3) / 1e9, "alg_bytes_pair": 2 * alg_bytes(n, n, 1),
        "frac_pair": 2 * alg_bytes(n, n, 1) / (ms_p * 1e-3) / 1e9 / ctx.peak,
        "reconstruction_max_err": err, **res,
        "note": "1 MiB image: L2-resident and launch-bound, frac is against HBM only for scale"}}


def c2_sweep(ctx, x16384=None):
    """One FP32 gradient image (seed 2) at 2048^2, 8192^2 and 16384^2, 1 and 5
    levels, non-separable, reduced and separable lifting (FP32, and FP16
    coefficients at 16384^2), plus integer 5/3 on round(x) by non-separable
    and separable lifting; each plan autotuned.  2048^2 (16 MiB) fits in L2:
    it is reported L2-flushed (a 2 x L2 write before every call) and warm."""
    import torch

    from paper_1704_08657_gb300 import synth
    from paper_1704_08657_gb300.dwt import Plan
    out = {}
    for n in (2048, 8192, 16384):
        xh = x16384 if (n == 16384 and x16384 is not None) else synth.gradient(n, n, seed=2)
        x = torch.from_numpy(xh).to(ctx.dev)
        xi = torch.from_numpy(synth.to_int(xh)).to(ctx.dev)
        steps = 400 if n == 2048 else (100 if n == 8192 else 40)
        variants = [("cdf97", s, torch.float32) for s in ("nonsep", "reduced", "sep")]
        if n == 16384:
            variants += [("cdf97", "reduced", torch.float16), ("cdf97", "sep", torch.float16)]
        variants += [("cdf53", s, torch.int32) for s in ("nonsep", "sep")]
        for wav, scheme, cdt in variants:
            for levels in (1, 5):
                src = xi if wav == "cdf53" else x
                p = Plan.single(n, n, levels, wavelet=wav, scheme=scheme, coef_dtype=cdt, device=ctx.dev)
                c = torch.empty_like(src, dtype=cdt)
                tuned = p.autotune(src, c, ctx.stream)
                cb = 2 if cdt in (torch.float16, torch.bfloat16) else 4
                nb = alg_bytes(n, n, levels, cb)
                key = f"C2/{n}x{n}/L{levels}/{'cdf53i' if wav == 'cdf53' else 'cdf97'}/{scheme}/" \
                      f"{ {torch.float32: 'f32', torch.float16: 'f16', torch.int32: 'i32'}[cdt]}"
                if n == 2048:
                    ms_w = _time(lambda: p.forward(src, c, ctx.stream), steps, ctx.stream, ctx.barrier)
                    ms_f = _time_flushed(lambda: p.forward(src, c, ctx.stream), 100, ctx)
                    out[key] = _entry(ctx, n * n, ms_f, nb, l2="flushed before every call", autotuned_choice=tuned,
                                      warm=_entry(ctx, n * n, ms_w, nb, l2="warm, back to back"))
                else:
                    ms = _time(lambda: p.forward(src, c, ctx.stream), steps, ctx.stream, ctx.barrier)
                    l1 = level_ms(p, lambda: p.forward(src, c, ctx.stream), ctx, 1)[0]
                    out[key] = _entry(ctx, n * n, ms, nb, l2="inputs larger than L2, back to back",
                                      level1_ms=l1, level1_frac=alg_bytes(n, n, 1, cb) / (l1 * 1e-3) / 1e9 / ctx.peak,
                                      autotuned_choice=tuned,
                                      per_level_config=[dict(zip(("ql", "qr", "nst", "nw", "interior_loop", "seg_rows"),
                                                                 c_)) for c_ in tuned_levels(tuned, levels, False)])
                assert p.status() == 0
                p.close()
                del c
        del x, xi
    return out


def c3_precision(ctx):
    """8192^2 image u + N(0, 10^2) (seed 3, unclipped), 5-level CDF 9/7 with
    FP16 and BF16 coefficient storage and FP32 lifting: throughput and, per
    subband, the max abs error and the max relative error (max |q - ref| /
    max |ref band|) against the FP64 oracle; the integer 5/3 path on
    round(clip(x, 0, 255)) compared bit for bit."""
    import numpy as np
    import torch

    import oracle
    from paper_1704_08657_gb300 import synth
    from paper_1704_08657_gb300.dwt import Plan, band_slices
    n, levels = 8192, 5
    xh = synth.noisy(n, n, seed=3)
    ref = oracle.forward97(xh.astype(np.float64), levels)
    x = torch.from_numpy(xh).to(ctx.dev)
    out = {}
    for scheme in ("reduced", "sep"):
        for cdt, name in ((torch.float16, "f16"), (torch.bfloat16, "bf16"), (torch.float32, "f32")):
            p = Plan.single(n, n, levels, scheme=scheme, coef_dtype=cdt, device=ctx.dev)
            c = torch.empty_like(x, dtype=cdt)
            p.autotune(x, c, ctx.stream)
            ms = _time(lambda: p.forward(x, c, ctx.stream), 100, ctx.stream, ctx.barrier)
            p.forward(x, c, ctx.stream)
            assert p.status() == 0
            got = c.float().cpu().numpy()
            bands = []
            for lev, bn, rs, cs in band_slices(n, n, levels):
                g, r = got[rs, cs].astype(np.float64), ref[rs, cs]
                e = float(np.abs(g - r).max())
                m = float(np.abs(r).max())
                bands.append({"level": lev, "band": bn, "max_abs": e, "max_rel": e / max(m, 1e-30), "band_max": m})
            worst = max(b["max_rel"] for b in bands)
            bound = {"f16": 1e-3, "bf16": 8e-3}.get(name)
            out[f"C3/8192x8192/L5/cdf97/{scheme}/{name}"] = _entry(
                ctx, n * n, ms, alg_bytes(n, n, levels, 2 if name != "f32" else 4), bands=bands,
                worst_rel=worst, rel_bound=bound, within_bound=(worst <= bound) if bound else None)
            p.close()
            del c
    xi = synth.to_int(xh, clip=True)
    refi = oracle.forward53i(xi.astype(np.int64), levels)
    xid = torch.from_numpy(xi).to(ctx.dev)
    for scheme in ("nonsep", "sep"):
        p = Plan.single(n, n, levels, wavelet="cdf53", scheme=scheme, coef_dtype=torch.int32, device=ctx.dev)
        c = torch.empty_like(xid)
        p.autotune(xid, c, ctx.stream)
        ms = _time(lambda: p.forward(xid, c, ctx.stream), 100, ctx.stream, ctx.barrier)
        p.forward(xid, c, ctx.stream)
        assert p.status() == 0
        same = bool(np.array_equal(c.cpu().numpy().astype(np.int64), refi))
        out[f"C3/8192x8192/L5/cdf53i/{scheme}/i32"] = _entry(ctx, n * n, ms, alg_bytes(n, n, levels), bit_exact=same)
        p.close()
    return out


def c4_batch(ctx):
    """512 images, sides log-uniform in [64, 2048] rounded to even (seed 4),
    uniform pixels (seed 5), 3-level CDF 9/7 forward: one persistent launch in
    a CUDA graph, grouped launches (eager and in a graph), and one launch per
    image and level (eager and in a graph)."""
    import torch

    from paper_1704_08657_gb300 import abi, synth
    from paper_1704_08657_gb300.dwt import Plan
    out = {}
    shapes = synth.batch_shapes(512, seed=4)
    buf, descs = synth.batch_pack(shapes, seed=5)
    px = sum(h * w for h, w in shapes)
    nb = sum(alg_bytes(h, w, 3) for h, w in shapes)
    xb = torch.from_numpy(buf).to(ctx.dev)
    cb = torch.empty_like(xb)

    def graph_of(fn):
        fn()  # launch blocks built for these buffers outside the capture
        ctx.barrier()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(ctx.dev)
        s.wait_stream(ctx.stream)
        with torch.cuda.graph(g, stream=s):
            fn(s)
        return g

    grp = Plan(descs, 3, device=ctx.dev)
    choice_g = grp.autotune(xb, cb, ctx.stream)
    ms = _time(lambda: grp.forward(xb, cb, ctx.stream), 20, ctx.stream, ctx.barrier)
    out["C4/batch512/L3/grouped"] = _entry(ctx, px, ms, nb, pixels=px, autotuned_choice=choice_g,
                                           launches=3 * ((len(shapes) + 75) // 76))
    g = graph_of(lambda s=None: grp.forward(xb, cb, s or ctx.stream))
    ms = _time(lambda: g.replay(), 50, ctx.stream, ctx.barrier)
    out["C4/batch512/L3/grouped_graph"] = _entry(ctx, px, ms, nb)
    assert grp.status() == 0
    del g
    grp.close()
    per = Plan(descs, 3, flags=abi.DWT2_FLAG_PERSISTENT, device=ctx.dev)
    choice_p = per.autotune(xb, cb, ctx.stream)
    g = graph_of(lambda s=None: per.forward(xb, cb, s or ctx.stream))
    ms = _time(lambda: g.replay(), 50, ctx.stream, ctx.barrier)
    out["C4/batch512/L3/persistent_graph"] = _entry(ctx, px, ms, nb, autotuned_choice=choice_p, launches=1)
    assert per.status() == 0
    del g
    per.close()
    # one plan per image: one launch per image and level
    plans = [Plan([(0, h, w, p)], 3, device=ctx.dev) for (o, h, w, p) in descs]
    xp = xb.data_ptr()
    cp = cb.data_ptr()

    def each(s=None):
        st = (s or ctx.stream).cuda_stream
        for pl, (o, h, w, p) in zip(plans, descs):
            abi.dwt2_forward(pl.handle, xp + 4 * o, cp + 4 * o, pl.workspace.data_ptr(), st)
    ms = _time(each, 5, ctx.stream, ctx.barrier)
    out["C4/batch512/L3/one_launch_per_image"] = _entry(ctx, px, ms, nb, launches=3 * len(shapes))
    g = graph_of(each)
    ms = _time(lambda: g.replay(), 20, ctx.stream, ctx.barrier)
    out["C4/batch512/L3/one_launch_per_image_graph"] = _entry(ctx, px, ms, nb, launches=3 * len(shapes))
    for pl in plans:
        assert pl.status() == 0
        pl.close()
    del g, xb, cb
    return out


def c5_grad(ctx):
    """16 x 4096^2 uniform FP32 images (seed 6), 4-level CDF 9/7 forward and
    the hand-written adjoint of the mean-L1 loss over the detail bands."""
    import torch

    from paper_1704_08657_gb300 import abi
    from paper_1704_08657_gb300.dwt import Plan
    out = {}
    side, nimg, levels = 4096, 16, 4
    descs = [(i * side * side, side, side, side) for i in range(nimg)]
    x = torch.randint(0, 256, (nimg * side * side,), device=ctx.dev,
                      generator=torch.Generator(ctx.dev).manual_seed(6)).float()
    cbuf = torch.empty_like(x)
    gin = torch.empty_like(x)
    npx = nimg * side * side
    nb_f = nimg * alg_bytes(side, side, levels)
    for name, flags in (("grouped_forward", 0), ("persistent_forward", abi.DWT2_FLAG_PERSISTENT)):
        pl = Plan(descs, levels, scheme="reduced", flags=flags, device=ctx.dev)
        pl.autotune(x, cbuf, ctx.stream)
        scale = 1.0 / pl.n_detail()

        def fwd_bwd():
            pl.forward(x, cbuf, ctx.stream)
            pl.adjoint_l1(cbuf, scale, gin, ctx.stream)
        ms = _time(fwd_bwd, 20, ctx.stream, ctx.barrier)
        ms_f = _time(lambda: pl.forward(x, cbuf, ctx.stream), 20, ctx.stream, ctx.barrier)
        ms_a = _time(lambda: pl.adjoint_l1(cbuf, scale, gin, ctx.stream), 20, ctx.stream, ctx.barrier)
        assert pl.status() == 0
        out[f"C5/grad16x4096/L4/{name}+adjoint_l1"] = _entry(
            ctx, npx, ms, 2 * nb_f, forward_ms=ms_f, adjoint_ms=ms_a,
            forward_frac=nb_f / (ms_f * 1e-3) / 1e9 / ctx.peak, adjoint_frac=nb_f / (ms_a * 1e-3) / 1e9 / ctx.peak)
        pl.close()
    return out


def f_schemes(ctx, x16384=None):
    """The paper's other schemes and its third wavelet on the 16384^2 bench
    image, 1 and 5 levels, FP32: polyconvolution, separable and non-separable
    convolution (CDF 9/7), and DD 13/7 by non-separable, reduced and separable
    lifting; each plan autotuned."""
    import torch

    from paper_1704_08657_gb300 import synth
    from paper_1704_08657_gb300.dwt import Plan
    n = 16384
    x = torch.from_numpy(x16384 if x16384 is not None else synth.gradient(n, n, seed=2)).to(ctx.dev)
    out = {}
    for wav, scheme in [("cdf97", "polyconv"), ("cdf97", "conv"), ("cdf97", "nsconv"), ("dd137", "nonsep"),
                        ("dd137", "reduced"), ("dd137", "sep")]:
        for levels in (1, 5):
            p = Plan.single(n, n, levels, wavelet=wav, scheme=scheme, device=ctx.dev)
            c = torch.empty_like(x)
            tuned = p.autotune(x, c, ctx.stream)
            ms = _time(lambda: p.forward(x, c, ctx.stream), 40, ctx.stream, ctx.barrier)
            l1 = level_ms(p, lambda: p.forward(x, c, ctx.stream), ctx, 1)[0]
            assert p.status() == 0
            out[f"F/{n}x{n}/L{levels}/{wav}/{scheme}/f32"] = _entry(
                ctx, n * n, ms, alg_bytes(n, n, levels), level1_ms=l1,
                level1_frac=alg_bytes(n, n, 1) / (l1 * 1e-3) / 1e9 / ctx.peak, autotuned_choice=tuned)
            p.close()
            del c
    return out


def inverse_adjoint(ctx, x16384=None):
    """The inverse and the adjoint of the 16384^2 bench image's pyramid (FP32
    coefficients of the reduced scheme), 1 and 5 levels: 4 B read + 4 B written
    per pixel and level, like the forward."""
    import torch

    from paper_1704_08657_gb300 import synth
    from paper_1704_08657_gb300.dwt import Plan
    n = 16384
    x = torch.from_numpy(x16384 if x16384 is not None else synth.gradient(n, n, seed=2)).to(ctx.dev)
    out = {}
    for levels in (1, 5):
        p = Plan.single(n, n, levels, scheme="reduced", device=ctx.dev)
        coef = p.forward(x, None, ctx.stream)
        back = torch.empty_like(x)
        for name, fn in (("inverse", lambda: p.inverse(coef, back, ctx.stream)),
                         ("adjoint", lambda: p.adjoint(coef, back, ctx.stream))):
            ms = _time(fn, 40, ctx.stream, ctx.barrier)
            l1 = level_ms(p, fn, ctx, 1)[0]
            out[f"I/{n}x{n}/L{levels}/cdf97/{name}/f32"] = _entry(
                ctx, n * n, ms, alg_bytes(n, n, levels), level1_ms=l1,
                level1_frac=alg_bytes(n, n, 1) / (l1 * 1e-3) / 1e9 / ctx.peak)
        assert p.status() == 0
        p.close()
        del coef, back
    return out


def oracle_baseline(levels: int):
    """The oracle on a 4096^2 image of the bench recipe, with OpenMP on all
    host cores and single-threaded."""
    import oracle
    per_s, runs, secs, threads = time_oracle(4096, levels, budget_s=8.0)
    prev = oracle.threads()
    oracle.set_threads(1)
    per_1, runs1, secs1, _ = time_oracle(4096, levels, budget_s=6.0)
    oracle.set_threads(prev)
    return {"value": per_s / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "single_thread_value": per_1 / 1e9,
            "sample": f"oracle (C, FP64 separable lifting, gcc -O3, OpenMP on {threads} threads) on a 4096x4096 "
                      f"image of the bench recipe, {levels} levels, {runs} runs in {secs:.1f} s; single-threaded "
                      f"{runs1} runs in {secs1:.1f} s"}


def main():
    a = parse_args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
