"""Throughput of the space-variant box-spline filter on one GB300 (or N replicas).

Workload (the filter's space-variant benchmark): one 2048 x 2048 float32 blob
image (200 Gaussian blobs, sigma 5-60 px, amplitude U[0,1], plus N(0, 0.05^2)
noise, seed 0); N = 4 directions, order n = 2 (81 taps); per-pixel covariance
with sigma rising 1 -> 16 px across x, theta = pi (0.5 + 0.5 sin(2 pi y / H)),
anisotropy 1 -> 4 along the diagonal; symmetric extension; uint64 fixed-point
running sums; float32 output.

A step is one whole forward pass through the C ABI (bsf_filter): per-pixel
step solve, extension + quantisation + running sums along d1, d3, d2, d4, and
the 81-tap finite differences.  Inputs are resident in HBM; L2 is flushed
(a 256 MB write) before every timed step and each step is timed with CUDA
events on the launch stream.  The e2e figure times the same call with the
image and covariance copied from pinned host memory and the output copied
back, inside the timed region.

The default line also carries the batching workload (64 images of uneven
sizes, key batch64) and the differentiation workload (8 x 1024^2, continuous
steps, image and field gradients, key diff8x1024), a few steps each, and the
CPU baseline: the oracle on all host cores (row bands with their halos) and
on one core, and the direct definition on sampled pixels.

--impl reference times the CPU oracle (oracle.modular, the running-sum
pipeline in exact integer arithmetic) on all host cores over the same
workload.

Prints one JSON line.  Under torchrun (N > 1) every rank filters its own
replica (no data exchange: the single-image path does not shard here) and
rank 0 reports the whole-job aggregate over the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Mpixel/s fwd and fwd+bwd vs plain FP64 GPU form at stated error; % of HBM peak"
UNIT = "Mpixel/s"
H = W = 2048
ORDER = 2
WORKLOAD = ("space-variant filter: 2048x2048 fp32 blob image, N=4, n=2 (81 taps), "
            "per-pixel covariance field (sigma 1-16 px across x, theta(y), anisotropy 1-4 "
            "along the diagonal), symmetric extension, uint64 fixed-point running sums, fp32 out")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def make_inputs():
    import workloads as wl
    img = wl.blob_image(H, W, seed=0)
    cov = wl.diagonal_ramp_cov_field(H, W)
    return img, cov


class ClockSampler:
    """nvidia-smi samples (every 20 ms, timestamped) of the SM clock and the
    throttle reasons; summary() keeps the samples taken inside the timed
    regions recorded with mark(), or, when a region is shorter than the
    sampling interval, the samples within 0.5 s around them."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.regions = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.5)  # let the sampler start before the first timed region
        except OSError:
            self.proc = None
        return self

    def mark(self, t0: float, t1: float):
        """Record a timed region (host wall-clock seconds)."""
        self.regions.append((t0, t1))

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        import datetime
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[1]), float(parts[2]),
                             {nm for nm, v in zip(names, parts[5:9]) if v.lower().startswith("active")}))
            except ValueError:
                continue

        def pick(slack):
            return [r for r in rows if any(t0 - slack <= r[0] <= t1 + slack for t0, t1 in self.regions)]

        sel, window = pick(0.0), "inside the timed regions"
        if len(sel) < 3:
            sel, window = pick(0.5), "within 0.5 s of the timed regions"
        reasons = set()
        for r in sel:
            reasons |= r[3]
        return {"sm_mhz": statistics.median(r[1] for r in sel) if sel else None,
                "sm_max_mhz": sel[-1][2] if sel else None, "reasons": sorted(reasons),
                "samples": len(sel), "window": window}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def init_group(world: int):
    """NCCL process group of the replicas (once; nested runs reuse it)."""
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl")


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_gpu(args):
    import torch
    from paper_1109_5114_gb300 import bsf

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    init_group(world)
    img, cov = make_inputs()
    vmax = float(np.abs(img).max())
    d_img = torch.from_numpy(img).cuda()
    d_cov = torch.from_numpy(cov).cuda()
    d_out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    f = bsf.BoxSplineFilter(H, W, ORDER, "symmetric", precision=1, frac_bits=-1, value_bound=vmax)
    f.set_option(bsf.BSF_OPT_SCAN_MODE, bsf.BSF_SCAN_THREE_PHASE)
    kernels_per_vscan = 2  # the three-phase scheme: reduction, then the rescan that folds the carries
    info = f.plan(d_cov)
    stream = torch.cuda.current_stream()

    def step():
        f.filter(d_img, d_cov, out=d_out)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    rc = f.status()
    if rc != 0:
        raise RuntimeError(f"device status {rc}: {bsf.bsf_last_error(f.handle).decode()}")
    info = f.info()

    # ---- per-phase times (a separate, untimed pass: the event records
    # between the phases would otherwise sit inside the timed steps) ------
    f.set_profiling(True)
    f.read_profile()
    for _ in range(args.steps):
        flush.zero_()
        step()
    prof = f.read_profile()
    f.set_profiling(False)

    # ---- device-resident timed region -------------------------------------
    clk = ClockSampler(local).__enter__()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.time()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    clk.mark(t0, time.time())
    barrier(world)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = max_over_ranks(sum(step_ms), world)
    rc = f.status()
    if rc != 0:
        raise RuntimeError(f"device status {rc}")

    # ---- the plain float64 GPU form: float64 running sums, same kernels ---
    f64 = bsf.BoxSplineFilter(H, W, ORDER, "symmetric", precision=bsf.BSF_F64ACC, frac_bits=-1,
                              max_reach=info.R)
    d_out64 = torch.empty_like(d_out)
    for _ in range(args.warmup):
        flush.zero_()
        f64.filter(d_img, d_cov, out=d_out64)
    torch.cuda.synchronize()
    fs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    fe = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    t0 = time.time()
    for i in range(args.steps):
        flush.zero_()
        fs[i].record(stream)
        f64.filter(d_img, d_cov, out=d_out64)
        fe[i].record(stream)
    torch.cuda.synchronize()
    clk.mark(t0, time.time())
    barrier(world)
    f64_ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(fs, fe)), world)
    ref = d_out.double()
    err64 = (d_out64.double() - ref).abs()
    scale = float(ref.abs().max())
    fp64_form = {"ms_per_step": round(f64_ms / args.steps, 5),
                 "max_abs_err": float(err64.max()), "max_err_rel_to_max_out": float(err64.max()) / scale,
                 "fixed_point_error": "exact integer sums and one final rounding: within 3 float32 "
                                      "ulp of the exact value, bit-exact against the CPU oracle"}
    f64.close()

    # ---- Algorithm 1: the isotropic pass, then the residual pass ------------
    # (bsf_filter_two_pass: the condition-2 minimum and the field split on
    # the device, then two filters through a float32 intermediate image)
    tp = bsf.BoxSplineFilter(H, W, ORDER, "symmetric", precision=1, frac_bits=-1, value_bound=vmax)
    tp.set_option(bsf.BSF_OPT_SCAN_MODE, bsf.BSF_SCAN_THREE_PHASE)
    d_out2 = torch.empty_like(d_out)
    _, sigma2 = tp.filter_two_pass(d_img, d_cov, 0.5, out=d_out2, want_sigma2=True)
    for _ in range(args.warmup):
        flush.zero_()
        tp.filter_two_pass(d_img, d_cov, 0.5, out=d_out2)
    torch.cuda.synchronize()
    ts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    te = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    t0 = time.time()
    for i in range(args.steps):
        flush.zero_()
        ts[i].record(stream)
        tp.filter_two_pass(d_img, d_cov, 0.5, out=d_out2)
        te[i].record(stream)
    torch.cuda.synchronize()
    clk.mark(t0, time.time())
    barrier(world)
    tp_ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(ts, te)), world)
    rc = tp.status()
    if rc != 0:
        raise RuntimeError(f"device status {rc} (two passes)")
    algorithm1 = {"ms_per_step": round(tp_ms / args.steps, 5), "sigma2": sigma2, "frac": 0.5,
                  "R": tp.info().R, "passes": 2}
    tp.close()

    # ---- the second direction set (Algorithm 3) and the pair (Algorithm 2) --
    # same workload; each its own context (plan, running sums, stencil)
    def time_dirs(directions):
        g = bsf.BoxSplineFilter(H, W, ORDER, "symmetric", precision=1, frac_bits=-1, value_bound=vmax,
                                directions=directions)
        g.set_option(bsf.BSF_OPT_SCAN_MODE, bsf.BSF_SCAN_THREE_PHASE)
        o = torch.empty_like(d_out)
        g.plan(d_cov)
        for _ in range(args.warmup):
            flush.zero_()
            g.filter(d_img, d_cov, out=o)
        torch.cuda.synchronize()
        g.set_profiling(True)
        g.read_profile()
        for _ in range(args.steps):
            flush.zero_()
            g.filter(d_img, d_cov, out=o)
        pr = g.read_profile()
        g.set_profiling(False)
        es = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ee = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        barrier(world)
        t0 = time.time()
        for i in range(args.steps):
            flush.zero_()
            es[i].record(stream)
            g.filter(d_img, d_cov, out=o)
            ee[i].record(stream)
        torch.cuda.synchronize()
        clk.mark(t0, time.time())
        barrier(world)
        ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(es, ee)), world)
        if g.status() != 0:
            raise RuntimeError(f"device status (directions {directions})")
        gi = g.info()
        g.close()
        return {"ms_per_step": round(ms / args.steps, 5), "R": gi.R, "clamped_px": gi.clamp_count,
                "phases_ms": {k: round(v / max(c, 1), 5) for k, (v, c) in pr.items() if c}}, ms

    second, second_ms = time_dirs(bsf.BSF_DIRS_SECOND)
    pair, pair_ms = time_dirs(bsf.BSF_DIRS_PAIR)

    # ---- the sampled continuous box spline (order 1, the paper's mesh) -----
    gs = bsf.BoxSplineFilter(H, W, 1, "symmetric", precision=1, frac_bits=-1, value_bound=vmax,
                             step_rule=bsf.BSF_STEP_SAMPLED)
    gs.set_option(bsf.BSF_OPT_SCAN_MODE, bsf.BSF_SCAN_THREE_PHASE)
    o_s = torch.empty_like(d_out)
    gs.plan(d_cov)
    for _ in range(args.warmup):
        flush.zero_()
        gs.filter(d_img, d_cov, out=o_s)
    torch.cuda.synchronize()
    gs.set_profiling(True)
    gs.read_profile()
    for _ in range(args.steps):
        flush.zero_()
        gs.filter(d_img, d_cov, out=o_s)
    pr_s = gs.read_profile()
    gs.set_profiling(False)
    es = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ee = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    t0 = time.time()
    for i in range(args.steps):
        flush.zero_()
        es[i].record(stream)
        gs.filter(d_img, d_cov, out=o_s)
        ee[i].record(stream)
    torch.cuda.synchronize()
    clk.mark(t0, time.time())
    barrier(world)
    ms_s = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(es, ee)), world)
    if gs.status() != 0:
        raise RuntimeError("device status (sampled box spline)")
    sampled = {"ms_per_step": round(ms_s / args.steps, 5), "n": 1, "R": gs.info().R,
               "frac_bits": gs.info().frac_bits,
               "value": round(world * H * W * args.steps / (ms_s * 1e-3) / 1e6, 2), "unit": UNIT,
               "phases_ms": {k: round(v / max(c, 1), 5) for k, (v, c) in pr_s.items() if c}}
    gs.close()

    # ---- 8-bit image, small kernels: what 32-bit running sums buy ---------
    # (the blob image as uint8, sigma 1..3 px, rho 1..3, n = 2: the bound
    # 255 x max prod L^n stays below 2^31, so BSF_FIX takes 32 bits), and
    # what the fused tiles buy against the global passes
    import workloads as wl
    u8 = torch.from_numpy(wl.blob_image_u8(H, W, seed=0)).cuda()
    cov_s = torch.from_numpy(wl.diagonal_ramp_cov_field(H, W, sigma_hi=3.0, rho_hi=3.0)).cuda()
    small = {"workload": f"{H}x{W} uint8 blob image, sigma 1-3 px, rho 1-3, n={ORDER}"}
    outs = {}
    for name, prec, tiles in (("fix_auto", bsf.BSF_FIX, 1), ("fix_auto_global_passes", bsf.BSF_FIX, 0),
                              ("fix64", bsf.BSF_FIX64, 1), ("fix64_global_passes", bsf.BSF_FIX64, 0)):
        g = bsf.BoxSplineFilter(H, W, ORDER, "symmetric", precision=prec, frac_bits=-1)
        g.set_option(bsf.BSF_OPT_SCAN_MODE, bsf.BSF_SCAN_THREE_PHASE)
        g.set_option(bsf.BSF_OPT_TILES, tiles)
        o = torch.empty((H, W), dtype=torch.float32, device="cuda")
        g.plan(cov_s)
        for _ in range(args.warmup):
            flush.zero_()
            g.filter(u8, cov_s, out=o)
        torch.cuda.synchronize()
        es = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ee = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        barrier(world)
        t0 = time.time()
        for i in range(args.steps):
            flush.zero_()
            es[i].record(stream)
            g.filter(u8, cov_s, out=o)
            ee[i].record(stream)
        torch.cuda.synchronize()
        clk.mark(t0, time.time())
        barrier(world)
        ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(es, ee)), world)
        if g.status() != 0:
            raise RuntimeError(f"device status ({name})")
        gi = g.info()
        small[name] = {"ms_per_step": round(ms / args.steps, 5), "elem_bytes": gi.elem_bytes,
                       "frac_bits": gi.frac_bits,
                       "value": round(world * H * W * args.steps / (ms * 1e-3) / 1e6, 2), "unit": UNIT}
        outs[name] = o
        g.close()
    # both are exact integer pipelines; they differ only where q differs
    small["max_abs_diff"] = float((outs["fix_auto"] - outs["fix64"]).abs().max())

    # ---- forward + backward (image gradient of <out, gout>) ---------------
    gen = torch.Generator(device="cuda").manual_seed(0)
    d_gout = torch.randn((H, W), generator=gen, device="cuda", dtype=torch.float32)
    d_gimg = torch.empty_like(d_gout)
    for _ in range(args.warmup):
        flush.zero_()
        step()
        f.backward(d_gout, d_cov, gimg=d_gimg)
    torch.cuda.synchronize()
    f.set_profiling(True)
    f.read_profile()
    for _ in range(args.steps):
        flush.zero_()
        step()
        f.backward(d_gout, d_cov, gimg=d_gimg)
    prof_fb = f.read_profile()
    f.set_profiling(False)
    bs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    be = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    t0 = time.time()
    for i in range(args.steps):
        flush.zero_()
        bs[i].record(stream)
        step()
        f.backward(d_gout, d_cov, gimg=d_gimg)
        be[i].record(stream)
    torch.cuda.synchronize()
    clk.mark(t0, time.time())
    barrier(world)
    fb_ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(bs, be)), world)
    rc = f.status()
    if rc != 0:
        raise RuntimeError(f"device status {rc} (backward)")

    # ---- end to end through the public API with host buffers --------------
    # bsf_filter_host: pinned host image and field in, pinned host output
    # back, transfers overlapped with the work; synchronous, so it is timed
    # on the host clock around the steps
    h_img = torch.from_numpy(img).pin_memory()
    h_cov = torch.from_numpy(cov).pin_memory()
    h_out = torch.empty((H, W), dtype=torch.float32).pin_memory()

    def e2e_step():
        f.filter_host(h_img, h_cov, h_out)

    for _ in range(max(1, args.warmup)):
        flush.zero_()
        e2e_step()
    torch.cuda.synchronize()
    barrier(world)
    e2e_ms = 0.0
    t_start = time.time()
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    clk.mark(t_start, time.time())
    clk.__exit__(None, None, None)
    barrier(world)
    e2e_ms = max_over_ranks(e2e_ms, world)
    h2d = img.nbytes + cov.nbytes
    d2h = H * W * 4
    gpu_out = d_out.cpu().numpy()
    assert np.array_equal(h_out.numpy(), gpu_out)  # same result both ways
    f.close()

    # the host link's own floor for the same bytes: the uploads and the
    # download as plain copies (one stream each way, overlapped), no filter
    # work; the e2e figure is compared with it
    d_img_l = torch.empty(h_img.shape, dtype=h_img.dtype, device="cuda")
    d_cov_l = torch.empty(h_cov.shape, dtype=h_cov.dtype, device="cuda")
    h_out_l = torch.empty((H, W), dtype=torch.float32).pin_memory()
    up, down = torch.cuda.Stream(), torch.cuda.Stream()

    def link_step():
        with torch.cuda.stream(up):
            d_img_l.copy_(h_img, non_blocking=True)
            d_cov_l.copy_(h_cov, non_blocking=True)
        with torch.cuda.stream(down):
            h_out_l.copy_(d_out, non_blocking=True)
        torch.cuda.synchronize()

    for _ in range(2):
        link_step()
    link_ms = 0.0
    for _ in range(5):
        t0 = time.perf_counter()
        link_step()
        link_ms += (time.perf_counter() - t0) * 1e3
    link_ms /= 5
    del d_img_l, d_cov_l

    # ---- the batching and differentiation workloads, a few steps each ------
    sub = argparse.Namespace(**vars(args))
    sub.steps, sub.warmup = min(args.steps, 10), 3
    batch_line = run_batch(sub)
    diff_line = run_diff(sub)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return None

    px = H * W
    value = world * px * args.steps / (total_ms * 1e-3) / 1e6
    fp64_form["value"] = round(world * px * args.steps / (f64_ms * 1e-3) / 1e6, 2)
    fp64_form["unit"] = UNIT
    # an accuracy comparison: at the float64 form's error no speed ratio
    # at equal accuracy exists, so only its time is reported beside it
    fp64_form["comparison"] = ("accuracy: the float64 running sums lose the output's digits "
                               "(max_abs_err) while the fixed-point sums are exact; not a speed-up")
    algorithm1["value"] = round(world * px * args.steps / (tp_ms * 1e-3) / 1e6, 2)
    algorithm1["unit"] = UNIT
    for d, ms in ((second, second_ms), (pair, pair_ms)):
        d["value"] = round(world * px * args.steps / (ms * 1e-3) / 1e6, 2)
        d["unit"] = UNIT
    fb_value = world * px * args.steps / (fb_ms * 1e-3) / 1e6
    e2e_value = world * px * args.steps / (e2e_ms * 1e-3) / 1e6

    # ---- roofline of the dominant kernel ------------------------------------
    per_phase = {k: (ms / max(c, 1), c) for k, (ms, c) in prof.items()}
    dominant = max(per_phase, key=lambda k: per_phase[k][0] * per_phase[k][1])
    elem = info.elem_bytes
    Sbytes = info.Hp * info.Wp * elem
    alg = {
        # S read once (the taps of neighbouring pixels overlap), covariance in
        # (the step solve is fused into the stencil), output out
        "stencil": Sbytes + px * 12 + px * 4,
        "steps": px * 12 + px * 8,
        "rows": px * 4 + Sbytes,
        "d3": 2 * Sbytes, "d2": 2 * Sbytes, "d4": 2 * Sbytes,
    }
    # our kernels per timed step: steps (only when planning), rows, two kernels
    # per vertical direction and the stencil (the phase counts come from the
    # profiled pass, which runs as many steps as the timed one)
    launches = sum(c for k, (ms, c) in prof.items() if k in ("steps", "rows", "stencil"))
    launches += sum(c * kernels_per_vscan for k, (ms, c) in prof.items() if k in ("d3", "d2", "d4"))
    hbm_peak, peak_src = peaks()
    dom_ms = per_phase[dominant][0]
    achieved = alg[dominant] / (dom_ms * 1e-3) / 1e9
    traffic = None  # ncu DRAM bytes of one launch, valid while the kernel's sources are unchanged
    tfile = os.path.join(ROOT, "profiles", "traffic_stencil_spacevariant_2048_n2.txt")
    if dominant in KERNEL_SOURCES and os.path.exists(tfile):
        ent = {}
        with open(tfile) as fh:
            for line in fh:
                if "=" in line and not line.lstrip().startswith("#"):
                    k, v = line.split("=", 1)
                    ent[k.strip()] = v.strip()
        if ent.get("kernel") == dominant and ent.get("kernel_rev") == kernel_revision(dominant):
            traffic = int(ent["bytes_per_launch"])

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(info.frac_bits, info.R, world,
                                  "flushed before every timed step (256 MB write)"),
        "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms / args.steps, 5),
                "link_floor_ms": round(link_ms, 5),
                "link_floor_note": "the same uploads and download as plain overlapped copies, no work",
                "frac_of_link_floor": round(link_ms / (e2e_ms / args.steps), 3)},
        "gpu_launches": launches,
        "fp64_form": fp64_form,
        "algorithm1": algorithm1,
        "algorithm3_second_set": second,
        "algorithm2_pair": pair,
        "u8_small_kernels": small,
        "sampled_box_spline": sampled,
        "fwd_bwd": {"value": round(fb_value, 2), "unit": UNIT,
                    "ms_per_step": round(fb_ms / args.steps, 5),
                    "phases_ms": {k: round(ms / max(c, 1), 5) for k, (ms, c) in prof_fb.items() if c}},
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": round(achieved, 1),
                     "peak": hbm_peak, "peak_source": peak_src, "unit": "GB/s",
                     "frac": round(achieved / hbm_peak, 4), "traffic": traffic,
                     "algorithmic_bytes_per_launch": alg[dominant]},
        "phases_ms": {k: round(v[0], 5) for k, v in per_phase.items()},
        "clocks": clocks,
        "batch64": {k: batch_line[k] for k in ("value", "unit", "ms_per_step", "steps", "config", "modes",
                                                "gpu_launches_per_step")},
        "diff8x1024": {"fwd_bwd": {k: diff_line[k] for k in ("value", "unit", "ms_per_step", "phases_ms")},
                       "fwd": diff_line["fwd"], "steps": diff_line["steps"], "config": diff_line["config"],
                       "loss": diff_line["loss"], "clocks": diff_line["clocks"]},
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(img, cov, info.R, info.frac_bits, rows=args.cpu_rows,
                                            gpu_out=gpu_out)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line


KERNEL_SOURCES = {
    "stencil": ["bsf_stencil.cu", "bsf_stencil.cuh", "bsf_solve.cuh", "bsf_device.cuh", "bsf_internal.h"],
    "stencil_d2": ["bsf_continuous.cuh", "bsf_continuous128.cu", "bsf_solve.cuh", "bsf_device.cuh",
                   "bsf_internal.h"],
}


def kernel_revision(kernel: str = "stencil") -> str:
    """Hash of the code that builds one kernel (its sources with their
    comments and spacing removed, and the build script with its flags), to
    tell whether stored ncu traffic still applies to it."""
    import hashlib
    import re
    hsh = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_1109_5114_gb300", "csrc")
    for fn in KERNEL_SOURCES[kernel] + ["../../include/bsf.h"]:
        with open(os.path.join(cs, fn)) as fh:
            code = re.sub(r"/\*.*?\*/", " ", fh.read(), flags=re.S)
        code = " ".join(re.sub(r"//[^\n]*", " ", code).split())
        hsh.update(os.path.basename(fn).encode() + code.encode())
    with open(os.path.join(cs, "..", "build.py"), "rb") as fh:
        hsh.update(b"build.py" + fh.read())
    return hsh.hexdigest()[:16]


def host_cores() -> int:
    return len(os.sched_getaffinity(0))


def _oracle_band(job):
    """One process's share of the all-cores oracle run: rows [y0, y1) of the
    workload from the band [y0 - R, y1 + R) (clipped to the image), whose
    running sums restart above it; the rows it returns are exact (every tap
    of a band pixel lies in the padded band)."""
    y0, y1, R, q = job
    from oracle import modular
    img, cov = _WORKER_INPUTS
    a0, a1 = max(0, y0 - R), min(H, y1 + R)
    out = modular.filter_modular(np.ascontiguousarray(img[a0:a1]), np.ascontiguousarray(cov[:, a0:a1]),
                                 ORDER, 2, q=q, bits=64, out_dtype=np.float32, R=R)
    return y0, out[y0 - a0:y1 - a0]


class OraclePool:
    """The oracle's running-sum pipeline on all host cores, one process per
    core (spawned: the workers start fresh interpreters, no CUDA state),
    each filtering a band of rows with its R-row halos."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        self.cores = cores or host_cores()
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_init_worker)

    def run(self, rows: int, R: int, q: int):
        """Filter image rows [0, rows) split into one band per core; returns
        (output rows, seconds)."""
        per = -(-rows // self.cores)
        jobs = [(y, min(rows, y + per), R, q) for y in range(0, rows, per)]
        t0 = time.perf_counter()
        parts = self.pool.map(_oracle_band, jobs)
        dt = time.perf_counter() - t0
        parts.sort(key=lambda p: p[0])
        return np.concatenate([p[1] for p in parts]), dt

    def close(self):
        self.pool.close()
        self.pool.join()


_WORKER_INPUTS = None


def _init_worker():
    """Once per worker process, outside the timed runs: one thread for numpy,
    the oracle imported, the workload generated."""
    global _WORKER_INPUTS
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    import oracle  # noqa: F401
    _WORKER_INPUTS = make_inputs()


def cpu_baseline(img, cov, R, q, rows: int = 512, gpu_out=None):
    """The oracle timed on the host: its running-sum pipeline (oracle.modular)
    on all cores by row bands over the whole image, and on one core on a band
    of `rows` rows; the definition (oracle.kernels.correlate_f64, the direct
    correlation) on a seeded sample of pixels, extrapolated."""
    from oracle import kernels, modular, params
    pool = OraclePool()
    pool.run(H, R, q)                      # warm-up: the workers' start-up is not timed
    full, dt_all = pool.run(H, R, q)
    pool.close()
    if gpu_out is not None:   # the oracle's whole image is the GPU's, bit for bit
        assert np.array_equal(full, gpu_out)
    band_img = np.ascontiguousarray(img[:rows])
    band_cov = np.ascontiguousarray(cov[:, :rows])
    t0 = time.perf_counter()
    modular.filter_modular(band_img, band_cov, ORDER, 2, q=q, bits=64, out_dtype=np.float32, R=R)
    dt1 = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    pix = sorted({(int(y), int(x)) for y, x in zip(rng.integers(0, H, 400), rng.integers(0, W, 400))})
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], ORDER)
    t0 = time.perf_counter()
    kernels.correlate_f64(img.astype(np.float64), L, ORDER, 2, pixels=pix)
    dtd = time.perf_counter() - t0
    return {"value": round(H * W / dt_all / 1e6, 4), "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": f"the whole 2048x2048 workload, oracle.modular (numpy) in {pool.cores} spawned "
                      f"processes, one band of rows each with its R-row halos, {dt_all:.2f} s "
                      f"(os.sched_getaffinity: {pool.cores} cores)"
                      + ("; equal to the GPU output bit for bit" if gpu_out is not None else ""),
            "one_core": {"value": round(rows * W / dt1 / 1e6, 4), "unit": UNIT, "cores": 1,
                         "sample": f"rows 0-{rows - 1} ({rows}x{W} px), oracle.modular, one process, "
                                   f"{dt1:.1f} s"},
            "direct_definition": {"value": round(len(pix) / dtd / 1e6, 6), "unit": UNIT, "cores": 1,
                                  "sample": f"{len(pix)} seeded pixels of the workload, "
                                            f"oracle.kernels.correlate_f64 (the direct correlation "
                                            f"with each pixel's kernel), {dtd:.1f} s, extrapolated "
                                            "per pixel"}}


# the fraction bits the GPU arm's automatic rule picks on this workload (its
# value bound and the steps of its field); the reference arm quantises alike
REF_FRAC_BITS = 24


def workload_config(frac_bits: int, R: int, world: int, l2: str) -> dict:
    return {"workload": WORKLOAD, "H": H, "W": W, "n": ORDER, "N": 4, "boundary": "symmetric",
            "precision": "fix64", "frac_bits": frac_bits, "R": R, "l2": l2,
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return None
    img, cov = make_inputs()
    from oracle import config
    R = config.padding(cov, ORDER)
    q = REF_FRAC_BITS
    rows = args.ref_rows if args.ref_rows > 0 else H
    pool = OraclePool()
    for _ in range(args.warmup):
        pool.run(rows, R, q)
    dt = 0.0
    for _ in range(args.steps):
        dt += pool.run(rows, R, q)[1]
    pool.close()
    value = rows * W * args.steps / dt / 1e6
    sample = (f"rows 0-{rows - 1} of the 2048x2048 workload ({rows}x{W} px) per step, oracle.modular in "
              f"{pool.cores} spawned processes (one band of rows each, with R-row halos)")
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(q, R, 1, "not applicable (host cores)"),
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


BATCH_WORKLOAD = ("batch: 64 fp32 blob images, sides log-uniform in [128, 2048] (H and W "
                  "independent, seed 1), each with its own smooth random covariance field "
                  "(sigma 1-24 px, rho 1-3, random orientation), N=4, n=2, uint64 running sums")


def run_batch(args):
    """Batched form of 64 images: the whole batch as one persistent launch
    replayed from a CUDA graph (the headline, its parameters autotuned on the
    batch), against one launch per phase over the batch (direct and
    graph-replayed), the persistent launch without a graph, and the same
    kernels launched image by image."""
    import torch
    import workloads as wl
    from paper_1109_5114_gb300 import bsf

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    init_group(world)
    sizes = wl.batch_sizes_loguniform(64, seed=1, lo=128, hi=2048)
    imgs, covs = [], []
    for i, (h, w) in enumerate(sizes):
        imgs.append(torch.from_numpy(wl.blob_image(h, w, seed=1000 + i)).cuda())
        covs.append(torch.from_numpy(wl.random_cov_field(h, w, seed=2000 + 3 * i,
                                                         sigma_range=(1.0, 24.0),
                                                         rho_range=(1.0, 3.0))).cuda())
    outs = [torch.empty_like(im) for im in imgs]
    vmax = max(float(im.abs().max()) for im in imgs)
    px = sum(h * w for h, w in sizes)
    bf = bsf.BatchFilter(ORDER, "symmetric", frac_bits=-1, value_bound=vmax)
    torch.cuda.synchronize()
    info = bf.plan(imgs, covs, outs, autotune=True)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    bstream = bf.stream()
    results = {}
    P = bsf.BSF_BATCH_PERSISTENT
    for name, flags in [("per_image", bsf.BSF_BATCH_PER_IMAGE), ("batched", 0),
                        ("graph", bsf.BSF_BATCH_GRAPH), ("persistent", P),
                        ("persistent_graph", P | bsf.BSF_BATCH_GRAPH)]:
        for _ in range(args.warmup):
            bf.run(flags)
        assert bf.status() == 0
        total = 0.0
        for _ in range(args.steps):
            with torch.cuda.stream(bstream):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(bstream)
            bf.run(flags)
            with torch.cuda.stream(bstream):
                e1.record(bstream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        assert bf.status() == 0
        total = max_over_ranks(total, world)
        results[name] = {"ms_per_step": round(total / args.steps, 4),
                         "value": round(world * px * args.steps / (total * 1e-3) / 1e6, 2)}
    info = bf.info()
    bf.close()
    if rank != 0:
        return None
    g = results["persistent_graph"]
    return {
        "metric": METRIC, "value": g["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": g["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "images": len(sizes), "pixels": px, "n": ORDER,
                   "frac_bits": info.frac_bits, "scan_chunk_by_class": list(info.scan_chunk),
                   "persistent": {"work_items": info.persist_items, "blocks": info.persist_grid,
                                  "image_groups": info.persist_groups,
                                  "rows_per_item": info.rows_per_item,
                                  "stencil_tile": f"32x{info.stencil_tile_rows}",
                                  "tuned": "coordinate descent over chunk heights, item shapes and "
                                           "blocks per SM, timing the batch itself"},
                   "arena_bytes": info.arena_bytes,
                   "l2": "flushed before every timed step (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "modes": results,
        "gpu_launches_per_step": {"per_image": 8 * len(sizes), "batched": 8, "graph": 8,
                                  "persistent": 1, "persistent_graph": 1},
    }


DIFF_WORKLOAD = ("differentiation: 8 fp32 blob images of 1024x1024 (seeds 0-7), smooth fields "
                 "log sigma in [0, 3], theta in [0, pi), log rho in [0, 1.1] per image (fp32, "
                 "requiring grad); target = filter(img, fields + smooth perturbation of amplitude "
                 "0.1 per field, seed 1); loss = 1/2 ||out - target||^2, gradients with respect to "
                 "the image and the three fields; continuous steps (D2), n=2, 625 samples per "
                 "pixel, uint128 running sums and adjoint sums, symmetric extension")


def diff_inputs(B=8, side=1024):
    import workloads as wl
    imgs, fields, targets_fields = [], [], []
    for i in range(B):
        imgs.append(wl.blob_image(side, side, seed=i))
        fl = wl.param_fields_logsig_theta_logrho(side, side, seed=100 + 3 * i,
                                                 logsig_range=(0.0, 3.0), logrho_range=(0.0, 1.1))
        pert = np.stack([wl.smooth_field(side, side, seed=1 + 10 * i + j, lo=-0.1, hi=0.1)
                         for j in range(3)]).astype(np.float32)
        fields.append(fl)
        targets_fields.append(np.ascontiguousarray(fl + pert, dtype=np.float32))
    return imgs, fields, targets_fields


def run_diff(args):
    """Forward with the covariance Jacobian and the parameter gradient of an L2
    loss (continuous steps), image by image through one context."""
    import torch
    from paper_1109_5114_gb300 import bsf

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    init_group(world)
    side = 1024
    imgs, fields, tfields = diff_inputs(8, side)
    vmax = max(float(np.abs(im).max()) for im in imgs)
    d_imgs = [torch.from_numpy(im).cuda() for im in imgs]
    d_fields = [torch.from_numpy(fl).cuda() for fl in fields]
    f = bsf.BoxSplineFilter(side, side, ORDER, "symmetric", precision=bsf.BSF_FIX128, frac_bits=-1,
                            value_bound=vmax, step_rule=bsf.BSF_STEP_D2,
                            cov_kind=bsf.BSF_COV_LOGSIG_THETA_LOGRHO)
    f.set_option(bsf.BSF_OPT_PLAN_UNION, 1)
    d_tfields = [torch.from_numpy(fl).cuda() for fl in tfields]
    for fl in d_fields + d_tfields:
        f.plan(fl)
    # targets: the filter at the perturbed fields (input preparation, untimed)
    targets = [f.filter(im, tf).clone() for im, tf in zip(d_imgs, d_tfields)]
    del d_tfields
    outs = [torch.empty((side, side), dtype=torch.float32, device="cuda") for _ in range(8)]
    jacs = [torch.empty((3, side, side), dtype=torch.float32, device="cuda") for _ in range(8)]
    grads = [torch.empty((3, side, side), dtype=torch.float32, device="cuda") for _ in range(8)]
    gimgs = [torch.empty((side, side), dtype=torch.float32, device="cuda") for _ in range(8)]
    gouts = [torch.empty((side, side), dtype=torch.float32, device="cuda") for _ in range(8)]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def fwd_bwd():
        for i in range(8):
            f.filter_jacobian(d_imgs[i], d_fields[i], out=outs[i], jac=jacs[i])
            torch.sub(outs[i], targets[i], out=gouts[i])          # d loss / d out
            f.jacobian_vjp(gouts[i], jacs[i], gcov=grads[i])      # d loss / d fields
            f.backward(gouts[i], d_fields[i], gimg=gimgs[i], want_gimg=True)  # d loss / d image

    def fwd():
        for i in range(8):
            f.filter(d_imgs[i], d_fields[i], out=outs[i])

    clk = ClockSampler(local)

    def timed(fn, prof=False):
        for _ in range(args.warmup):
            flush.zero_()
            fn()
        torch.cuda.synchronize()
        rc = f.status()
        if rc != 0:
            raise RuntimeError(f"device status {rc}: {bsf.bsf_last_error(f.handle).decode()}")
        p = None
        if prof:  # per-phase times from a separate, untimed pass
            f.set_profiling(True)
            f.read_profile()
            for _ in range(args.steps):
                flush.zero_()
                fn()
            p = f.read_profile()
            f.set_profiling(False)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        barrier(world)
        t0 = time.time()
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        clk.mark(t0, time.time())
        barrier(world)
        return max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world), p

    with clk:
        fb_ms, prof_fb = timed(fwd_bwd, prof=True)
        fw_ms, prof_fw = timed(fwd, prof=True)
    info = f.info()
    loss = sum(float(0.5 * ((o - t) ** 2).sum()) for o, t in zip(outs, targets))
    f.close()
    if rank != 0:
        return None
    px = 8 * side * side
    per_phase = {k: (ms / max(c, 1), c) for k, (ms, c) in prof_fb.items() if c}
    clocks = clk.summary()
    return {
        "metric": "Mpixel/s fwd+bwd (image and parameter gradients) of the differentiation workload",
        "value": round(world * px * args.steps / (fb_ms * 1e-3) / 1e6, 2), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(fb_ms / args.steps, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u128", "data": "synthetic",
        "config": {"workload": DIFF_WORKLOAD, "images": 8, "H": side, "W": side, "n": ORDER,
                   "R": info.R, "frac_bits": info.frac_bits, "max_mass": info.max_mass,
                   "l2": "flushed before every timed step (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "fwd": {"value": round(world * px * args.steps / (fw_ms * 1e-3) / 1e6, 2), "unit": UNIT,
                "ms_per_step": round(fw_ms / args.steps, 4),
                "phases_ms": {k: round(ms / max(c, 1), 5) for k, (ms, c) in prof_fw.items() if c}},
        "phases_ms": {k: round(v[0], 5) for k, v in per_phase.items()},
        # over the timed steps, per image: rows, 3 x (agg + apply), stencil,
        # vjp; backward: absmax, scatter, 3 x (agg + apply), suffix rows, the
        # fused extension fold
        "gpu_launches": args.steps * 8 * ((1 + 3 * 2 + 1 + 1) + (1 + 1 + 3 * 2 + 1 + 1)),
        "loss": loss,
        "clocks": clocks,
    }


def run_single(args):
    """One filter configuration on its own (few launches, for profiling and
    for its own throughput): tiles4096 (8-bit 4096^2 blob image, sigma 1-3 px,
    rho 1-3, n = 2, automatic width, fused tiles), sampled2048 (the benchmark's
    image and field, n = 1, the sampled continuous box spline), sampledsecond2048
    (the same with the second direction set: Algorithm 3 as printed), pair2048 (the
    benchmark's image and field, n = 2, both direction sets switched by
    sector)."""
    import torch
    import workloads as wl
    from paper_1109_5114_gb300 import bsf

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    init_group(world)
    if args.workload == "tiles4096":
        h = w = 4096
        img = torch.from_numpy(wl.blob_image_u8(h, w, seed=0)).cuda()
        cov = torch.from_numpy(wl.diagonal_ramp_cov_field(h, w, sigma_hi=3.0, rho_hi=3.0)).cuda()
        f = bsf.BoxSplineFilter(h, w, 2, "symmetric", precision=bsf.BSF_FIX, frac_bits=-1)
        desc = "4096x4096 uint8 blob image, sigma 1-3 px, rho 1-3, n=2, automatic width, fused tiles"
    else:
        h, w = H, W
        im, cv = make_inputs()
        img, cov = torch.from_numpy(im).cuda(), torch.from_numpy(cv).cuda()
        vmax = float(np.abs(im).max())
        if args.workload == "sampled2048":
            f = bsf.BoxSplineFilter(h, w, 1, "symmetric", frac_bits=-1, value_bound=vmax,
                                    step_rule=bsf.BSF_STEP_SAMPLED)
            desc = WORKLOAD.replace("n=2 (81 taps)", "n=1") + "; sampled continuous box spline"
        elif args.workload == "sampledsecond2048":
            f = bsf.BoxSplineFilter(h, w, 1, "symmetric", frac_bits=-1, value_bound=vmax,
                                    step_rule=bsf.BSF_STEP_SAMPLED, directions=bsf.BSF_DIRS_SECOND)
            desc = WORKLOAD.replace("n=2 (81 taps)", "n=1") + "; the second set's sampled box spline (Algorithm 3)"
        else:
            f = bsf.BoxSplineFilter(h, w, 2, "symmetric", frac_bits=-1, value_bound=vmax,
                                    directions=bsf.BSF_DIRS_PAIR)
            desc = WORKLOAD + "; both direction sets, switched per pixel"
    f.set_option(bsf.BSF_OPT_SCAN_MODE, bsf.BSF_SCAN_THREE_PHASE)
    f.plan(cov)
    out = torch.empty((h, w), dtype=torch.float32, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        flush.zero_()
        f.filter(img, cov, out=out)
    torch.cuda.synchronize()
    clk = ClockSampler(local).__enter__()
    es = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ee = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    t0 = time.time()
    for i in range(args.steps):
        flush.zero_()
        es[i].record(stream)
        f.filter(img, cov, out=out)
        ee[i].record(stream)
    torch.cuda.synchronize()
    clk.mark(t0, time.time())
    clk.__exit__(None, None, None)
    barrier(world)
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(es, ee)), world)
    if f.status() != 0:
        raise RuntimeError("device status")
    info = f.info()
    f.close()
    if rank != 0:
        return None
    return {"metric": METRIC, "value": round(world * h * w * args.steps / (ms * 1e-3) / 1e6, 2), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms / args.steps, 5), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": f"u{8 * info.elem_bytes}", "data": "synthetic",
            "config": {"workload": desc, "H": h, "W": w, "R": info.R, "frac_bits": info.frac_bits,
                       "l2": "flushed before every timed step (256 MB write)",
                       "parallelism": f"replicas x{world}"},
            "clocks": clk.summary()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="bsf", choices=["bsf", "reference"])
    ap.add_argument("--cpu-rows", type=int, default=1536,
                    help="rows of the workload the cpu_baseline leg filters (one pass)")
    ap.add_argument("--ref-rows", type=int, default=0,
                    help="rows of the workload each --impl reference step filters (0: all)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="spacevariant2048",
                    choices=["spacevariant2048", "batch64", "diff8x1024", "tiles4096", "sampled2048",
                             "sampledsecond2048", "pair2048"],
                    help="spacevariant2048: the benchmark line; batch64: the batched form; "
                         "diff8x1024: continuous steps with the parameter gradient; "
                         "tiles4096, sampled2048, sampledsecond2048, pair2048: one configuration each "
                         "(run_single)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "bsf":
        args.warmup = 3
    if args.impl == "reference":
        line = run_reference(args)
    elif args.workload == "batch64":
        line = run_batch(args)
    elif args.workload == "diff8x1024":
        line = run_diff(args)
    elif args.workload in ("tiles4096", "sampled2048", "sampledsecond2048", "pair2048"):
        line = run_single(args)
    else:
        line = run_gpu(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
