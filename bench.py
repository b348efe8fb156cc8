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

--impl reference times the CPU oracle (oracle.modular, the running-sum
pipeline in exact integer arithmetic) on a bounded band of the same workload.

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
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


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


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_gpu(args):
    import torch
    from paper_1109_5114_gb300 import bsf

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    img, cov = make_inputs()
    vmax = float(np.abs(img).max())
    d_img = torch.from_numpy(img).cuda()
    d_cov = torch.from_numpy(cov).cuda()
    d_out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    f = bsf.BoxSplineFilter(H, W, ORDER, "symmetric", precision=1, frac_bits=-1, value_bound=vmax)
    f.set_option(bsf.BSF_OPT_SCAN_MODE, bsf.BSF_SCAN_THREE_PHASE)
    kernels_per_vscan = 3
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

    # ---- device-resident timed region -------------------------------------
    f.set_profiling(True)
    f.read_profile()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            step()
            ends[i].record(stream)
        torch.cuda.synchronize()
    barrier(world)
    prof = f.read_profile()
    f.set_profiling(False)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = max_over_ranks(sum(step_ms), world)
    rc = f.status()
    if rc != 0:
        raise RuntimeError(f"device status {rc}")

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
    bs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    be = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    for i in range(args.steps):
        flush.zero_()
        bs[i].record(stream)
        step()
        f.backward(d_gout, d_cov, gimg=d_gimg)
        be[i].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    prof_fb = f.read_profile()
    f.set_profiling(False)
    fb_ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(bs, be)), world)
    rc = f.status()
    if rc != 0:
        raise RuntimeError(f"device status {rc} (backward)")

    # ---- end to end through the public API with host buffers --------------
    h_img = torch.from_numpy(img).pin_memory()
    h_cov = torch.from_numpy(cov).pin_memory()
    h_out = torch.empty((H, W), dtype=torch.float32).pin_memory()
    e_img = torch.empty_like(d_img)
    e_cov = torch.empty_like(d_cov)
    e_out = torch.empty_like(d_out)

    def e2e_step():
        e_img.copy_(h_img, non_blocking=True)
        e_cov.copy_(h_cov, non_blocking=True)
        f.filter(e_img, e_cov, out=e_out)
        h_out.copy_(e_out, non_blocking=True)

    for _ in range(max(1, args.warmup)):
        flush.zero_()
        e2e_step()
    torch.cuda.synchronize()
    es = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ee = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    for i in range(args.steps):
        flush.zero_()
        es[i].record(stream)
        e2e_step()
        ee[i].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    e2e_ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(es, ee)), world)
    h2d = img.nbytes + cov.nbytes
    d2h = H * W * 4
    assert np.array_equal(h_out.numpy(), d_out.cpu().numpy())  # same result both ways
    f.close()

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return None

    px = H * W
    value = world * px * args.steps / (total_ms * 1e-3) / 1e6
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
    # our kernels per timed step: steps (only when planning), rows, one kernel
    # per vertical direction (look-back) and the stencil
    launches = sum(c for k, (ms, c) in prof.items() if k in ("steps", "rows", "stencil"))
    launches += sum(c * kernels_per_vscan for k, (ms, c) in prof.items() if k in ("d3", "d2", "d4"))
    hbm_peak, peak_src = peaks()
    dom_ms = per_phase[dominant][0]
    achieved = alg[dominant] / (dom_ms * 1e-3) / 1e9
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        with open(tfile) as fh:
            tj = json.load(fh)
        ent = tj.get(dominant)
        if ent and ent.get("kernel_rev") == kernel_revision():
            traffic = ent.get("bytes_per_launch")

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": H, "W": W, "n": ORDER, "N": 4,
                   "boundary": "symmetric", "precision": "fix64", "frac_bits": info.frac_bits,
                   "R": info.R, "l2": "flushed before every timed step (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "fwd_bwd": {"value": round(fb_value, 2), "unit": UNIT,
                    "ms_per_step": round(fb_ms / args.steps, 5),
                    "phases_ms": {k: round(ms / max(c, 1), 5) for k, (ms, c) in prof_fb.items() if c}},
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": round(achieved, 1),
                     "peak": hbm_peak, "peak_source": peak_src, "unit": "GB/s",
                     "frac": round(achieved / hbm_peak, 4), "traffic": traffic,
                     "algorithmic_bytes_per_launch": alg[dominant]},
        "phases_ms": {k: round(v[0], 5) for k, v in per_phase.items()},
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                   "reasons": clocks["reasons"]},
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(img, cov, info.R, info.frac_bits, rows=args.cpu_rows)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line


def kernel_revision() -> str:
    """Hash of the CUDA sources, to tell whether stored ncu traffic still applies."""
    import hashlib
    hsh = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_1109_5114_gb300", "csrc")
    for fn in sorted(os.listdir(cs)):
        with open(os.path.join(cs, fn), "rb") as fh:
            hsh.update(fn.encode() + fh.read())
    return hsh.hexdigest()[:16]


def cpu_baseline(img, cov, R, q, rows: int = 512):
    """The oracle's running-sum pipeline on a band of `rows` rows of the workload."""
    from oracle import modular
    band_img = np.ascontiguousarray(img[:rows])
    band_cov = np.ascontiguousarray(cov[:, :rows])
    t0 = time.perf_counter()
    modular.filter_modular(band_img, band_cov, ORDER, 2, q=q, bits=64, out_dtype=np.float32, R=R)
    dt = time.perf_counter() - t0
    return {"value": round(rows * W / dt / 1e6, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"rows 0-{rows - 1} of the 2048x2048 workload ({rows}x{W} px), "
                      f"oracle.modular (numpy, one thread), {dt:.1f} s"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return None
    img, cov = make_inputs()
    from oracle import modular, params
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], ORDER)
    R = max(int(params.reach(L, ORDER).max()), 3 * ORDER)
    q = 22
    rows = args.ref_rows
    band_img = np.ascontiguousarray(img[:rows])
    band_cov = np.ascontiguousarray(cov[:, :rows])
    for _ in range(args.warmup):
        modular.filter_modular(band_img, band_cov, ORDER, 2, q=q, bits=64, out_dtype=np.float32, R=R)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        modular.filter_modular(band_img, band_cov, ORDER, 2, q=q, bits=64, out_dtype=np.float32, R=R)
    dt = time.perf_counter() - t0
    value = rows * W * args.steps / dt / 1e6
    sample = f"rows 0-{rows - 1} of the 2048x2048 workload ({rows}x{W} px) per step"
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": H, "W": W, "n": ORDER, "sample_rows": rows},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


BATCH_WORKLOAD = ("batch: 64 fp32 blob images, sides log-uniform in [128, 2048] (H and W "
                  "independent, seed 1), each with its own smooth random covariance field "
                  "(sigma 1-24 px, rho 1-3, random orientation), N=4, n=2, uint64 running sums")


def run_batch(args):
    """Batched form: one launch per phase over 64 images, replayed from a CUDA
    graph, against the same kernels launched image by image."""
    import torch
    import workloads as wl
    from paper_1109_5114_gb300 import bsf

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
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
    for name, flags in [("per_image", bsf.BSF_BATCH_PER_IMAGE), ("batched", 0),
                        ("graph", bsf.BSF_BATCH_GRAPH)]:
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
    bf.close()
    if rank != 0:
        return None
    g = results["graph"]
    return {
        "metric": METRIC, "value": g["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": g["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "images": len(sizes), "pixels": px, "n": ORDER,
                   "frac_bits": info.frac_bits, "scan_chunk_by_class": list(info.scan_chunk),
                   "arena_bytes": info.arena_bytes,
                   "l2": "flushed before every timed step (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "modes": results,
        "gpu_launches_per_step": {"per_image": 8 * len(sizes), "batched": 8, "graph": 1},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="bsf", choices=["bsf", "reference"])
    ap.add_argument("--cpu-rows", type=int, default=1536,
                    help="rows of the workload the cpu_baseline leg filters (one pass)")
    ap.add_argument("--ref-rows", type=int, default=256,
                    help="rows of the workload each --impl reference step filters")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="spacevariant2048", choices=["spacevariant2048", "batch64"],
                    help="spacevariant2048: the benchmark line; batch64: the batched form")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "bsf":
        args.warmup = 3
    if args.impl == "reference":
        line = run_reference(args)
    elif args.workload == "batch64":
        line = run_batch(args)
    else:
        line = run_gpu(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
