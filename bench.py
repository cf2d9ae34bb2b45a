"""Benchmark: MAR-DEAM iterations/s on the full-size 3D helical workload.

Workload: 512x512x64 voxels (0.98 x 0.98 x 0.75 mm) per basis component, 16-row
x 816-channel curved detector, 1160 views/rotation x 5 rotations (5800 views),
pitch 0.6, two spectra x 120 one-keV bins, bilateral stainless-steel hip inserts
(dense metal trace), Poisson I0 = 1e5 plus Gaussian electronic noise sigma = 5.
Synthetic seeded data (no scanner data offline).

One step = one MAR-DEAM iteration: forward projection + fused spectral sums,
metal substitution, p-step ratio and objective; objective reduction; gather
backprojection fused with the c-step.  value = iterations/s with the data
resident in HBM; e2e = the same through the C ABI with host buffers (data,
mask and image copied in, image and objective copied out, every step).

--impl reference times the FP64 CPU oracle (the reference arm of this build) on
a bounded view sample of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DEAM iterations/s"
UNIT = "it/s"
WORKLOAD = ("3D helical MAR-DEAM, 512x512x64 voxels x 2 components (0.98x0.98x0.75 mm), "
            "16x816 curved detector, 5800 views (1160/rot x 5, pitch 0.6), 2 spectra x 120 bins, "
            "bilateral steel hips, I0=1e5 + sigma 5")
FP32_LANES_PER_SM = 128
# Algorithmic on-chip bytes per Joseph sample: the forward gathers 4 taps x 2
# components x 4 B; the gather backprojection reads each sample's 16-byte
# payload once for each of the 2 columns it taps.
L1_BYTES_PER_SAMPLE = 32.0
# DRAM bytes (read + write) per Joseph sample of one launch, from ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum) of the current kernels on the
# one-rotation cut of this scan (6.484e9 samples per launch; the commands are
# in profiles/); traffic grows with the views, so it is scaled by the sample
# count of the measured launch.  Kernels without a capture of their current
# build are absent (traffic null): the backprojection's capture (3.04 GB per
# 6.4845e9 samples) predates its row loop losing its unroll.
DRAM_BYTES_PER_SAMPLE = {"fwd_kernel<FWD_DEAM>": (1.9193e9 + 0.2392e9) / 6.4845e9}
# L1/TEX utilisation of the same kernels in those captures.
L1_BUSY = {"fwd_kernel<FWD_DEAM>": 0.682}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for n, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_config(args, case, world):
    """The `config` object of both arms' JSON lines (the same keys and values,
    so the two lines name one workload)."""
    n = case.geo.n_rays
    return {"workload": WORKLOAD, "case": args.config, "parallelism": f"replicas x{world}",
            "l2": (f"working set larger than L2 (payload {16 * n / 1e9:.2f} GB + data {8 * n / 1e9:.2f} GB "
                   f"per iteration)")}


def build_workload(name, device):
    import torch

    import synth
    case = synth.make_case(name)
    d, metal = synth.measure(case, device=device, seed=1)
    truth, M = synth.voxelize(case, device=device)
    mask = (metal >= case.metal_threshold).to(torch.uint8)
    c0 = synth.initial_image(case, truth).to(device)
    return case, d, mask, c0


def dist_init(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if (args.impl != "reference" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def reduce_max(pg, x, device):
    """Max of a float over all ranks (the slowest rank's time); x itself at N = 1."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_rate(case, d, mask, c0, seconds=15.0, views=None):
    """Oracle iterations/s measured on a bounded view sample (the oracle's rays
    restricted to a contiguous view range; the c-step runs over all voxels).
    Returns (value, sample description, threads, seconds spent)."""
    import numpy as np

    import oracle
    O = oracle.from_case(case)
    dn = d.detach().cpu().double().numpy()
    mn = mask.detach().cpu().numpy()
    cn = c0.detach().cpu().double().numpy()
    V = case.geo.n_views
    Z = O.normaliser() if case.geo.n_rays < 2e6 else 1.0   # Z only scales the update; not timed
    mid = V // 2
    if views is None:
        nv = max(1, V // 400)
        t = time.perf_counter()
        O.iterate(cn, dn, mn, n_iter=1, Z=Z, v0=mid, v1=mid + nv)
        dt = time.perf_counter() - t
        views = int(max(1, min(V, nv * seconds / max(dt, 1e-3))))
    v0 = max(0, mid - views // 2)
    v1 = min(V, v0 + views)
    t = time.perf_counter()
    O.iterate(cn, dn, mn, n_iter=1, Z=Z, v0=v0, v1=v1)
    dt = time.perf_counter() - t
    # the per-iteration work that does not scale with the views (the c-step
    # over every voxel and the clearing of the backprojection volumes), timed
    # with an empty view range and not scaled
    t = time.perf_counter()
    O.iterate(cn, dn, mn, n_iter=1, Z=Z, v0=mid, v1=mid)
    t_fixed = min(time.perf_counter() - t, dt)
    frac = (v1 - v0) / V
    full = (dt - t_fixed) / frac + t_fixed   # seconds for one whole iteration
    rate = 1.0 / full
    desc = (f"one oracle iteration over views [{v0},{v1}) = {v1 - v0}/{V} views "
            f"({100 * frac:.2f}%) plus the full c-step; {dt:.2f} s, of which {t_fixed:.2f} s do not "
            f"scale with the views; the view-dependent part scaled by views")
    return rate, desc, oracle.lib().or_num_threads(), dt


def run_reference(args):
    import torch
    world, rank, local, pg = dist_init(args)
    if rank != 0:
        return 0
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    case, d, mask, c0 = build_workload(args.config, dev)
    import oracle
    oracle.build()
    budget = max(5.0, 120.0 / max(1, args.steps + args.warmup))
    rate, desc, cores, _ = cpu_oracle_rate(case, d, mask, c0, seconds=budget)
    # fixed sample size from the calibration, then W warm-up and K timed steps
    views = max(1, int(round(rate * budget * case.geo.n_views)))
    times, rates = [], []
    frac = 1.0
    for i in range(args.warmup + args.steps):
        r, desc, cores, dt = cpu_oracle_rate(case, d, mask, c0, views=views)
        frac = min(views, case.geo.n_views) / case.geo.n_views
        if i >= args.warmup:
            times.append(dt)
            rates.append(r)
    sec_per_step = sum(times) / len(times)   # one step = one oracle pass over the view sample
    value = len(rates) / sum(1.0 / x for x in rates)   # full iterations per second
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec_per_step,
            "sample_fraction_per_step": frac,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, case, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import numpy as np
    import torch

    import paper_2202_00116_gb300 as pkg
    from paper_2202_00116_gb300 import build
    world, rank, local, pg = dist_init(args)
    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    case, d, mask, c0 = build_workload(args.config, dev)
    geo = case.geo
    torch.cuda.synchronize(dev)
    t_ctx = time.perf_counter()
    gpu = pkg.from_case(case)
    gpu.set_data(d)
    gpu.set_metal_mask(mask, "ray")
    torch.cuda.synchronize(dev)
    t_ctx = time.perf_counter() - t_ctx
    samples = gpu.count_samples()
    stream = torch.cuda.current_stream(dev)
    args._l1_gbs = pkg.l1_bandwidth() / 1e9   # on-chip peak for the roofline's L1 view
    # one-time setup next to the iterations: the MAR initialisation (NMAR + FBP
    # of both spectra + Eq. 4), timed on the device; the decomposition weights
    # here are the spectrum-weighted mean attenuations (the timing does not
    # depend on them)
    w = case.I0 / case.I0.sum(axis=1, keepdims=True)
    calib = [float((w[0] * case.mu[0]).sum()), float((w[0] * case.mu[1]).sum()),
             float((w[1] * case.mu[0]).sum()), float((w[1] * case.mu[1]).sum())]
    mar_kw = dict(t_air=0.005, t_bone=0.026, soft_value=0.0195, prior_spectrum=1)
    gpu.mar_init(calib, **mar_kw)
    torch.cuda.synchronize(dev)
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m0.record(stream)
    gpu.mar_init(calib, **mar_kw)
    m1.record(stream)
    torch.cuda.synchronize(dev)
    args._setup = {"context_s": t_ctx, "mar_init_ms": m0.elapsed_time(m1)}

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize(dev)

    # ---- device-resident timing ----
    c = c0.clone()
    gpu.iterate(c, args.warmup)
    barrier()
    gpu.profile(True)
    gpu.kernel_times(reset=True)
    with ClockSampler(local) as clk:
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hist = gpu.iterate(c, args.steps)
        e1.record(stream)
        barrier()
    gpu.profile(False)
    ms = reduce_max(pg, e0.elapsed_time(e1), dev)
    kms, kn = gpu.kernel_times(reset=True)
    value = world * args.steps / (ms / 1e3)

    # ---- end to end through the C ABI with host buffers ----
    if args.no_e2e:
        return finish_line(args, world, rank, pg, gpu, case, d, mask, c0, samples, ms, value, kms, kn, hist, clk,
                           None)
    d_h = d.cpu().pin_memory()
    m_h = mask.cpu().pin_memory()
    c_h = c0.cpu().pin_memory()
    e2e_steps = max(1, args.steps)

    def e2e_step():
        gpu.set_data(d_h)
        gpu.set_metal_mask(m_h, "ray")
        gpu.iterate(c_h, 1)      # copies c in, iterates, copies c and F out (synchronous)

    e2e_step()                   # untimed: the host path's first call sets up its staging buffer
    barrier()
    with ClockSampler(local) as clk_e2e:
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        barrier()
        e2e_s = reduce_max(pg, time.perf_counter() - t0, dev)
    e2e_val = world * e2e_steps / e2e_s
    h2d = d_h.numel() * 4 + m_h.numel() + c_h.numel() * 4
    d2h = c_h.numel() * 4 + 8
    e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
           "ms_per_step": 1e3 * e2e_s / e2e_steps, "clocks": clk_e2e.summary()}
    return finish_line(args, world, rank, pg, gpu, case, d, mask, c0, samples, ms, value, kms, kn, hist, clk, e2e)


def finish_line(args, world, rank, pg, gpu, case, d, mask, c0, samples, ms, value, kms, kn, hist, clk, e2e):
    geo = case.geo
    # ---- roofline of the dominant kernel ----
    # No step is a dense contraction: the stated ceiling is HBM on the bytes the
    # method must move (each kernel's compulsory bytes over its CUDA-event
    # duration, against the measured copy bandwidth); the realistic bound of
    # both projector kernels is the on-chip L1 data path (algorithmic 32 B per
    # Joseph sample against the measured shared-load throughput of this GPU).
    stages = ["layout", "forward", "reduce", "backproject"]
    avg = {s: kms[i] / max(kn[i], 1) * (2 if s == "layout" else 1) for i, s in enumerate(stages)}
    dom = max(["forward", "backproject"], key=lambda s: avg[s])
    peaks = _peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    hbm = peaks.get("hbm_gbs")
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)"
    if hbm is None:
        hbm, hbm_src = 6800.0, "profiling recipe fallback 6.8 TB/s (of fallback)"
    # the library's slab depth for this scan (2 for one or two slices, 8 for thin
    # rows, else 13)
    slab = (2 if geo.nz <= 2 else
            8 if (geo.n_rows == 1 or geo.dz >= 1.5 * geo.row_pitch * geo.sid / geo.sdd) else 13)
    kname = {"forward": "fwd_kernel<FWD_DEAM>", "backproject": f"bwd_kernel<1,{slab}>"}[dom]
    nvox, nrays = geo.n_voxels, geo.n_rays
    # compulsory bytes per launch: forward reads c (via its two layouts, 8 B per
    # voxel each way counted once: 16 B/voxel), d~ (8 B/ray) and the mask
    # (1 B/ray) and writes the payload (16 B/ray); the backprojection reads the
    # payload (16 B/ray) and reads and writes c (16 B/voxel)
    comp_bytes = {"forward": 16 * nvox + 8 * nrays + nrays + 16 * nrays,
                  "backproject": 16 * nrays + 16 * nvox}[dom]
    t_s = avg[dom] / 1e3
    achieved = comp_bytes / t_s / 1e9
    l1_peak = getattr(args, "_l1_gbs", None)
    l1_ach = L1_BYTES_PER_SAMPLE * samples / t_s / 1e9
    fp32_peak = 152 * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12   # TFLOP/s, FMA = 2 flops
    # algorithmic flops per Joseph sample: forward = 6 two-point interpolations of
    # 2 components (12 flops); backprojection = 4 taps x 4 accumulators FMA (32
    # flops) + 4 tap weights (4 flops)
    flops = {"forward": 12.0, "backproject": 36.0}[dom] * samples / t_s / 1e12
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": hbm_src,
                "traffic": (DRAM_BYTES_PER_SAMPLE[kname] * samples if kname in DRAM_BYTES_PER_SAMPLE else None),
                "bytes_per_launch": comp_bytes, "ms_per_launch": avg[dom],
                "l1": {"achieved": l1_ach, "peak": l1_peak, "unit": "GB/s",
                       "frac": (l1_ach / l1_peak if l1_peak else None),
                       "bytes_per_sample": L1_BYTES_PER_SAMPLE, "samples_per_launch": samples,
                       "peak_source": "deam_l1_bandwidth: shared-memory load throughput measured in this run",
                       "l1tex_busy_ncu": L1_BUSY.get(kname)},
                "fp32": {"achieved": flops, "peak": fp32_peak, "unit": "TFLOP/s", "frac": flops / fp32_peak,
                         "peak_source": f"152 SMs x 128 FP32 lanes x 2 flops x {sm_max:.0f} MHz (derived)"}}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded phantom, analytic polyenergetic projections, Poisson + Gaussian noise)",
            "config": workload_config(args, case, world),
            "ray_samples_per_projection": samples,
            "ray_samples_per_s": samples * value,
            "stage_ms": {s: avg[s] for s in stages},
            "objective_first_last": [float(hist[0]), float(hist[-1])],
            "gpu_launches": int(sum(kn)),
            "setup": getattr(args, "_setup", None),
            "e2e": e2e,
            "roofline": roofline,
            "clocks": clk.summary()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, desc, cores, _ = cpu_oracle_rate(case, d, mask, c0, seconds=args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    gpu.close()
    if pg is not None:
        pg.destroy_process_group()
    return 0


def run_batch(args):
    """Batched MAR-DEAM over seeded scans of uneven size (2D slices and 3D helical
    slabs, 180-1160 views, 1-3 metal inserts each): one batch iteration = one
    MAR-DEAM iteration of every scan.  The same iterations run scan by scan through
    deam_iterate for comparison, and the two results are compared."""
    import numpy as np
    import torch

    import paper_2202_00116_gb300 as pkg
    import synth
    from paper_2202_00116_gb300 import build
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    cases = synth.make_batch_cases(args.batch_scans)
    scans, imgs = [], []
    samples = 0
    for case in cases:
        d, metal = synth.measure(case, device=dev, seed=1)
        truth, _ = synth.voxelize(case, device=dev)
        mask = (metal >= case.metal_threshold).to(torch.uint8)
        g = pkg.from_case(case)
        g.set_data(d)
        g.set_metal_mask(mask, "ray")
        samples += g.count_samples()
        scans.append(g)
        imgs.append(synth.initial_image(case, truth).to(dev))
        del d, metal, truth, mask
    stream = torch.cuda.current_stream(dev)
    batch = pkg.DeamBatch(scans, autotune=True)
    cb = [c.clone() for c in imgs]
    batch.iterate(cb, args.warmup)                  # includes the tuning and the graph capture
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.iterate(cb, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1)
    # the same iterations scan by scan
    cs = [c.clone() for c in imgs]
    for g, c in zip(scans, cs):
        g.iterate(c, args.warmup)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        for g, c in zip(scans, cs):
            g.iterate(c, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    diff = max(float(torch.linalg.vector_norm((a - b).double()) / torch.linalg.vector_norm(b.double()))
               for a, b in zip(cb, cs))
    line = {"metric": "batched DEAM iterations/s", "value": args.steps / (ms_batch / 1e3), "unit": "it/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": f"{len(cases)} seeded scans of uneven size "
                                                         "(2D 128^2-512^2, 3D slabs 256^2x16-512^2x48, "
                                                         "180-1160 views/rotation, 1-3 metal inserts)",
                                            "rays": int(sum(c.geo.n_rays for c in cases)),
                                            "voxels": int(sum(c.geo.n_voxels for c in cases))},
            "ray_samples_per_s": samples * args.steps / (ms_batch / 1e3),
            "sequential_deam_iterate": {"value": args.steps / (ms_seq / 1e3), "ms_per_step": ms_seq / args.steps},
            "speedup_vs_sequential": ms_seq / ms_batch,
            "max_rel_l2_batched_vs_sequential": diff,
            "tuning": batch.info(), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    batch.close()
    return 0

def _timed_iterate(g, c, n, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    h = g.iterate(c, n)
    e1.record(stream)
    torch.cuda.synchronize()
    return h, e0.elapsed_time(e1)


def run_compare(args):
    """The default (mixed-precision) DEAM, its adjoint (gradient) form and its
    batched form, each next to the plain-FP32 GPU DEAM (deam_options.precision
    = 1: uncompensated FP32 spectral sums and FP32 objective accumulation):

    precision  at 512x512x64 helical: iterations/s of both; payload error on
               seeded sampled rays against the FP64 oracle; the FP32 objective's
               deviation from the FP64-reduced one; at the 2D fan case, each
               output's error after 10 iterations against the full oracle run.
    adjoint    at 256x256x32 helical: DEAM iterations against Barzilai-Borwein
               gradient descent on the same objective (gradients from the
               adjoint kernel), compared at the same objective value.
    batched    24 seeded scans of uneven size: one batch against scan-by-scan
               plain-FP32 and mixed deam_iterate.
    """
    import numpy as np
    import torch

    import oracle
    import paper_2202_00116_gb300 as pkg
    import synth
    from paper_2202_00116_gb300 import build, solvers
    build.build()
    oracle.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream(dev)
    rng = np.random.default_rng(11)
    out = {}

    def rel(a, b):
        a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    # precision, full size
    case, d, mask, c0 = build_workload("c2", dev)
    O = oracle.from_case(case)
    rays = np.sort(rng.choice(case.geo.n_rays, size=4096, replace=False))
    _, _, po, fo = O.ray_model(c0.cpu().double().numpy(), d.cpu().double().numpy(), mask.cpu().numpy(), rays)
    prec = {}
    for p in ("mixed", "fp32"):
        g = pkg.from_case(case, precision=p)
        g.set_data(d)
        g.set_metal_mask(mask, "ray")
        pay, F = g.ray_terms(c0)
        pg = pay.reshape(-1, 4)[torch.from_numpy(rays).to(dev)].cpu().double().numpy()
        c = c0.clone()
        g.iterate(c, args.warmup)
        h, ms = _timed_iterate(g, c, args.steps, stream)
        prec[p] = {"it_per_s": args.steps / (ms / 1e3), "ms_per_it": ms / args.steps, "objective_at_c0": F,
                   "sampled_rays_rel_l2": {"B_tilde": rel(pg[:, :2], po[:, :2]),
                                           "B_hat": rel(pg[:, :2] + pg[:, 2:], po[:, 2:])},
                   "image": c}
        g.close()
    prec["fp32"]["objective_rel_dev_from_fp64_reduction"] = abs(
        prec["fp32"]["objective_at_c0"] - prec["mixed"]["objective_at_c0"]) / prec["mixed"]["objective_at_c0"]
    prec["image_rel_l2_fp32_vs_mixed_after_iterations"] = rel(prec["fp32"].pop("image").cpu().numpy(),
                                                              prec["mixed"].pop("image").cpu().numpy())
    del d, mask, c0
    case, d, mask, c0 = build_workload("c0", dev)
    O = oracle.from_case(case)
    c_ref, h_ref, _ = O.iterate(c0.cpu().double().numpy(), d.cpu().double().numpy(), mask.cpu().numpy(),
                                n_iter=10)
    for p in ("mixed", "fp32"):
        g = pkg.from_case(case, precision=p)
        g.set_data(d)
        g.set_metal_mask(mask, "ray")
        c = c0.clone()
        h = g.iterate(c, 10)
        prec[p]["fan2d_10_iterations_vs_oracle"] = {
            "image_rel_l2": rel(c.cpu().numpy(), c_ref),
            "objective_history_max_rel": float(np.max(np.abs(h - h_ref) / h_ref))}
        g.close()
    out["precision"] = prec

    # adjoint form against DEAM, 256x256x32 helical
    case, d, mask, c0 = build_workload("c1", dev)
    runs = {}
    for p in ("fp32", "mixed"):
        g = pkg.from_case(case, precision=p)
        g.set_data(d)
        g.set_metal_mask(mask, "ray")
        c = c0.clone()
        g.iterate(c.clone(), 2)
        h, ms = _timed_iterate(g, c, 50, stream)
        runs[p] = (np.append(h, g.objective(c)), ms / 50)
        if p == "mixed":
            gm = g
        else:
            g.close()
    cg = c0.clone()
    gm.gradient(cg)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(5):
        gm.gradient(cg)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_grad = e0.elapsed_time(e1) / 5
    hf, ms_f = runs["fp32"]
    target = hf[20]   # the plain-FP32 DEAM's objective after 20 iterations

    def solver_leg(pre):
        x = c0.clone()
        r = solvers.gradient_descent(gm, x, 200, precondition=pre)
        reach = np.nonzero(r["objective"][1:] <= target)[0]
        return {"steps": len(r["objective"]) - 1,
                "evaluations": int(r["evaluations"][-1]) if r["evaluations"] else 0,
                "seconds": r["seconds"][-1] if r["seconds"] else 0.0,
                "objective": {k: float(r["objective"][k]) for k in (0, 1, 10, 20, 50, 100, 200)
                              if k < len(r["objective"])},
                "steps_to_deam20": int(reach[0]) + 1 if reach.size else None,
                "seconds_to_deam20": r["seconds"][int(reach[0])] if reach.size else None}
    adj = {"workload": "256x256x32 helical, 16x672, 3480 views, 2 x 60 bins",
           "deam_fp32": {"ms_per_iteration": ms_f, "objective": {k: float(hf[k]) for k in (0, 1, 5, 10, 20, 50)}},
           "deam_mixed": {"ms_per_iteration": runs["mixed"][1],
                          "objective": {k: float(runs["mixed"][0][k]) for k in (0, 1, 5, 10, 20, 50)}},
           "ms_per_gradient": ms_grad,
           "gradient_descent_bb": solver_leg(False),
           "gradient_descent_bb_preconditioned_1_over_Z_btilde": solver_leg(True),
           "same_accuracy_target": "objective of plain-FP32 DEAM after 20 iterations",
           "deam_fp32_seconds_to_deam20": 20 * ms_f / 1e3}
    gm.close()
    out["adjoint"] = adj
    del d, mask, c0

    # batched form
    cases = synth.make_batch_cases(args.batch_scans)
    bat = {}
    for p in ("fp32", "mixed"):
        scans, imgs = [], []
        for cs in cases:
            dd, metal = synth.measure(cs, device=dev, seed=1)
            truth, _ = synth.voxelize(cs, device=dev)
            g = pkg.from_case(cs, precision=p)
            g.set_data(dd)
            g.set_metal_mask((metal >= cs.metal_threshold).to(torch.uint8), "ray")
            scans.append(g)
            imgs.append(synth.initial_image(cs, truth).to(dev))
            del dd, metal, truth
        cs_ = [c.clone() for c in imgs]
        for g, c in zip(scans, cs_):
            g.iterate(c, 1)
        torch.cuda.synchronize()
        e0.record(stream)
        for g, c in zip(scans, cs_):
            g.iterate(c, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        bat[f"sequential_{p}"] = {"it_per_s": args.steps / (e0.elapsed_time(e1) / 1e3)}
        if p == "mixed":
            batch = pkg.DeamBatch(scans, autotune=True)
            cb = [c.clone() for c in imgs]
            batch.iterate(cb, 2)
            torch.cuda.synchronize()
            e0.record(stream)
            batch.iterate(cb, args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            bat["batched_mixed"] = {"it_per_s": args.steps / (e0.elapsed_time(e1) / 1e3),
                                    "plan": batch.info()["plan"]}
            batch.close()
        for g in scans:
            g.close()
    bat["scans"] = len(cases)
    out["batched"] = bat
    line = {"metric": "comparison with the plain-FP32 GPU DEAM", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "data": "synthetic", "comparisons": out}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg (profiling runs)")
    ap.add_argument("--batch-scans", type=int, default=24)
    args = ap.parse_args()
    if args.config == "batch":
        return run_batch(args)
    if args.config == "compare":
        return run_compare(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
