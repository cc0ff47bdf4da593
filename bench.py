#!/usr/bin/env python3
"""Benchmark of the render hot path on the 256^3 eight-room floor workload:
512 kd fields, W=64/H=3 tiny MLPs, one 1024x512 equirectangular view plus one
1920x1080 perspective view (90 degree FOV), <= 128 samples per ray.

One step = one roam_render call over both views: ray generation, march,
field lookup, bucketing, encoding + grouped MLPs, compositing with early
termination.  Inputs (grid, labels, weights) are resident on the device;
L2 is flushed (256 MiB write) between timed steps.

value = composited samples per second (samples that reach the image, up to
each ray's termination), summed over ranks; under torchrun every rank renders
its own replica of the workload (weak scaling, no collective on the data
path).

--impl reference times the FP64 CPU oracle (the reference arm of this
benchmark) on bounded samples of the same workload.
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
sys.path.insert(0, ROOT)

METRIC = "samples/s & 1024×512 frame ms, BF16-TC vs FP32 on GB300 at ≥40 dB PSNR vs oracle"
UNIT = "samples/s"


def macs_per_sample(W, H):
    return 63 * W + (H - 1) * W * W + W * (1 + W) + (W + 27) * W + 3 * W


def workload_config(wl, views):
    return {"workload": "floor256_kd512_w64h3_equirect1024x512_persp1920x1080",
            "grid": "256^3 bit-packed, %.1f%% occupied" % (100.0 * wl.scene.n_occupied / 256 ** 3),
            "fields": wl.part.n_fields, "mlp": f"W={wl.W} H={wl.H} ({macs_per_sample(wl.W, wl.H)} MACs/sample)",
            "views": views, "n_max": wl.n_max, "delta": "vox/4", "t_stop": 1e-4,
            "l2": "flushed between timed steps (256 MiB write)"}


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def oracle_sample_rays(wl, n, seed):
    import numpy as np
    rng = np.random.default_rng(seed)
    sizes = [c.n_pixels for c in wl.cams]
    view = rng.integers(0, len(sizes), n)
    pix = np.array([rng.integers(0, sizes[v]) for v in view], dtype=np.int64)
    return np.stack([view, pix], 1).astype(np.uint32)


def cpu_oracle_rate(wl, target_s: float, seed: int = 1234):
    """Times the FP64 oracle (as it stands) on a bounded ray sample sized for
    about target_s seconds.  Returns (samples/s, cores, description)."""
    import fixtures as F
    import oracle as O
    g = O.Grid(wl.scene, wl.part)
    cams = F.camera_array(wl.cams)
    probe = oracle_sample_rays(wl, 2000, seed)
    t0 = time.perf_counter()
    r = O.render(g, wl.weights, wl.affine, wl.W, wl.H, wl.sigma_scale, cams, probe, wl.delta, wl.n_max)
    dt = time.perf_counter() - t0
    n = int(max(2000, min(2_000_000, 2000 * target_s / max(dt, 1e-3))))
    rays = oracle_sample_rays(wl, n, seed + 1)
    t0 = time.perf_counter()
    r = O.render(g, wl.weights, wl.affine, wl.W, wl.H, wl.sigma_scale, cams, rays, wl.delta, wl.n_max)
    dt = time.perf_counter() - t0
    used = int(r["n_used"].sum())
    return used / dt, O.threads(), f"{n} random pixels of both views ({used} composited samples, {dt:.1f} s)", n / dt


def cpu_oracle_frames(wl, rate_rays_all, one_core_s: float = 4.0):
    """The rest of the CPU baseline plan: the oracle on one core (samples/s
    on a bounded sample), and per-frame times -- the 128x64 room rendered
    whole on all cores, the 1024x512 floor view extrapolated from the
    all-core ray rate measured on a sample (stated as such)."""
    import fixtures as F
    import oracle as O
    g = O.Grid(wl.scene, wl.part)
    cams = F.camera_array(wl.cams)
    all_cores = O.threads()
    O.set_threads(1)
    try:
        probe = oracle_sample_rays(wl, 300, 77)
        t0 = time.perf_counter()
        O.render(g, wl.weights, wl.affine, wl.W, wl.H, wl.sigma_scale, cams, probe, wl.delta, wl.n_max)
        dt = time.perf_counter() - t0
        n1 = int(max(300, min(200_000, 300 * one_core_s / max(dt, 1e-3))))
        rays = oracle_sample_rays(wl, n1, 78)
        t0 = time.perf_counter()
        r = O.render(g, wl.weights, wl.affine, wl.W, wl.H, wl.sigma_scale, cams, rays, wl.delta, wl.n_max)
        dt1 = time.perf_counter() - t0
    finally:
        O.set_threads(all_cores)
    one = {"value": int(r["n_used"].sum()) / dt1, "unit": UNIT, "cores": 1,
           "sample": f"{n1} random pixels of both views ({dt1:.1f} s)"}
    room = F.room32()
    gr = O.Grid(room.scene, room.part)
    t0 = time.perf_counter()
    O.render(gr, room.weights, room.affine, room.W, room.H, room.sigma_scale, F.camera_array(room.cams), None,
             room.delta, room.n_max)
    room_ms = 1000 * (time.perf_counter() - t0)
    eq_pixels = wl.cams[0].n_pixels
    frames = {"room32_128x64_ms": room_ms, "cores": all_cores,
              "floor256_equirect_1024x512_ms_extrapolated": 1000.0 * eq_pixels / rate_rays_all,
              "extrapolation": "all-core ray rate of the sampled pixels (both views) times the view's pixel count"}
    return one, frames


def reference_arm(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import fixtures as F
    import oracle as O
    wl = F.floor256()
    g = O.Grid(wl.scene, wl.part)
    cams = F.camera_array(wl.cams)
    n_rays = 6000
    times, used = [], []
    for step in range(args.warmup + args.steps):
        rays = oracle_sample_rays(wl, n_rays, 100 + step)
        t0 = time.perf_counter()
        r = O.render(g, wl.weights, wl.affine, wl.W, wl.H, wl.sigma_scale, cams, rays, wl.delta, wl.n_max)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            used.append(int(r["n_used"].sum()))
    value = sum(used) / sum(times)
    views = ["equirect 1024x512", "perspective 1920x1080 fov 90"]
    sample = f"each step: {n_rays} random pixels of both views"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(wl, views),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.threads(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_steps(r, cams, opts, steps, warmup, flush, stream):
    import torch
    for _ in range(warmup):
        r.render(cams, opts, stream=stream)
    torch.cuda.synchronize()
    total = 0.0
    per = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r.render(cams, opts, stream=stream)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        per.append(ms)
        total += ms
    return total, per


def peaks_bf16():
    """Dense BF16 burst TFLOP/s: the driver's measurement on this machine, else
    the recipe's fallback (1.9 PFLOP/s)."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except (OSError, ValueError, KeyError):
        return 1900.0


def train_step_bench(roam, F, torch, wl, args, stream):
    """One fine-tuning step = forward (BF16 tensor cores) + L2 loss + adjoint
    (composite + BF16 tensor-core MLP adjoint) + Adam, on 65,536 rays of 16
    1024x512 equirect views of the floor (targets rendered once, untimed)."""
    import numpy as np
    cams = F.make_cameras(wl.scene, 3, [(F.EQUIRECT, 1024, 512, 0.0)] * 16)
    teacher = roam.Roam(torch.cuda.current_device())
    teacher.load_workload(wl)
    rgb_t, _, _ = teacher.render(cams, roam.render_opts(wl.delta, wl.n_max, precision=roam.ROAM_BF16))
    n = 65536
    rays_np = F.ray_batch(3, cams, n)
    rays = torch.from_numpy(rays_np.astype(np.int32)).cuda()
    gidx = torch.from_numpy((rays_np[:, 0].astype(np.int64) * 1024 * 512 + rays_np[:, 1]).astype(np.int64)).cuda()
    noise = torch.from_numpy(F.rng_for(3, F.ROLE_NOISE).normal(0, 0.01, (n, 3)).astype(np.float32)).cuda()
    target = (rgb_t[gidx] + noise).contiguous()
    teacher.close()
    student = F.xavier_weights(2, F.ROLE_STUDENT, wl.part.n_fields, wl.W, wl.H)
    r = roam.Roam(torch.cuda.current_device())
    r.load_grid(wl.scene.bits, wl.scene.dims, wl.scene.origin, wl.scene.vox)
    r.load_fields(wl.part.field_of_rank, wl.affine)
    r.load_weights(student, wl.W, wl.H, wl.sigma_scale)
    opts = roam.render_opts(wl.delta, wl.n_max, precision=roam.ROAM_BF16)

    def step(k):
        loss, g = r.local_grad(cams, rays, target, opts, 3.0 * n, stream=stream)
        r.adam_step(g, lr=1e-3, step=k, stream=stream)
        return loss

    for k in range(1, 4):
        step(k)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    steps = max(3, args.steps)
    losses = []
    # the step time without per-kernel events, then the same number of steps
    # again with them for the kernel breakdown
    a.record(stream)
    for k in range(4, 4 + steps):
        losses.append(step(k))
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b) / steps
    r.profile(True)
    a.record(stream)
    for k in range(4 + steps, 4 + 2 * steps):
        losses.append(step(k))
    b.record(stream)
    b.synchronize()
    prof = r.profile_read()
    r.profile(False)
    ms_profiled = a.elapsed_time(b) / steps
    st = r.get_stats()
    r.close()
    out = {"workload": "floor256_kd512_w64h3, 16 equirect 1024x512 views, 65536 random rays, teacher+N(0,0.01^2) targets",
           "ms_per_step": ms, "rays_per_s": n / (ms / 1000.0), "samples_per_step": int(st.n_samples),
           "composited_per_step": int(st.n_used),
           "ms_per_step_with_kernel_events": ms_profiled,
           "loss_first_last": [float(losses[0]), float(losses[-1])],
           "kernels": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in prof.items()},
           "precision": "forward BF16 tcgen05, adjoint BF16 tcgen05 (FP32 accumulation), FP32 master weights"}
    bw = prof.get("mlp_bwd_bf16_tcgen05")
    if bw and bw[1] > 0:
        # adjoint work per sample: forward recompute + wgrad + dgrad (no dgrad into the encoding)
        macs = macs_per_sample(wl.W, wl.H)
        flops = 2.0 * (3 * macs - wl.W * 63)
        per_launch_s = bw[1] / bw[0] / 1000.0
        # the adjoint runs over the composited samples (each ray's samples up
        # to its termination, the ones the loss reaches), not every evaluated one
        samples = st.n_used
        out["mlp_adjoint"] = {"flops_per_sample": flops, "samples_per_launch": int(samples),
                              "tflops": flops * samples / per_launch_s / 1e12,
                              "frac_of_bf16_peak": flops * samples / per_launch_s / 1e12 / peaks_bf16(),
                              "ms_per_launch": bw[1] / bw[0]}
    return out



def accuracy(r, roam, F, g, wl, rays, prec, got, ref, quant=0, widths=None):
    """Sampled pixels against the FP64 oracle under the render parity rule
    (oracle.parity): every ray is held to the bar of its precision, against
    the oracle's render where the library's kept-sample list equals the
    oracle's, and against the oracle recomputed on the library's own list
    where it differs (certified near-ties, counted).  Also gives the raw max
    over all pixels against the oracle's own march."""
    import numpy as np
    import torch
    import oracle.parity as P
    opts = roam.render_opts(wl.delta, wl.n_max, precision=prec)
    cnt, recs = r.march(wl.cams, opts, rays=torch.from_numpy(rays.astype(np.int32)).cuda())
    torch.cuda.synchronize()
    tol = 1e-4 if prec == roam.ROAM_F32 else 2e-2
    W = wl.W if widths is None else 0
    rep = P.check_render(g, wl.weights, wl.affine, W, wl.H, wl.sigma_scale, F.camera_array(wl.cams), rays, wl.delta,
                         wl.n_max, cnt.cpu().numpy(), recs.cpu().numpy(), got, tol=tol, quant=quant, widths=widths,
                         ref=ref)
    raw = np.abs(got - ref["rgb"]).max(axis=1)
    return {"psnr_db": rep.psnr(got), "max_abs": rep.max_err, "bar": tol, "over_bar": int(rep.over.size),
            "pixels": rep.n, "records_equal": rep.n_equal, "certified_mismatches": len(rep.certified),
            "uncertified_mismatches": len(rep.uncertified), "termination_ties": rep.term_ties,
            "max_abs_vs_oracle_own_march": float(raw.max()) if raw.size else 0.0}


def large_scene_bench(roam, F, torch, args, stream, flush, peaks):
    """The 512^3 twenty-room floor: 4096 kd fields of W=128/H=4 MLPs, one
    2048x1024 equirectangular view, <= 192 samples per ray; BF16 and FP8
    E4M3 tensor-core paths and the FP32 SIMT form, each with its frame time,
    MLP-kernel roofline and accuracy on sampled pixels against the FP64
    oracle (FP8 also against the oracle's FP8 reading)."""
    import numpy as np
    import oracle as O
    wl = F.floor512()
    r = roam.Roam(torch.cuda.current_device())
    r.load_workload(wl)
    flops_per = 2.0 * macs_per_sample(wl.W, wl.H)
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    out = {"workload": f"floor512_kd4096_w128h4_equirect2048x1024 ({100.0 * wl.scene.n_occupied / 512 ** 3:.1f}% "
                       f"occupied, n_max {wl.n_max})", "paths": {}}
    g = O.Grid(wl.scene, wl.part)
    rays = oracle_sample_rays(wl, 2000, 17)
    cams = F.camera_array(wl.cams)
    ref = O.render(g, wl.weights, wl.affine, wl.W, wl.H, wl.sigma_scale, cams, rays, wl.delta, wl.n_max)
    ref8 = O.render(g, wl.weights, wl.affine, wl.W, wl.H, wl.sigma_scale, cams, rays, wl.delta, wl.n_max, quant=1)
    gi = rays[:, 1].astype(np.int64)
    steps = max(3, args.steps // 2)
    for prec, tag, key, peak in ((roam.ROAM_BF16, "bf16", "mlp_bf16_tcgen05", bf16_peak),
                                 (roam.ROAM_FP8, "fp8_e4m3", "mlp_fp8_tcgen05", 2.0 * bf16_peak),
                                 (roam.ROAM_F32, "f32", "mlp_f32_simt", None)):
        opts = roam.render_opts(wl.delta, wl.n_max, precision=prec)
        for _ in range(3):
            r.render(wl.cams, opts, stream=stream)
        torch.cuda.synchronize()
        r.profile(True)
        tot, per = time_steps(r, wl.cams, opts, steps, 0, flush, stream)
        prof = r.profile_read()
        r.profile(False)
        st = r.get_stats()
        rgb, _, _ = r.render(wl.cams, opts, stream=stream)
        torch.cuda.synchronize()
        got = rgb.cpu().numpy()[gi].astype(np.float64)
        acc = {}
        for name, rr, quant in (("vs_fp64_oracle", ref, 0), ("vs_oracle_fp8_reading", ref8, 1)):
            if name == "vs_oracle_fp8_reading" and prec != roam.ROAM_FP8:
                continue
            acc[name] = accuracy(r, roam, F, g, wl, rays, prec, got, rr, quant=quant)
        launches, mlp_ms = prof.get(key, (0, float("nan")))
        tflops = flops_per * st.n_samples * steps / (mlp_ms / 1000.0) / 1e12
        path = {"frame_ms": statistics.median(per), "samples_per_s": st.n_used * steps / (tot / 1000.0),
                "mlp_ms_per_frame": mlp_ms / steps, "mlp_tflops": tflops,
                "kernels": {k: round(v[1] / steps, 4) for k, v in prof.items() if v[0]}, "accuracy": acc,
                "samples_per_frame": {"composited": int(st.n_used), "evaluated": int(st.n_samples)}}
        if peak:
            path["mlp_frac_of_peak"] = tflops / peak
            path["peak"] = ("measured bf16 burst" if prec == roam.ROAM_BF16 else
                            "2 x measured bf16 burst (nominal fp8:bf16 ratio)") if peaks else "fallback"
        out["paths"][tag] = path
    r.close()
    return out


def multiview_bench(roam, F, torch, args, stream, flush):
    """The 384^3 twelve-room floor: 2048 kd fields with per-field widths drawn
    from 32/64/128, H=3, and 32 views (24 equirectangular from 512x256 to
    2048x1024, 8 perspective 1280x720), BF16 tensor cores.  One batched call
    over all views (round size from roam_tune_round_size), CUDA-graph
    replayed and plain, against one render call per view; sampled pixels
    against the FP64 oracle."""
    import numpy as np
    import oracle as O
    wl = F.floor384()
    r = roam.Roam(torch.cuda.current_device())
    r.load_workload(wl)
    base = roam.render_opts(wl.delta, wl.n_max, precision=roam.ROAM_BF16)
    R, R0, tune_ms = r.tune_round_size(wl.cams, base, stream=stream)
    opts = roam.render_opts(wl.delta, wl.n_max, precision=roam.ROAM_BF16, round_size=R, first_round_size=R0)
    gopts = roam.render_opts(wl.delta, wl.n_max, precision=roam.ROAM_BF16, round_size=R, first_round_size=R0,
                             use_graph=True)
    steps = max(3, args.steps // 2)
    out = {"workload": "floor384_kd2048_mixed_w32_64_128_h3, 32 views (24 equirect 512x256..2048x1024, "
                       "8 perspective 1280x720)", "rays_per_batch": int(sum(c.n_pixels for c in wl.cams)),
           "round_size_tuned": R, "first_round_size_tuned": R0, "tuned_render_ms": tune_ms}
    for _ in range(2):
        r.render(wl.cams, gopts, stream=stream)
    tot_g, per_g = time_steps(r, wl.cams, gopts, steps, 0, flush, stream)
    st = r.get_stats()
    tot_b, per_b = time_steps(r, wl.cams, opts, steps, 1, flush, stream)
    # one call per view, the same options
    per_v = []
    for k in range(steps + 1):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for cam in wl.cams:
            r.render([cam], opts, stream=stream)
        b.record(stream)
        b.synchronize()
        if k:
            per_v.append(a.elapsed_time(b))
    out.update({"batched_graph_ms": statistics.median(per_g), "batched_plain_ms": statistics.median(per_b),
                "per_view_calls_ms": statistics.median(per_v),
                "speedup_batched_graph_vs_per_view": statistics.median(per_v) / statistics.median(per_g),
                "samples_per_s": st.n_used * steps / (tot_g / 1000.0),
                "samples_per_batch": {"composited": int(st.n_used), "evaluated": int(st.n_samples)}})
    rgb, _, _ = r.render(wl.cams, gopts, stream=stream)
    torch.cuda.synchronize()
    g = O.Grid(wl.scene, wl.part)
    rays = oracle_sample_rays(wl, 2000, 31)
    ref = O.render(g, wl.weights, wl.affine, 0, wl.H, wl.sigma_scale, F.camera_array(wl.cams), rays, wl.delta,
                   wl.n_max, widths=wl.widths)
    starts = np.concatenate([[0], np.cumsum([c.n_pixels for c in wl.cams])])
    gi = starts[rays[:, 0].astype(np.int64)] + rays[:, 1].astype(np.int64)
    out["accuracy_vs_oracle"] = accuracy(r, roam, F, g, wl, rays, roam.ROAM_BF16, rgb.cpu().numpy()[gi].astype(np.float64),
                                         ref, widths=wl.widths)
    r.close()
    return out


def occupancy_bench(roam, F, torch, args, stream):
    """Progressive occupancy update (Eq. 6) on the floor256 lattice: depth
    and opacity of 16 equirect 1024x512 views rendered once (BF16, untimed),
    then 16 scans per step (ray traversal + per-voxel log-odds update)."""
    import numpy as np
    wl = F.floor256(views="equirect")
    r = roam.Roam(torch.cuda.current_device())
    r.load_workload(wl)
    cams = F.make_cameras(wl.scene, 3, [(F.EQUIRECT, 1024, 512, 0.0)] * 16)
    _, depth, op = r.render(cams, roam.render_opts(wl.delta, wl.n_max, precision=roam.ROAM_BF16))
    n_vox = 256 ** 3
    L = torch.zeros(n_vox, dtype=torch.float32, device="cuda")
    bits = torch.zeros(n_vox // 32, dtype=torch.int32, device="cuda")
    for _ in range(2):
        r.occupancy_update(cams, depth, op, L, bits, stream=stream)
    torch.cuda.synchronize()
    steps = max(3, args.steps // 2)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        r.occupancy_update(cams, depth, op, L, bits, stream=stream)
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b) / steps
    n_rays = 16 * 1024 * 512
    occ = int(np.unpackbits(bits.cpu().numpy().view(np.uint8)).sum())
    r.close()
    # per scan the voxel pass reads the log-odds, hit word and free word and
    # writes the occupancy word (the updated voxels' log-odds on top)
    bytes_scan = n_vox * (4 + 4) + n_vox // 8 * 2
    return {"workload": "floor256 lattice, 16 scans of 1024x512 equirect depth+opacity per step",
            "ms_per_step": ms, "rays_per_s": n_rays / (ms / 1000.0),
            "voxel_pass_min_bytes_per_scan": bytes_scan, "occupied_voxels_after": occ}


def stereo_bench(roam, F, torch, stream):
    """Stereoscopic roaming on the floor256 scene: a 120-frame walk, both
    eyes (1280x720 perspective, 90 degree FOV, 64 mm apart) rendered in one
    graph-replayed BF16 call per frame; per-frame device latency."""
    import numpy as np
    from paper_2208_02705_gb300.roaming import roam_frames
    wl = F.floor256(views="equirect")
    r = roam.Roam(torch.cuda.current_device())
    r.load_workload(wl)
    poses = F.roaming_path(wl.scene, 2, 128)
    gopts = roam.render_opts(wl.delta, wl.n_max, precision=roam.ROAM_BF16, use_graph=True)
    roam_frames(r, poses[:8], gopts, stream=stream)           # capture + warm-up
    times, _ = roam_frames(r, poses[8:], gopts, stream=stream)
    r.close()
    t = np.array(times)
    return {"workload": "floor256_kd512_w64h3, 120-frame walk, 2 x 1280x720 perspective eyes per frame",
            "frame_ms_median": float(np.median(t)), "frame_ms_p95": float(np.percentile(t, 95)),
            "fps_at_median": 1000.0 / float(np.median(t))}


def distill_bench(roam, F, torch, args, stream, peaks):
    """One distillation step (Eq. 7) on the floor256 partition: the global
    360NeRF teacher (8x256, 595,844 parameters, FP32 cuBLAS layers) labels
    256 points per field in each of the 512 fields; the W=64/H=3 students
    are evaluated (BF16 tensor cores), the loss and its output gradient
    formed, the adjoint run (BF16 tensor cores) and Adam applied."""
    import numpy as np
    wl = F.floor256(views="equirect")
    I = 256
    p, d, f = F.distill_points(wl.scene, wl.part, 2, I)
    pt, dt = torch.from_numpy(p).cuda(), torch.from_numpy(d).cuda()
    ft = torch.from_numpy(f.astype(np.int16)).cuda()
    student = F.xavier_weights(2, F.ROLE_STUDENT, wl.part.n_fields, wl.W, wl.H, bias_scale=0.1)
    r = roam.Roam(torch.cuda.current_device())
    r.load_grid(wl.scene.bits, wl.scene.dims, wl.scene.origin, wl.scene.vox)
    r.load_fields(wl.part.field_of_rank, wl.affine)
    r.load_weights(student, wl.W, wl.H, 2.0)
    r.teacher_load(F.teacher_weights(3, bias_scale=0.1), F.scene_affine(wl.scene))
    losses = []

    def step(k):
        return r.distill_step(pt, dt, ft, float(I), lr=1e-3, step=k, precision=roam.ROAM_BF16,
                              teacher_precision=roam.ROAM_BF16, stream=stream)

    for k in range(1, 4):
        step(k)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    steps = max(5, args.steps)
    r.profile(True)
    a.record(stream)
    for k in range(4, 4 + steps):
        losses.append(step(k))
    b.record(stream)
    b.synchronize()
    prof = r.profile_read()
    r.profile(False)
    ms = a.elapsed_time(b) / steps
    # the teacher alone, in both arithmetics
    n = int(p.shape[0])
    teacher = {}
    peak = peaks.get("bf16_tflops", 1900.0)
    for name, prec in (("bf16_tcgen05", roam.ROAM_BF16), ("f32_simt", roam.ROAM_F32)):
        for _ in range(2):
            r.teacher_eval(pt, dt, precision=prec, stream=stream)
        a.record(stream)
        for _ in range(steps):
            r.teacher_eval(pt, dt, precision=prec, stream=stream)
        b.record(stream)
        b.synchronize()
        t_ms = a.elapsed_time(b) / steps
        tf = 2.0 * 595844 * n / (t_ms / 1000.0) / 1e12
        teacher[name] = {"ms": t_ms, "tflops": tf}
        if prec == roam.ROAM_BF16:
            teacher[name]["frac_of_bf16_peak"] = tf / peak
            teacher[name]["peak"] = "measured bf16 burst" if peaks else "fallback"
    # a larger batch (the teacher's own roofline: many tiles per SM)
    n_big = 1 << 20
    rng = np.random.default_rng(5)
    pb = torch.from_numpy(p[rng.integers(0, n, n_big)]).cuda()
    db = torch.from_numpy(d[rng.integers(0, n, n_big)]).cuda()
    for _ in range(2):
        r.teacher_eval(pb, db, precision=roam.ROAM_BF16, stream=stream)
    a.record(stream)
    for _ in range(steps):
        r.teacher_eval(pb, db, precision=roam.ROAM_BF16, stream=stream)
    b.record(stream)
    b.synchronize()
    t_ms = a.elapsed_time(b) / steps
    tf = 2.0 * 595844 * n_big / (t_ms / 1000.0) / 1e12
    teacher["bf16_tcgen05_1M_points"] = {"ms": t_ms, "tflops": tf, "frac_of_bf16_peak": tf / peak}
    r.close()
    return {"workload": f"floor256_kd512_w64h3 students, 360NeRF teacher, {I} points per field ({n} per step)",
            "ms_per_step": ms, "points_per_s": n / (ms / 1000.0), "teacher": teacher,
            "loss_first_last": [float(losses[0]), float(losses[-1])],
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in prof.items()},
            "precision": "teacher BF16 tcgen05 (FP32 accumulation), students BF16 tcgen05 forward "
                         "and adjoint, FP32 master weights"}


def partition_bench(roam, F, torch, args, stream, flush):
    """Partitions of the floor256 scene into 512 fields compared on the
    1024x512 equirect view (W=64/H=3, BF16): kd (median splits), Alg. 1
    stage II (anchor + nearest neighbours, computed on the GPU) and the
    uniform 8x8x8 split -- samples per field, tile padding and MLP time."""
    import numpy as np
    wl = F.floor256(views="equirect")
    out = {"workload": "floor256, 512 fields, W=64 H=3, 1024x512 equirect, BF16", "partitions": {}}
    r = roam.Roam(torch.cuda.current_device())
    r.load_grid(wl.scene.bits, wl.scene.dims, wl.scene.origin, wl.scene.vox)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    labels, boxes = r.assign_fields(512, stream=stream)
    b.record(stream)
    b.synchronize()
    alg1 = F.Partition(boxes.cpu().numpy().reshape(512, 2, 3).astype(np.int32),
                       labels.cpu().numpy().view(np.uint16).copy())
    out["alg1_assign_ms"] = a.elapsed_time(b)
    parts = {"kd_median": wl.part, "alg1_nearest": alg1, "uniform_8x8x8": F.uniform_partition(wl.scene, (8, 8, 8))}
    w = F.xavier_weights(2, F.ROLE_TEACHER, 512, 64, 3)
    for name, part in parts.items():
        r.load_fields(part.field_of_rank, F.field_affine(wl.scene, part))
        r.load_weights(w, 64, 3, wl.sigma_scale)
        opts = roam.render_opts(wl.delta, wl.n_max, precision=roam.ROAM_BF16)
        cnt, recs = r.march(wl.cams, roam.render_opts(wl.delta, wl.n_max))
        k = torch.arange(wl.n_max, device=cnt.device)[None, :] < cnt[:, None].long()
        per = torch.bincount((recs[k].long() >> 16) & 0xffff, minlength=512).cpu().numpy()
        used = per[per > 0]
        tiles = int(np.sum(np.ceil(used / 128 / 4) * 4))
        for _ in range(3):
            r.render(wl.cams, opts, stream=stream)
        torch.cuda.synchronize()
        r.profile(True)
        tot, frame = time_steps(r, wl.cams, opts, max(3, args.steps // 2), 0, flush, stream)
        prof = r.profile_read()
        r.profile(False)
        st = r.get_stats()
        steps = max(3, args.steps // 2)
        out["partitions"][name] = {
            "fields_with_samples": int(used.size), "marched_samples_max_per_field": int(per.max()),
            "marched_samples_mean_per_field": float(used.mean()), "cv": float(used.std() / used.mean()),
            "tiles_all_marched": tiles, "tile_fill": float(per.sum() / (tiles * 128)),
            "frame_ms": statistics.median(frame), "mlp_ms": prof["mlp_bf16_tcgen05"][1] / steps,
            "evaluated_per_frame": int(st.n_samples)}
    r.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="roam", choices=["roam", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--quick", action="store_true",
                    help="headline loop only (no FP32 comparison, accuracy, e2e or CPU baseline): for profilers")
    ap.add_argument("--views", default="both", choices=["both", "equirect", "perspective"])
    ap.add_argument("--precision", default=None, choices=["bf16", "f32"],
                    help="with --quick: the arithmetic of the timed loop (default BF16 tensor cores)")
    ap.add_argument("--rounds", default=None,
                    help="FIRST,LATER: round sizes of the headline render instead of the library's tuner "
                         "(profilers use it for a fixed launch sequence)")
    ap.add_argument("--section", default=None, choices=["train", "distill"],
                    help="run one secondary section alone and print its JSON (for profilers)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch

    import fixtures as F
    import paper_2208_02705_gb300 as roam

    if args.section is not None:
        stream = torch.cuda.current_stream()
        if args.section == "train":
            res = train_step_bench(roam, F, torch, F.floor256(), args, stream)
        else:
            pk = {}
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
                pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
            res = distill_bench(roam, F, torch, args, stream, pk)
        print(json.dumps({"section": args.section, **res}), flush=True)
        return 0

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = F.floor256(views=args.views)
    r = roam.Roam(local)
    r.load_workload(wl)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB > L2
    views = [{"equirect": "equirect 1024x512", "perspective": "perspective 1920x1080 fov 90"}[m]
             for m in (["equirect", "perspective"] if args.views == "both" else [args.views])]

    if args.quick and args.precision == "f32":
        head_prec, dtype = roam.ROAM_F32, "f32"
    else:
        try:
            r.render(wl.cams, roam.render_opts(wl.delta, wl.n_max, precision=roam.ROAM_BF16))
            head_prec, dtype = roam.ROAM_BF16, "bf16"
        except roam.RoamError:
            head_prec, dtype = roam.ROAM_F32, "f32"
    # round sizes from the library's tuner (set-up, before the timed region)
    if args.rounds:
        R0, R = (int(x) for x in args.rounds.split(","))
    else:
        R, R0, _ = r.tune_round_size(wl.cams, roam.render_opts(wl.delta, wl.n_max, precision=head_prec),
                                     stream=stream)
    opts = roam.render_opts(wl.delta, wl.n_max, precision=head_prec, round_size=R, first_round_size=R0)

    # ---- headline: K timed steps, event-timed per-kernel record on ----
    for _ in range(args.warmup):
        r.render(wl.cams, opts, stream=stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    r.profile(True)
    total_ms, per = time_steps(r, wl.cams, opts, args.steps, 0, flush, stream)
    prof = r.profile_read()
    r.profile(False)
    torch.cuda.synchronize()
    clocks = clk.stop()
    st = r.get_stats()
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    used_per_step = st.n_used
    evaluated_per_step = st.n_samples
    # this library's kernels in the timed region, from the per-launch event
    # record: one launch per recorded entry, and the bucket entry is two
    # kernels (scan, scatter)
    gpu_launches = int(sum(v[0] for v in prof.values()) + prof.get("bucket", (0, 0.0))[0])
    value = world * used_per_step * args.steps / (total_ms / 1000.0)
    ms_per_step = total_ms / args.steps
    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "metric": METRIC, "value": value, "unit": UNIT, "dtype": dtype,
                              "ms_per_step": ms_per_step, "views": views, "kernels": prof, "clocks": clocks,
                              "evaluated_per_step": int(evaluated_per_step), "rounds": int(st.n_rounds),
                              "round_sizes": [R0, R]}),
                  flush=True)
        r.close()
        return 0

    # ---- per-view frame times and the FP32 SIMT form ----
    frame = {}
    for prec, tag in ((head_prec, dtype), (roam.ROAM_F32, "f32")):
        if tag in frame:
            continue
        o = roam.render_opts(wl.delta, wl.n_max, precision=prec)
        frame[tag] = {}
        for cam, name in zip(wl.cams, ("equirect_1024x512", "persp_1920x1080")):
            tot, per_v = time_steps(r, [cam], o, max(3, args.steps // 2), 2, flush, stream)
            frame[tag][name] = statistics.median(per_v)
    o32 = roam.render_opts(wl.delta, wl.n_max, precision=roam.ROAM_F32)
    t32, _ = time_steps(r, wl.cams, o32, max(3, args.steps // 2), 2, flush, stream)
    st32 = r.get_stats()
    f32_value = st32.n_used * max(3, args.steps // 2) / (t32 / 1000.0)

    # ---- roofline of the dominant kernel, from the live event record ----
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    mlp_key = "mlp_bf16_tcgen05" if head_prec == roam.ROAM_BF16 else "mlp_f32_simt"
    shares = {k: {"launches": v[0], "ms": round(v[1], 4), "share": round(v[1] / sum(x[1] for x in prof.values()), 4)}
              for k, v in prof.items()}
    # the HBM-side kernels: algorithmic bytes over the timed region's launches
    # (lower bounds: the march writes a 4 B record per evaluated sample and
    # 64 B of ray state per ray; the bucket reads 8 B and writes 4 B per
    # sample; the composite reads 16 B of (sigma, rgb) and a 4 B record per
    # sample and writes 20 B per ray), against the measured copy rate
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    n_rays_step = sum(c.n_pixels for c in wl.cams)
    alg = {"march": 4 * evaluated_per_step + 64 * n_rays_step, "bucket": 12 * evaluated_per_step,
           "composite": 20 * evaluated_per_step + 20 * n_rays_step}
    for k, nbytes in alg.items():
        if k in prof and prof[k][1] > 0:
            gbs = nbytes * args.steps / (prof[k][1] / 1000.0) / 1e9
            shares[k].update({"alg_bytes_per_step": int(nbytes), "alg_gbs": round(gbs, 1),
                              "frac_of_hbm": round(gbs / hbm, 4)})
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else mlp_key
    launches, mlp_ms = prof.get(mlp_key, (0, float("nan")))
    flops = 2.0 * macs_per_sample(wl.W, wl.H) * evaluated_per_step * args.steps
    achieved = flops / (mlp_ms / 1000.0) / 1e12
    if head_prec == roam.ROAM_BF16:
        peak, bound, src = peaks.get("bf16_tflops", 1900.0), "tensor", "measured bf16 burst" if peaks else "fallback"
    else:
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        bound, src = "alu", "152 SMs x 128 FP32 lanes x 2 FLOP x max SM clock"
    # DRAM traffic per launch: bytes per evaluated sample from an ncu capture of
    # this kernel on the 1024x512 equirect view of the same scene (dram bytes
    # read + written over one render's 4 launches: 254.1 MB for 8,372,992
    # evaluated samples), scaled by the samples of this run's launches
    traffic = 30.35 * evaluated_per_step * args.steps / launches if (launches and head_prec == roam.ROAM_BF16) \
        else None
    roofline = {"kernel": mlp_key, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "peak_source": src, "traffic": traffic,
                "flops_per_sample": 2 * macs_per_sample(wl.W, wl.H), "launches": launches,
                "dominant_kernel": dom, "kernel_shares": shares}

    # ---- accuracy against the FP64 oracle on sampled pixels ----
    acc = {}
    if rank == 0:
        import oracle as O
        g = O.Grid(wl.scene, wl.part)
        rays = oracle_sample_rays(wl, 3000, 7)
        ref = O.render(g, wl.weights, wl.affine, wl.W, wl.H, wl.sigma_scale, F.camera_array(wl.cams), rays,
                       wl.delta, wl.n_max)
        starts = np.concatenate([[0], np.cumsum([c.n_pixels for c in wl.cams])])
        gi = starts[rays[:, 0].astype(np.int64)] + rays[:, 1].astype(np.int64)
        for prec, tag in ((head_prec, dtype), (roam.ROAM_F32, "f32")):
            rgb, _, _ = r.render(wl.cams, roam.render_opts(wl.delta, wl.n_max, precision=prec))
            torch.cuda.synchronize()
            acc[tag] = accuracy(r, roam, F, g, wl, rays, prec, rgb.cpu().numpy()[gi].astype(np.float64), ref)

    # ---- end to end through the C ABI with host buffers ----
    n_pix = sum(c.n_pixels for c in wl.cams)
    rgb_h = torch.empty((n_pix, 3), dtype=torch.float32, pin_memory=True).numpy()
    dep_h = torch.empty(n_pix, dtype=torch.float32, pin_memory=True).numpy()
    op_h = torch.empty(n_pix, dtype=torch.float32, pin_memory=True).numpy()
    for _ in range(2):
        r.render_host(wl.cams, opts, rgb_h, dep_h, op_h)
    e2e_times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r.render_host(wl.cams, opts, rgb_h, dep_h, op_h)
        e2e_times.append(time.perf_counter() - t0)
    e2e_value = world * used_per_step * args.steps / sum(e2e_times)
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 64 * len(wl.cams),
           "d2h_bytes_per_step": 20 * n_pix, "ms_per_step": 1000 * sum(e2e_times) / args.steps}

    # ---- training step: 65,536 random rays of 16 equirect views, targets
    # from the teacher weights + N(0, 0.01^2), student weights trained ----
    train = None
    if rank == 0:
        train = train_step_bench(roam, F, torch, wl, args, stream)

    large = multiview = occupancy = stereo = partition = distill = None
    if rank == 0:
        distill = distill_bench(roam, F, torch, args, stream, peaks)
        large = large_scene_bench(roam, F, torch, args, stream, flush, peaks)
        multiview = multiview_bench(roam, F, torch, args, stream, flush)
        occupancy = occupancy_bench(roam, F, torch, args, stream)
        stereo = stereo_bench(roam, F, torch, stream)
        partition = partition_bench(roam, F, torch, args, stream, flush)

    cpu = None
    if rank == 0 and world == 1:
        v, cores, desc, rays_s = cpu_oracle_rate(wl, args.cpu_seconds)
        one, frames = cpu_oracle_frames(wl, rays_s)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "rays_per_s": rays_s, "one_core": one, "frames": frames}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": dtype, "data": "synthetic (seeded generators)",
                "config": workload_config(wl, views),
                "samples_per_step": {"composited": int(used_per_step), "evaluated": int(evaluated_per_step),
                                     "rays": int(st.n_rays), "rounds": int(st.n_rounds),
                                     "round_sizes_tuned": {"first": R0, "later": R}},
                "frame_ms": frame,
                "fp32_simt": {"value": f32_value, "unit": UNIT, "ms_per_step": t32 / max(3, args.steps // 2)},
                "accuracy_vs_oracle": acc, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "train_step": train, "large_scene": large, "multi_view": multiview,
                "occupancy_update": occupancy, "stereo_roaming": stereo,
                "partitions": partition, "distillation": distill,
                "gpu_launches": gpu_launches, "clocks": clocks}
        print(json.dumps(line), flush=True)
    r.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
