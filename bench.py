#!/usr/bin/env python3
"""Benchmark of the reconstruction hot path on one GB300 (or N replicas).

One step is the whole path over one batch of the 1920x1080, 16-deep workload
(33,177,600 seeded synthetic samples, FP32 colours): empty the deep buffer,
ingest the batch (section 4), estimate gradients (4.1), reproject to t_now
(6.2), filter every pixel (5.1, 5.2) and finalise the tile statistics (4.2,
6.1). The batch (1.3 GB) and the buffers are far larger than L2, so no flush
is needed between steps.

The same run also times the FP16- and BF16-stored forms of that step, the
forward+backward of the 512x512x8 differentiation workload, the batched form
(48 streams, one persistent launch in a CUDA graph, against 48 sequential
single-stream launches), the step end to end through the Python API with the
batch in pinned host memory (FP32 and FP16 colours), adaptive footprints
(section 6.2), the tile error and gain control (6.1, 4.1), the global FIFO
buffer against the per-pixel queues (5.2, on the 1024x1024x8 workload), the
device's measured FP32 and ex2 rates (the filter's roofline), and the CPU
oracle's whole path on the whole image (every host core, and one), whose
image also gives the end-to-end parity of the GPU image.

Prints one JSON line. --impl reference times the CPU oracle instead (its whole
path on the whole image each step, on every host core).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "c3_1920x1080x16"
METRIC = "1080p reconstructions/s (16-deep buffer)"
T_NOW = 1.0
# kernels launched per call of the step (memsets and copies excluded), as the
# launch sequences in csrc/ issue them
LAUNCHES = {"ingest": 7, "gradients": 2, "reproject": 7, "reconstruct": 2, "feedback": 1}
STAGES = ["ingest", "gradients", "reproject", "reconstruct", "feedback"]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank value over all ranks (the whole job is as slow as
    its slowest replica)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        ok = [r for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        sm = [float(r[0]) for r in ok]
        mx = [float(r[1]) for r in ok if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in ok for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


# ------------------------------------------------------------------------------ workload bytes
# DRAM bytes (read + written) of one k_filter launch on the 1920x1080x16 workload with FP32
# colours, from one ncu capture, keyed by the sha256 of the sources the kernel was built from
# (csrc/k_filter.cu, csrc/afr_internal.cuh). Command (after the same command exited 0 without ncu):
#   ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum --clock-control none \
#       -c 20 --csv --log-file launches.csv python bench.py --profile --steps 1 --warmup 0 --no-cpu-baseline
# A changed kernel has no entry, and the line then reports null.
FILTER_TRAFFIC = {
    ("ac16c6118738c34c92934d753be73dd680a508500a2e32bf5f83788584569732",
     "19da060f812c9aa7e1bdab083bd343179dc94de2746a1a1f3fa7d22a8f801d02"): 0.988e9 + 0.031e9,
}


def filter_traffic(args, color):
    """(bytes, source) for roofline.traffic: a figure passed on the command line, else the
    recorded capture of this exact kernel source on the 1920x1080x16 FP32 workload, else null."""
    if args.filter_traffic is not None:
        return args.filter_traffic, "--filter-traffic"
    if args.workload != WORKLOAD or color != "f32":
        return None, "no capture for this workload"
    import hashlib
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2510_15876_gb300", "csrc")
    key = tuple(hashlib.sha256(open(os.path.join(csrc, f), "rb").read()).hexdigest()
                for f in ("k_filter.cu", "afr_internal.cuh"))
    if key in FILTER_TRAFFIC:
        return FILTER_TRAFFIC[key], "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of this kernel source"
    return None, "kernel source changed since the last capture"


def stage_bytes(P, n_batch, resident, frame, csize, ntiles):
    """Algorithmic HBM bytes of each stage (each operand read or written once).
    csize: stored colour bytes (16 FP32 / 8 16-bit). A buffered sample is
    x, y, mx, my (16 B), t (4), depth (4), seq (4) and its colour; a frame
    record is x', y', a^2, bin column (16 B), its colour and seq (4)."""
    ingest = n_batch * (16 + csize + 8) + resident * (16 + 4 + 4 + 4 + csize) + P * 8
    grads = resident * (4 + 4 + csize) + P * (4 + 4 + 16 + 4 + 16) + ntiles * 64
    reproj = resident * (16 + 4 + 4 + csize) + frame * (16 + csize + 4) + P * 12
    recon = frame * (16 + csize) + P * (16 + 8 + 4 + 8 + 16)
    feedback = ntiles * (64 + 32)
    return {"ingest": ingest, "gradients": grads, "reproject": reproj, "reconstruct": recon, "feedback": feedback}


def pairs_of(off, W, H, R):
    """Sample-pixel pairs the filter evaluates (integer disc footprint)."""
    cnt = np.diff(off.astype(np.int64)).reshape(H, W)
    tot = 0
    for dy in range(-R, R + 1):
        hw = int(np.floor(np.sqrt(R * R - dy * dy) + 1e-9))
        src = np.roll(cnt, -dy, axis=0)
        if dy > 0:
            src[H - dy:] = 0
        elif dy < 0:
            src[:-dy] = 0
        cs = np.concatenate([np.zeros((H, 1), np.int64), np.cumsum(src, axis=1)], axis=1)
        x = np.arange(W)
        tot += int((cs[:, np.minimum(W - 1, x + hw) + 1] - cs[:, np.maximum(0, x - hw)]).sum())
    return tot


def arm_config(workload, n, seed, world):
    """The workload description both arms print."""
    return {"workload": f"{workload} (1920x1080 image, 16-deep buffer, {n} samples per batch, 256 moving discs, "
                        f"10% occlusion-edge pixels, seed {seed})",
            "global_batch": n * world, "l2": "inputs larger than L2 (1.3 GB batch), no flush",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


# ------------------------------------------------------------------------------ our arm
def run_ours(args, rank, world):
    import torch
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    from workloads import scenes

    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl", device_id=dev)
        dist = dist_mod

    seed = rank
    t0 = time.time()
    scene, batch = scenes.config_stream(args.workload, seed)
    gen_s = time.time() - t0
    W, H, b = scene.width, scene.height, scene.spec.depth
    n = batch["pos"].shape[0]
    P = W * H

    def step(r, pos, col, mo, out, tiles, ev=None):
        if ev is not None:
            ev[0].record()
        r.reset()
        r.insert(pos, col, mo)
        if ev is not None:
            ev[1].record()
        r.estimate_gradients(T_NOW)
        if ev is not None:
            ev[2].record()
        r.reproject(T_NOW)
        if ev is not None:
            ev[3].record()
        r.reconstruct(T_NOW, out=out)
        if ev is not None:
            ev[4].record()
        r.tile_feedback(out=tiles)
        if ev is not None:
            ev[5].record()

    def step_overlap(r, pos, col, mo, out, tiles):
        # one step alone: gradients and tile statistics on a side stream while
        # the samples are reprojected, then the filter (Reconstructor.refresh)
        r.reset()
        r.insert(pos, col, mo)
        r.refresh(T_NOW, out=out, tiles=tiles)

    class Pipelined:
        """The timed steps: step k + 1's insert runs on an ingest stream. Its
        binning (counting, offsets, bucket records: the context's scratch)
        starts at once, beside step k's gradients and reprojection; its reset
        and commit wait until those are done with the sample buffers
        (afr_insert_samples_ex with reads_done) and run beside step k's
        filter, which reads none of them. Every step still does all of a1-a6."""

        def __init__(self, r):
            self.r = r
            self.ingest = torch.cuda.Stream(dev, priority=-1)
            self.reads_done, self.ingested = torch.cuda.Event(), torch.cuda.Event()
            self.reads_done.record(torch.cuda.current_stream())

        def step(self, pos, col, mo, out, tiles, ready=None, consumed=None):
            main = torch.cuda.current_stream()
            if ready is not None:
                self.ingest.wait_event(ready)
            self.r.insert(pos, col, mo, stream=self.ingest, reset=True, queues_free=self.reads_done)
            if consumed is not None:
                consumed.record(self.ingest)
            self.ingested.record(self.ingest)
            main.wait_event(self.ingested)
            self.r.refresh(T_NOW, out=out, tiles=tiles, reads_done=self.reads_done)

    results = {}
    gpu_image = None
    hbm_peak, peak_kind = _peaks()
    forms = ["f32", "f16", "bf16"] if not (args.quick or args.profile) else ["f32"]
    if args.color:
        forms = [args.color]
    keep = None
    for ct in forms:
        dtype = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[ct]
        rec = Reconstructor(W, H, b, color_type=ct, device=dev)
        rec.reserve(n)
        pos, col, mo = to_device_batch(batch, dev, dtype)
        out = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
        tiles = torch.empty((rec.n_tiles, 8), dtype=torch.float32, device=dev)
        pipe = Pipelined(rec)
        for _ in range(args.warmup):
            pipe.step(pos, col, mo, out, tiles)
        for _ in range(args.warmup):
            step_overlap(rec, pos, col, mo, out, tiles)
            step(rec, pos, col, mo, out, tiles)
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]

        def timed(fn):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for k in range(args.steps):
                fn(k)
            e.record()
            torch.cuda.synchronize()
            return max_over_ranks(a.elapsed_time(e), dist, dev) / args.steps

        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if ct == forms[0] else None
        if sampler:
            sampler.start()
        rec.profile_filter(True)
        pipe.reads_done.record()
        ms_pipe = timed(lambda k: pipe.step(pos, col, mo, out, tiles))
        filter_pipe = rec.profile_read()
        rec.profile_filter(False)
        # one step at a time (the filter runs alone), then the stages in
        # series for the per-stage times
        rec.profile_filter(True)
        ms_alone = timed(lambda k: step_overlap(rec, pos, col, mo, out, tiles))
        filter_ms = rec.profile_read()
        rec.profile_filter(False)
        ms_serial = timed(lambda k: step(rec, pos, col, mo, out, tiles, evs[k]))
        clocks = sampler.stop() if sampler else None
        if dist:
            dist.barrier()
        st_ms = {s: sum(e[i].elapsed_time(e[i + 1]) for e in evs) / args.steps for i, s in enumerate(STAGES)}
        results[ct] = {"ms_per_step": ms_pipe, "unpipelined_ms_per_step": ms_alone, "serial_ms_per_step": ms_serial,
                       "stage_ms": st_ms, "info": rec.query(),
                       "clocks": clocks, "csize": 16 if ct == "f32" else 8,
                       "filter_ms": sum(filter_ms) / max(1, len(filter_ms)),
                       "filter_ms_pipelined": sum(filter_pipe) / max(1, len(filter_pipe))}
        del pipe
        if ct == forms[0]:
            keep = (rec, pos, col, mo, out, tiles)
            gpu_image = out.cpu().numpy().reshape(-1, 4).astype(np.float64)   # the last step's image
        else:
            rec.close()
            del pos, col, mo
            torch.cuda.empty_cache()

    r0 = results[forms[0]]
    rec = keep[0]
    if args.profile:
        if rank == 0:
            print(json.dumps({"workload": args.workload, "color": forms[0], "ms_per_step": r0["ms_per_step"],
                              "unpipelined_ms_per_step": r0["unpipelined_ms_per_step"],
                              "serial_ms_per_step": r0["serial_ms_per_step"], "stage_ms": r0["stage_ms"],
                              "filter_kernel_ms": r0["filter_ms"], "filter_kernel_ms_pipelined": r0["filter_ms_pipelined"],
                              "info": r0["info"]}),
                  flush=True)
        rec.close()
        return

    info = r0["info"]
    off, _, _ = rec.export_frame()
    pairs = pairs_of(off, W, H, 4)
    resident, frame = int(info["resident"]), int(info["frame"])
    by = stage_bytes(P, n, resident, frame, r0["csize"], rec.n_tiles)
    step_ms = r0["ms_per_step"]
    st = r0["stage_ms"]
    total_bytes = sum(by.values())
    flops = pairs * 16.0
    from paper_2510_15876_gb300.api import measure_alu_peaks
    alu = measure_alu_peaks()
    fp32_peak = max(alu["fma_tflops"], alu["fma2_tflops"])
    ach = flops / (r0["filter_ms"] * 1e-3) / 1e12
    ex2_rate = pairs / (r0["filter_ms"] * 1e-3) / 1e12
    traffic, traffic_src = filter_traffic(args, forms[0])
    roof = {"bound": "alu", "kernel": "k_filter", "kernel_ms": round(r0["filter_ms"], 4), "achieved": round(ach, 2),
            "peak": round(fp32_peak, 1), "unit": "TFLOP/s", "frac": round(ach / fp32_peak, 4),
            "traffic": traffic,
            "traffic_source": traffic_src,
            "peak_source": f"measured in this run (afr_measure_alu_peaks, {alu['sms']} SMs): scalar FMA "
                           f"{alu['fma_tflops']:.1f}, paired FMA {alu['fma2_tflops']:.1f} TFLOP/s; the larger is the peak",
            "ex2": {"achieved_tops": round(ex2_rate, 3), "peak_tops": round(alu["ex2_tops"], 3),
                    "frac": round(ex2_rate / alu["ex2_tops"], 4), "what": "one ex2.approx per sample-pixel pair"}
            if alu["ex2_tops"] < alu["fma_tflops"] else None,
            "work": f"{pairs} sample-pixel pairs x 16 FLOP",
            "timed": "CUDA events around each k_filter launch of the unpipelined timed steps (the kernel alone on "
                     "the GPU); in the pipelined steps it shares the SMs with the next batch's ingest",
            "kernel_ms_pipelined": round(r0["filter_ms_pipelined"], 4)}
    stage_hbm = {s: round(by[s] / (st[s] * 1e-3) / 1e9 / hbm_peak, 4) for s in STAGES}

    # adaptive footprints (section 6.2): successive reconstructions of the
    # same frame view, each sizing footprints from the previous one's coverage
    from paper_2510_15876_gb300 import _lib as L
    adapt, tile_err, camera = {}, {}, {}
    if not args.quick:
        _, pos, col, mo, out, tiles = keep
        step(rec, pos, col, mo, out, tiles)
        flags = L.AFR_RECON_ADAPTIVE_SUPPORT
        rec.reconstruct(T_NOW, out=out, flags=flags | L.AFR_RECON_COVERAGE_RESET)
        for _ in range(5):
            rec.reconstruct(T_NOW, out=out, flags=flags)
        torch.cuda.synchronize()
        s3, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s3.record()
        for _ in range(args.steps):
            rec.reconstruct(T_NOW, out=out, flags=flags)
        e3.record()
        torch.cuda.synchronize()
        radius = np.floor(rec.export_map(L.AFR_MAP_FOOTPRINT) + 0.5).astype(int)
        cov = rec.export_map(L.AFR_MAP_COVERAGE)
        holes_fixed = int((rec.reconstruct(T_NOW)[..., 3] == 0).sum())
        adapt = {"ms_per_reconstruct": round(s3.elapsed_time(e3) / args.steps, 4),
                 "fixed_ms_per_reconstruct": round(st["reconstruct"], 4),
                 "footprint_radius_counts": {str(k): int((radius == k).sum()) for k in np.unique(radius)},
                 "median_samples_per_footprint": float(np.median(cov)),
                 "holes_fixed_R4": holes_fixed,
                 "what": "afr_reconstruct with AFR_RECON_ADAPTIVE_SUPPORT after 6 warm-up images (coverage converged)"}
        rec.reconstruct(T_NOW, out=out, flags=flags)
        torch.cuda.synchronize()
        adapt["holes_adaptive"] = int((out[..., 3] == 0).sum())
        # tile error and gain control (sections 6.1, 4.1) on the same buffer
        E, gain = rec.tile_error(0.5, 0.5, 1.0)
        s4, e4 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s4.record()
        for _ in range(args.steps):
            rec.tile_error(0.5, 0.5, 1.0)
        e4.record()
        torch.cuda.synchronize()
        te_out = (torch.empty_like(E), torch.empty(5, dtype=torch.float32, device=dev))
        s6, e6 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s6.record()
        for _ in range(args.steps):
            rec.tile_error(0.5, 0.5, 1.0, out=te_out, gain_on_device=True)
        e6.record()
        torch.cuda.synchronize()
        # camera-matrix reprojection (section 6.2) of the same batch with hit
        # points, against the screen-motion reprojection
        rec_w = Reconstructor(W, H, b, world_points=True, device=dev)
        gen = torch.Generator(device=dev)
        gen.manual_seed(0)
        hits = torch.rand((n, 4), generator=gen, device=dev) * torch.tensor([4.0, 4.0, 4.0, 0.0], device=dev) \
            - torch.tensor([2.0, 2.0, -2.0, 0.0], device=dev)
        rec_w.insert(pos, col, mo, world=hits)
        vp = np.array([[1.2, 0.1, 0.05, 0.02], [-0.05, 1.3, 0.1, -0.1], [0, 0, 1, 0], [0.01, 0.02, 0.4, 0.3]],
                      np.float32)
        cam_ms = {}
        for name, fn in (("screen_motion", lambda: rec_w.reproject(T_NOW)),
                         ("camera", lambda: rec_w.reproject_camera(T_NOW, vp))):
            fn()
            torch.cuda.synchronize()
            s5, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s5.record()
            for _ in range(args.steps):
                fn()
            e5.record()
            torch.cuda.synchronize()
            cam_ms[name] = round(s5.elapsed_time(e5) / args.steps, 4)
        camera = {"reproject_ms": cam_ms, "frame_records": int(rec_w.query()["frame"]),
                  "what": "1080p16 batch with random hit points in [-2, 2]^2 x [2, 6], perspective camera"}
        rec_w.close()
        del hits
        torch.cuda.empty_cache()
        tile_err = {"ms_per_call": round(s4.elapsed_time(e4) / args.steps, 4),
                    "device_ms_per_call": round(s6.elapsed_time(e6) / args.steps, 4), "tiles": int(E.numel()),
                    "gain": {k: round(v, 6) for k, v in gain.items()},
                    "what": "afr_tile_error (kappa = lambda = 0.5, no occlusion data); ms_per_call through "
                            "Reconstructor.tile_error, including the device-to-host read of the gain record; "
                            "device_ms_per_call with the outputs preallocated and the gain left on the device"}

    # end to end through the public API, batch in pinned host memory: every
    # step copies its inputs host -> device and its image device -> host inside
    # the timed region; step k+1's input copy (on a copy stream, into the other
    # of two device buffers) overlaps step k's compute, and the steps are
    # pipelined as in the device-resident timing
    import torch as _t

    def measure_e2e(rec_e, dev_bufs, out_e, tiles_e, color_dtype):
        hp = {"pos": _t.from_numpy(np.ascontiguousarray(batch["pos"], np.float32)).pin_memory(),
              "color": _t.from_numpy(np.ascontiguousarray(batch["color"], np.float32)).to(color_dtype).pin_memory(),
              "motion": _t.from_numpy(np.ascontiguousarray(batch["motion"], np.float32)).pin_memory()}
        host_img = [_t.empty((H, W, 4), dtype=_t.float32).pin_memory() for _ in range(2)]
        bufs = [dev_bufs, tuple(_t.empty_like(t) for t in dev_bufs)]
        comp, copy_s = _t.cuda.current_stream(), _t.cuda.Stream()
        copied = [_t.cuda.Event() for _ in range(2)]
        free = [_t.cuda.Event() for _ in range(2)]

        def issue_copy(j):
            dst = bufs[j % 2]
            copy_s.wait_event(free[j % 2])            # compute of step j - 2 done with this buffer
            with _t.cuda.stream(copy_s):
                for d, k in zip(dst, ("pos", "color", "motion")):
                    d.copy_(hp[k], non_blocking=True)
            copied[j % 2].record(copy_s)

        e2e_pipe = Pipelined(rec_e)

        def e2e_run(k_steps):
            for e in free:
                e.record(comp)
            e2e_pipe.reads_done.record(comp)
            issue_copy(0)
            for k in range(k_steps):
                if k + 1 < k_steps:
                    issue_copy(k + 1)
                # the insert waits for its batch's copy and marks the buffer free
                e2e_pipe.step(*bufs[k % 2], out_e, tiles_e, ready=copied[k % 2], consumed=free[k % 2])
                host_img[k % 2].copy_(out_e, non_blocking=True)
            comp.wait_stream(copy_s)
            comp.wait_stream(e2e_pipe.ingest)

        e2e_run(max(2, args.warmup // 2))
        _t.cuda.synchronize()
        s2, e2 = _t.cuda.Event(enable_timing=True), _t.cuda.Event(enable_timing=True)
        k2 = max(4, args.steps // 2)
        s2.record()
        e2e_run(k2)
        e2.record()
        _t.cuda.synchronize()
        ms = max_over_ranks(s2.elapsed_time(e2) / k2, dist, dev)
        # the copy alone, for reference
        c0, c1 = _t.cuda.Event(enable_timing=True), _t.cuda.Event(enable_timing=True)
        c0.record(copy_s)
        with _t.cuda.stream(copy_s):
            for d, k in zip(bufs[1], ("pos", "color", "motion")):
                d.copy_(hp[k], non_blocking=True)
        c1.record(copy_s)
        _t.cuda.synchronize()
        h2d_b = sum(hp[k].numel() * hp[k].element_size() for k in hp)
        d2h_b = host_img[0].numel() * 4
        return ms, h2d_b, d2h_b, h2d_b / (c0.elapsed_time(c1) * 1e-3) / 1e9

    _, pos, col, mo, out, tiles = keep
    e2e_ms, h2d, d2h, h2d_gbs = measure_e2e(rec, (pos, col, mo), out, tiles, _t.float32)
    rec.close()
    del keep, pos, col, mo
    _t.cuda.empty_cache()
    e2e_f16 = None
    if not (args.quick or args.profile or args.color):
        from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
        rec16 = Reconstructor(W, H, b, color_type="f16", device=dev)
        rec16.reserve(n)
        bufs16 = to_device_batch(batch, dev, _t.float16)
        out16 = _t.empty((H, W, 4), dtype=_t.float32, device=dev)
        tiles16 = _t.empty((rec16.n_tiles, 8), dtype=_t.float32, device=dev)
        ms16, h2d16, d2h16, gbs16 = measure_e2e(rec16, bufs16, out16, tiles16, _t.float16)
        e2e_f16 = {"value": round(world * 1000.0 / ms16, 3), "unit": "reconstructions/s", "h2d_bytes_per_step": h2d16,
                   "d2h_bytes_per_step": d2h16, "ms_per_step": round(ms16, 4), "h2d_gb_per_s_alone": round(gbs16, 1),
                   "what": "the same end-to-end step with FP16 colours in the pinned host batch (32 bytes a sample)"}
        rec16.close()
        del bufs16, out16, tiles16
        _t.cuda.empty_cache()

    fb = run_fwd_bwd(args, dev)
    fifo_cmp = None if args.quick else run_fifo_compare(args, dev)
    batched = None if (args.quick or args.no_batched) else run_batched(args, dev)

    value = world * 1000.0 / step_ms
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "reconstructions/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": arm_config(args.workload, n, seed, world),
        "mpixel_per_s": round(P * value / 1e6, 1),
        "samples_filtered_per_s": round(frame * value, 0),
        "pairs_per_step": pairs,
        "hbm_frac_step": round(total_bytes / (step_ms * 1e-3) / 1e9 / hbm_peak, 4),
        "hbm_frac_stage": stage_hbm,
        "step_bytes": total_bytes,
        "stage_ms": {k: round(v, 4) for k, v in st.items()},
        "roofline": roof,
        "recon_per_s_excl_ingest": round(world * 1000.0 / (r0["serial_ms_per_step"] - st["ingest"]), 3),
        "unpipelined_ms_per_step": round(r0["unpipelined_ms_per_step"], 4),
        "serial_ms_per_step": round(r0["serial_ms_per_step"], 4),
        "step_schedule": "timed steps pipelined: step k+1's reset and insert (ingest stream) overlap step k's filter; "
                         "each step's gradients and tile statistics (side stream) overlap its reprojection; "
                         "unpipelined_ms_per_step: one step at a time; serial_ms_per_step: every call in series "
                         "(stage_ms comes from this run)",
        "precision_forms": {ct: {"ms_per_step": round(results[ct]["ms_per_step"], 4),
                                 "unpipelined_ms_per_step": round(results[ct]["unpipelined_ms_per_step"], 4),
                                 "serial_ms_per_step": round(results[ct]["serial_ms_per_step"], 4),
                                 "filter_kernel_ms": round(results[ct]["filter_ms"], 4),
                                 "stage_ms": {k: round(v, 4) for k, v in results[ct]["stage_ms"].items()}}
                            for ct in results},
        "fwd_bwd": fb,
        "adaptive_footprint": adapt,
        "tile_error": tile_err,
        "fifo_vs_queue": fifo_cmp,
        "camera_reprojection": camera,
        "batched": batched,
        "e2e": {"value": round(world * 1000.0 / e2e_ms, 3), "unit": "reconstructions/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 4),
                "h2d_gb_per_s_alone": round(h2d_gbs, 1),
                "how": "pinned host batch copied to one of two device buffers on a copy stream, overlapping the "
                       "previous step's compute; image copied back every step; steps pipelined as in value"},
        "e2e_f16": e2e_f16,
        "gpu_launches": args.steps * sum(LAUNCHES.values()),
        "clocks": r0["clocks"],
        "resident": resident, "frame": frame, "generation_s": round(gen_s, 1),
    }
    if rank == 0 and not args.no_cpu_baseline:
        cb, single, parity = cpu_baseline(scene, batch, args.cpu_seconds, gpu_image, not args.no_single_thread)
        line["cpu_baseline"] = cb
        if single is not None:
            line["cpu_baseline_single_thread"] = single
        line["parity"] = parity
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_fwd_bwd(args, dev):
    """afr_reconstruct + afr_reconstruct_backward (colours and parameters) on
    the 512x512x8 differentiation workload."""
    import torch
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    from workloads import scenes
    sc, batch = scenes.config_stream("c4_512x512x8", 0)
    W, H, b = sc.width, sc.height, sc.spec.depth
    rec = Reconstructor(W, H, b, device=dev)
    rec.insert(*to_device_batch(batch, dev))
    rec.estimate_gradients(T_NOW)
    rec.reproject(T_NOW)
    n_frame = rec.query()["frame"]
    out = torch.empty((H, W, 4), device=dev)
    g = torch.randn((H, W, 4), device=dev)
    theta = (1.0, 0.0, 3.0, 1.0, 0.0, 1.0)
    for _ in range(3):
        rec.reconstruct(T_NOW, theta, out=out)
        rec.backward(g, n_frame=n_frame)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k = max(5, args.steps)
    s.record()
    for _ in range(k):
        rec.reconstruct(T_NOW, theta, out=out)
        rec.backward(g, n_frame=n_frame)
    e.record()
    torch.cuda.synchronize()
    rec.close()
    return {"config": "c4_512x512x8 (512x512, 8-deep, 2,097,152 samples, 32 moving discs)",
            "ms_per_step": round(s.elapsed_time(e) / k, 4),
            "what": "afr_reconstruct + afr_reconstruct_backward (frame colours and 6 parameters)"}


def run_fifo_compare(args, dev):
    """Section 5.2's reconstructor buffer against the per-pixel queues on the
    1024x1024x8 workload (importance-sampled, 8.4M samples): RMS error of the
    reconstruction at t = 1 against a 16-sample-per-pixel ground truth, and
    the time of one step (insert, gradients, reprojection, reconstruction)."""
    import torch
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    from workloads import scenes
    sc, batch = scenes.config_stream("c2_1024x1024x8", 0)
    gt = scenes.ground_truth(sc, T_NOW, 4)
    W, H, b = sc.width, sc.height, sc.spec.depth
    P = W * H
    res = {}
    for name, N in (("per_pixel_queue_b8", 0), ("fifo_4P", 4 * P), ("fifo_8P", 8 * P)):
        rec = Reconstructor(W, H, b, fifo_capacity=N, device=dev)
        pos, col, mo = to_device_batch(batch, dev)
        out = torch.empty((H, W, 4), dtype=torch.float32, device=dev)

        def step():
            rec.reset()
            rec.insert(pos, col, mo)
            rec.estimate_gradients(T_NOW)
            rec.reproject(T_NOW)
            rec.reconstruct(T_NOW, out=out)

        for _ in range(2):
            step()
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = max(3, args.steps // 4)
        s.record()
        for _ in range(k):
            step()
        e.record()
        torch.cuda.synchronize()
        img = out[..., :3].cpu().numpy().astype(np.float64)
        res[name] = {"rms": round(float(np.sqrt(np.mean((img - gt) ** 2))), 6),
                     "holes": int((out[..., 3] == 0).sum()), "frame_records": int(rec.query()["frame"]),
                     "ms_per_step": round(s.elapsed_time(e) / k, 4)}
        rec.close()
        del pos, col, mo
        torch.cuda.empty_cache()
    res["what"] = ("c2_1024x1024x8 (8,388,608 samples, importance-sampled); RMS over RGB against 4x4 jittered "
                   "point samples per pixel at t = 1; fifo_N keeps the N most recent accepted samples")
    return res


def run_batched(args, dev, n_streams: int = 48):
    """48 viewer streams (seeds 0-47; sizes, depths and disc counts drawn per
    stream), FP16 colours, each tuned by the autotuner. A step is every
    stream's gradients, reprojection, widths and filter. Timed forms:
    afr_batch_refresh (every context on the batch's worker streams) captured
    in a CUDA graph; the per-stream gradients and reprojection followed by one
    afr_batch_reconstruct, in a graph; and, as the baseline, the same work as
    48 sequential single-stream call sequences, eager and in a graph. The
    per-resolution breakdown times the sequential calls and the refresh graph
    on each resolution's streams alone."""
    import torch
    from paper_2510_15876_gb300 import autotune
    from paper_2510_15876_gb300.api import BatchReconstructor, Reconstructor
    from workloads import scenes
    from workloads.gpu_scenes import sample_stream_gpu
    t0 = time.time()
    recs = []
    for i, sp in enumerate(scenes.batched_specs(n_streams)):
        sc = scenes.make_scene(sp, i)
        pos, col, mo = sample_stream_gpu(sc, sp.n_samples, i, dev)
        rec = Reconstructor(sp.width, sp.height, sp.depth, color_type="f16", device=dev)
        rec.insert(pos, col.half().contiguous(), mo)
        del pos, col, mo
        rec.estimate_gradients(T_NOW)
        rec.reproject(T_NOW)
        recs.append(rec)
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    tuned = [autotune.tune(r, T_NOW) for r in recs]
    k = max(3, args.steps // 4)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(k):
            fn()
        e.record()
        torch.cuda.synchronize()
        return s.elapsed_time(e) / k

    def graphed(fn):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            fn()
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        return g

    def forms(group):
        outs = [torch.empty((r.H, r.W, 4), dtype=torch.float32, device=dev) for r in group]
        B = BatchReconstructor(group)

        def sequential_step():
            for r, o in zip(group, outs):
                r.estimate_gradients(T_NOW)
                r.reproject(T_NOW)
                r.reconstruct(T_NOW, out=o)

        def persistent_step():
            for r in group:
                r.estimate_gradients(T_NOW)
                r.reproject(T_NOW)
            B.run(T_NOW)

        def refresh_step():
            B.refresh(T_NOW)

        t = {"sequential": timed(sequential_step)}
        g_seq = graphed(sequential_step)
        t["sequential_graph"] = timed(g_seq.replay)
        t["refresh"] = timed(refresh_step)
        g_ref = graphed(refresh_step)
        t["refresh_graph"] = timed(g_ref.replay)
        g_per = graphed(persistent_step)
        t["persistent_graph"] = timed(g_per.replay)
        same = all(torch.equal(a, b) for a, b in zip(outs, B.outs))
        del g_seq, g_ref, g_per
        B.close()
        return t, same

    t_all, same_all = forms(recs)
    pixels = sum(r.W * r.H for r in recs)
    per_res = {}
    for key in sorted({(r.W, r.H) for r in recs}, key=lambda wh: wh[0] * wh[1]):
        group = [r for r in recs if (r.W, r.H) == key]
        tg, same = forms(group)
        same_all = same_all and same
        per_res[f"{key[0]}x{key[1]}"] = {
            "streams": len(group), "depths": sorted({r.b for r in group}),
            "sequential_ms": round(tg["sequential"], 3), "sequential_graph_ms": round(tg["sequential_graph"], 3),
            "refresh_graph_ms": round(tg["refresh_graph"], 3),
            "speedup_vs_sequential": round(tg["sequential"] / tg["refresh_graph"], 2)}
    status = [r.status() for r in recs]
    best = min(t_all["refresh_graph"], t_all["persistent_graph"])
    res = {
        "streams": n_streams, "pixels": pixels, "samples": sum(r.W * r.H * r.b for r in recs),
        "refresh_graph_ms_per_step": round(t_all["refresh_graph"], 3),
        "refresh_ms_per_step": round(t_all["refresh"], 3),
        "persistent_graph_ms_per_step": round(t_all["persistent_graph"], 3),
        "sequential_ms_per_step": round(t_all["sequential"], 3),
        "sequential_graph_ms_per_step": round(t_all["sequential_graph"], 3),
        "mpixel_per_s_batched": round(pixels / best / 1e3, 1),
        "mpixel_per_s_sequential": round(pixels / t_all["sequential"] / 1e3, 1),
        "speedup_vs_sequential": round(t_all["sequential"] / best, 2),
        "speedup_vs_sequential_graph": round(t_all["sequential_graph"] / best, 2),
        "per_resolution": per_res,
        "radius_counts": {str(rr): sum(1 for t in tuned if t[0] == rr) for rr in autotune.RADII},
        "tile_counts": {str(tt): sum(1 for t in tuned if t[1] == tt) for tt in autotune.TILES},
        "images_identical": bool(same_all),
        "status_ok": all(s_ == 0 for s_ in status), "generation_s": round(gen_s, 1),
        "what": "every stream's gradients, reprojection, widths and filter: afr_batch_refresh on worker streams "
                "(CUDA graph), or per stream gradients + reprojection then one afr_batch_reconstruct (graph), "
                "vs the per stream calls in series",
    }
    for r in recs:
        r.close()
    torch.cuda.empty_cache()
    return res


# ------------------------------------------------------------------------------ oracle arm
def _oracle_image(scene, batch, threads):
    """The oracle's whole path on the whole image (ingest, gradients, tile
    statistics, reprojection, widths, filter) with the given thread count."""
    import oracle
    oracle.set_threads(threads)
    W, H, b = scene.width, scene.height, scene.spec.depth
    t0 = time.perf_counter()
    ring = oracle.Ring(W, H, b)
    ring.insert(batch["pos"], batch["color"], batch["motion"])
    res = oracle.reconstruct(ring, T_NOW)
    return time.perf_counter() - t0, res


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def parity_stats(gpu_image, ref_image):
    """End-to-end colour error of the GPU image against the oracle's image of
    the same batch: relative per channel with denominator max(|ref|, 1e-3)."""
    hole = ref_image[:, 3] == 0
    err = np.abs(gpu_image[~hole, :3] - ref_image[~hole, :3]) / np.maximum(np.abs(ref_image[~hole, :3]), 1e-3)
    return {"max_rel_err": float(err.max()) if err.size else 0.0,
            "p99_9_rel_err": float(np.quantile(err, 0.999)) if err.size else 0.0,
            "channel_values_above_1e-5": int((err > 1e-5).sum()), "channel_values": int(err.size),
            "holes_match": bool(np.all(gpu_image[hole] == 0)),
            "what": "last timed step's FP32 image against the FP64 oracle's whole path on the same batch, every pixel"}


def cpu_baseline(scene, batch, budget_s, gpu_image, single_thread=True):
    """The oracle timed on the whole 1920x1080x16 image: on every host core
    (runs until budget_s, at most 3) and once on one core. Also the parity of
    the GPU image against the oracle's image."""
    cores = _host_cores()
    times, res = [], None
    t_start = time.perf_counter()
    while not times or (time.perf_counter() - t_start < budget_s and len(times) < 3):
        dt, res = _oracle_image(scene, batch, cores)
        times.append(dt)
    per_image = sum(times) / len(times)
    cb = {"value": round(1.0 / per_image, 6), "unit": "reconstructions/s", "cores": cores, "kind": "oracle",
          "sample": f"{len(times)} runs of the whole oracle path on the whole {scene.width}x{scene.height}x"
                    f"{scene.spec.depth} image ({batch['pos'].shape[0]} samples), OpenMP over pixels, rows and tiles "
                    f"on {cores} host threads; {per_image:.2f} s an image"}
    single = None
    if single_thread:
        dt1, _ = _oracle_image(scene, batch, 1)
        single = {"value": round(1.0 / dt1, 6), "unit": "reconstructions/s", "cores": 1, "kind": "oracle",
                  "sample": f"one run of the whole oracle path on the whole image on one thread; {dt1:.2f} s"}
    parity = parity_stats(gpu_image, res["image"]) if gpu_image is not None else None
    return cb, single, parity


def run_reference(args, rank, world):
    if rank != 0:
        return
    from workloads import scenes
    scene, batch = scenes.config_stream(WORKLOAD, 0)
    cores = _host_cores()
    for _ in range(args.warmup):
        _oracle_image(scene, batch, cores)
    t = []
    for _ in range(args.steps):
        dt, _ = _oracle_image(scene, batch, cores)
        t.append(dt)
    per_image = sum(t) / len(t)
    value = 1.0 / per_image
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "reconstructions/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per_image * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": arm_config(WORKLOAD, batch["pos"].shape[0], 0, 1),
        "cpu_baseline": {"value": round(value, 6), "unit": "reconstructions/s", "cores": cores, "kind": "oracle",
                         "sample": f"each step: the whole oracle path on the whole {scene.width}x{scene.height}x"
                                   f"{scene.spec.depth} image, OpenMP on {cores} host threads"},
        "e2e": {"value": round(value, 6), "unit": "reconstructions/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="FP32 form only, no batched form")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-single-thread", action="store_true", help="skip the single-thread oracle figure")
    ap.add_argument("--workload", default=WORKLOAD, help="workload key (workloads.scenes.CONFIGS)")
    ap.add_argument("--color", default=None, choices=["f32", "f16", "bf16"], help="one colour form only")
    ap.add_argument("--profile", action="store_true",
                    help="time the step only (no end-to-end, adjoint, batched or CPU legs); for profilers")
    ap.add_argument("--filter-traffic", type=float, default=None,
                    help="DRAM bytes per k_filter launch from an ncu capture of the current build")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
