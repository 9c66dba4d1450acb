#!/usr/bin/env python3
"""Benchmark of the reconstruction hot path on one GB300 (or N replicas).

One step is the whole path over one batch of the 1920x1080, 16-deep workload
(33,177,600 seeded synthetic samples, FP32 colours): empty the deep buffer,
ingest the batch (section 4), estimate gradients (4.1), reproject to t_now
(6.2), filter every pixel (5.1, 5.2) and finalise the tile statistics (4.2,
6.1). The batch (1.3 GB) and the buffers are far larger than L2, so no flush
is needed between steps.

Prints one JSON line. --impl reference times the CPU oracle instead (a band
of the same workload per step, scaled to whole images).
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
# kernels launched per call (memsets excluded), as the launch sequences in csrc/ issue them
LAUNCHES = {"ingest": 6, "gradients": 3, "reproject": 7, "reconstruct": 2, "feedback": 1}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


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
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 8 for k in range(4)
                          if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


# ------------------------------------------------------------------------------ workload bytes
def step_bytes(P, b, n_batch, resident, frame, csize, ntiles):
    """Algorithmic HBM bytes of one step (each operand read or written once).
    csize: stored colour bytes (16 FP32 / 8 FP16). Sample fields: x,y,mx,my
    (16 B), t (4), depth (4), seq (4), colour."""
    ingest = n_batch * (16 + csize + 8) + resident * (16 + 4 + 4 + 4 + csize) + P * 4
    grads = resident * (4 + csize + 4) + P * (4 + 16 + 16 + 4) + ntiles * 64
    reproj = resident * (16 + 4 + 4 + csize) + frame * (16 + csize) + P * 8
    recon = frame * (16 + csize) + P * (16 + 8 + 4 + 4 + 16)
    feedback = ntiles * (64 + 32)
    return {"ingest": ingest, "gradients": grads, "reproject": reproj, "reconstruct": recon,
            "feedback": feedback}


def pairs_of(off, W, H, R):
    """Sample-pixel pairs the filter evaluates (integer disc footprint)."""
    cnt = np.diff(off.astype(np.int64)).reshape(H, W)
    tot = 0
    for dy in range(-R, R + 1):
        hw = int(np.floor(np.sqrt(R * R - dy * dy) + 1e-9))
        rows = np.zeros((H, W), np.int64)
        src = np.roll(cnt, -dy, axis=0)
        if dy > 0:
            src[H - dy:] = 0
        elif dy < 0:
            src[:-dy] = 0
        cs = np.concatenate([np.zeros((H, 1), np.int64), np.cumsum(src, axis=1)], axis=1)
        x = np.arange(W)
        x0 = np.maximum(0, x - hw)
        x1 = np.minimum(W - 1, x + hw)
        rows = cs[:, x1 + 1] - cs[:, x0]
        tot += int(rows.sum())
    return tot


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
    stream = torch.cuda.current_stream()

    def make(ct):
        r = Reconstructor(W, H, b, color_type=ct, device=dev)
        r.reserve(n)
        return r

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

    results = {}
    hbm_peak, peak_kind = _peaks()
    forms = ["f32", "f16", "bf16"] if not (args.quick or args.profile) else ["f32"]
    if args.color:
        forms = [args.color]
    for ct in forms:
        dtype = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[ct]
        rec = make(ct)
        pos, col, mo = to_device_batch(batch, dev, dtype)
        out = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
        tiles = torch.empty((rec.n_tiles, 8), dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            step(rec, pos, col, mo, out, tiles)
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = None
        if ct == forms[0]:
            sampler = ClockSampler(local)
            sampler.start()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record()
        for k in range(args.steps):
            step(rec, pos, col, mo, out, tiles, evs[k])
        end.record()
        torch.cuda.synchronize()
        if ct == forms[0]:
            clocks = sampler.stop()
        ms_total = start.elapsed_time(end)
        if dist:
            tt = torch.tensor([ms_total], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            ms_total = float(tt.item())
            dist.barrier()
        stages = ["ingest", "gradients", "reproject", "reconstruct", "feedback"]
        st_ms = {s: sum(e[i].elapsed_time(e[i + 1]) for e in evs) / args.steps for i, s in enumerate(stages)}
        info = rec.query()
        off, _, _ = (None, None, None)
        results[ct] = {"ms_per_step": ms_total / args.steps, "stage_ms": st_ms, "info": info, "clocks": clocks,
                       "csize": 16 if ct == "f32" else 8, "rec": rec, "out": out}
        if ct != forms[0]:
            rec.close()
            del pos, col, mo
            torch.cuda.empty_cache()

    r32 = results[forms[0]]
    rec = r32["rec"]
    if args.profile:
        print(json.dumps({"workload": args.workload, "color": forms[0], "ms_per_step": r32["ms_per_step"],
                          "stage_ms": r32["stage_ms"], "info": r32["info"]}), flush=True)
        rec.close()
        return
    info = r32["info"]
    off, _, _ = rec.export_frame()
    pairs = pairs_of(off, W, H, 4)
    resident, frame = int(info["resident"]), int(info["frame"])
    by = step_bytes(P, b, n, resident, frame, r32["csize"], rec.n_tiles)
    step_ms = r32["ms_per_step"]
    total_bytes = sum(by.values())
    st = r32["stage_ms"]
    # dominant stage and its roofline
    dom = max(st, key=st.get)
    if dom == "reconstruct":
        flops = pairs * 16.0
        peak_tf = 152 * 128 * 2 * 2.07e9 / 1e12
        ach = flops / (st[dom] * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "k_filter (+k_sigma)", "achieved": round(ach, 2), "peak": round(peak_tf, 1),
                "unit": "TFLOP/s", "frac": round(ach / peak_tf, 4), "traffic": None,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 (FMA) x 2.07 GHz",
                "work": f"{pairs} pairs x 16 FLOP"}
    else:
        ach = by[dom] / (st[dom] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(ach / hbm_peak, 4), "traffic": None, "peak_source": peak_kind}

    # end to end through the public API with host buffers
    import torch as _t
    hp = {k: _t.from_numpy(np.ascontiguousarray(batch[k], np.float32)).pin_memory() for k in ("pos", "color", "motion")}
    dpos, dcol, dmo = (_t.empty_like(hp[k], device=dev) for k in ("pos", "color", "motion"))
    host_img = _t.empty((H, W, 4), dtype=_t.float32).pin_memory()
    tiles = _t.empty((rec.n_tiles, 8), dtype=_t.float32, device=dev)

    def e2e_step():
        dpos.copy_(hp["pos"], non_blocking=True)
        dcol.copy_(hp["color"], non_blocking=True)
        dmo.copy_(hp["motion"], non_blocking=True)
        step(rec, dpos, dcol, dmo, r32["out"], tiles)
        host_img.copy_(r32["out"], non_blocking=True)

    for _ in range(max(1, args.warmup // 2)):
        e2e_step()
    _t.cuda.synchronize()
    s2, e2 = _t.cuda.Event(enable_timing=True), _t.cuda.Event(enable_timing=True)
    k2 = max(3, args.steps // 2)
    s2.record()
    for _ in range(k2):
        e2e_step()
    e2.record()
    _t.cuda.synchronize()
    e2e_ms = s2.elapsed_time(e2) / k2
    h2d = sum(hp[k].numel() * 4 for k in hp)
    d2h = host_img.numel() * 4

    # fwd+bwd on the 512x512x8 differentiation workload
    fb = run_fwd_bwd(args, dev)

    value = world * 1000.0 / step_ms
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "reconstructions/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD} (1920x1080 image, 16-deep buffer, {n} samples per batch, 256 moving "
                               f"discs, 10% occlusion-edge pixels, seed {seed})",
                   "global_batch": n * world, "l2": "inputs larger than L2 (1.3 GB batch), no flush",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "mpixel_per_s": round(P * value / 1e6, 1),
        "samples_filtered_per_s": round(frame * value, 0),
        "pairs_per_step": pairs,
        "hbm_frac_step": round(total_bytes / (step_ms * 1e-3) / 1e9 / hbm_peak, 4),
        "step_bytes": total_bytes,
        "stage_ms": {k: round(v, 4) for k, v in st.items()},
        "roofline": roof,
        "precision_forms": {ct: {"ms_per_step": round(results[ct]["ms_per_step"], 4),
                                 "stage_ms": {k: round(v, 4) for k, v in results[ct]["stage_ms"].items()}}
                            for ct in results},
        "fwd_bwd": fb,
        "e2e": {"value": round(world * 1000.0 / e2e_ms, 3), "unit": "reconstructions/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * sum(LAUNCHES.values()),
        "clocks": r32["clocks"],
        "resident": resident, "frame": frame, "generation_s": round(gen_s, 1),
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(scene, batch, args.cpu_seconds)
    rec.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_fwd_bwd(args, dev):
    import torch
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    from workloads import scenes
    sc, batch = scenes.config_stream("c4_512x512x8", 0)
    W, H, b = sc.width, sc.height, sc.spec.depth
    rec = Reconstructor(W, H, b, device=dev)
    pos, col, mo = to_device_batch(batch, dev)
    rec.insert(pos, col, mo)
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
    return {"config": "c4_512x512x8 (512x512, 8-deep, 2,097,152 samples)", "ms_per_step": round(s.elapsed_time(e) / k, 4),
            "what": "afr_reconstruct + afr_reconstruct_backward (colours and 6 parameters)"}


# ------------------------------------------------------------------------------ oracle arm
def _oracle_band_step(scene, batch, band_rows, y0):
    """The oracle's whole path on the samples of one horizontal band, run as its
    own image of band_rows rows."""
    import oracle
    W, b = scene.width, scene.spec.depth
    pos = batch["pos"]
    sel = (pos[:, 1] >= y0) & (pos[:, 1] < y0 + band_rows)
    p = pos[sel].copy()
    p[:, 1] -= y0
    t0 = time.perf_counter()
    ring = oracle.Ring(W, band_rows, b)
    ring.insert(p, batch["color"][sel], batch["motion"][sel])
    res = oracle.reconstruct(ring, T_NOW)
    return time.perf_counter() - t0, res


def cpu_baseline(scene, batch, budget_s):
    H = scene.height
    band = 34
    secs, k = 0.0, 0
    y0 = (H - band) // 2
    t_start = time.perf_counter()
    while k == 0 or (time.perf_counter() - t_start < budget_s and k < 8):
        dt, _ = _oracle_band_step(scene, batch, band, y0)
        secs += dt
        k += 1
    per_image = secs / k * (H / band)
    return {"value": round(1.0 / per_image, 6), "unit": "reconstructions/s", "cores": 1, "kind": "oracle",
            "sample": f"{k} runs of the whole oracle path on a {scene.width}x{band} band of the workload "
                      f"(its samples only), scaled by {H}/{band} rows"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from workloads import scenes
    scene, batch = scenes.config_stream(WORKLOAD, 0)
    H = scene.height
    band = 34
    y0 = (H - band) // 2
    for _ in range(args.warmup):
        _oracle_band_step(scene, batch, band, y0)
    t = []
    for _ in range(args.steps):
        dt, _ = _oracle_band_step(scene, batch, band, y0)
        t.append(dt)
    per_image = sum(t) / len(t) * (H / band)
    value = 1.0 / per_image
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "reconstructions/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per_image * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD} (1920x1080 image, 16-deep buffer)", "parallelism": "single host thread"},
        "cpu_baseline": {"value": round(value, 6), "unit": "reconstructions/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step: the whole oracle path on a 1920x{band} band, scaled by {H}/{band}"},
        "e2e": {"value": round(value, 6), "unit": "reconstructions/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="FP32 form only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default=WORKLOAD, help="workload key (workloads.scenes.CONFIGS)")
    ap.add_argument("--color", default=None, choices=["f32", "f16", "bf16"], help="one colour form only")
    ap.add_argument("--profile", action="store_true",
                    help="time the step only (no end-to-end, adjoint or CPU legs); for profilers")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.gpus == 1 else 1)))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
