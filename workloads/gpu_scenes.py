"""The scenes of workloads.scenes evaluated on a CUDA device with torch.

Used where a workload is too large to draw on the host in reasonable time
(the batched form's 48 streams). Same scene model, samples drawn from a
seeded torch generator on the device; none of the reconstruction method's
arithmetic is here.
"""
from __future__ import annotations

import torch

from .scenes import Scene


def sample_stream_gpu(scene: Scene, n: int, seed: int, device, chunk: int = 1 << 22):
    W, H = scene.width, scene.height
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    x = torch.rand(n, generator=g, device=device, dtype=torch.float64) * W
    y = torch.rand(n, generator=g, device=device, dtype=torch.float64) * H
    t = torch.sort(torch.rand(n, generator=g, device=device, dtype=torch.float64)).values
    xf = torch.clamp(x.float(), max=float(torch.nextafter(torch.tensor(float(W)), torch.tensor(0.0))))
    yf = torch.clamp(y.float(), max=float(torch.nextafter(torch.tensor(float(H)), torch.tensor(0.0))))
    tf = t.float()
    pos = torch.empty((n, 4), dtype=torch.float32, device=device)
    col = torch.zeros((n, 4), dtype=torch.float32, device=device)
    mo = torch.empty((n, 2), dtype=torch.float32, device=device)
    cx = torch.tensor(scene.cx, device=device)
    cy = torch.tensor(scene.cy, device=device)
    vx = torch.tensor(scene.vx, device=device)
    vy = torch.tensor(scene.vy, device=device)
    r2 = torch.tensor(scene.r ** 2, device=device)
    rgb = torch.tensor(scene.rgb, device=device)
    dep = torch.tensor(scene.depth, device=device)
    s = scene.spec.check
    px, py = scene.spec.pan
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        X, Y, T = xf[a:b].double(), yf[a:b].double(), tf[a:b].double()
        white = ((torch.floor((X - px * T) / s) + torch.floor((Y - py * T) / s)).long() & 1) == 0
        c = white.double()[:, None].expand(-1, 3).clone()
        m = torch.empty((b - a, 2), dtype=torch.float64, device=device)
        m[:, 0], m[:, 1] = px, py
        best = torch.full((b - a,), float("inf"), dtype=torch.float64, device=device)
        for i in range(len(scene.r)):
            dx = X - (cx[i] + vx[i] * T)
            dy = Y - (cy[i] + vy[i] * T)
            d2 = dx * dx + dy * dy
            hit = (d2 <= r2[i]) & (dep[i] < best)
            if not bool(hit.any()):
                continue
            ci = rgb[i].expand(b - a, 3)
            if scene.spec.highlight:
                ci = ci + torch.exp(-d2 / (0.1 * torch.sqrt(r2[i])) ** 2)[:, None]
            c = torch.where(hit[:, None], ci, c)
            m[:, 0] = torch.where(hit, vx[i], m[:, 0])
            m[:, 1] = torch.where(hit, vy[i], m[:, 1])
            best = torch.where(hit, dep[i], best)
        pos[a:b, 0], pos[a:b, 1], pos[a:b, 2] = xf[a:b], yf[a:b], tf[a:b]
        pos[a:b, 3] = best.float()
        col[a:b, :3] = c.float()
        mo[a:b] = m.float()
    return pos, col, mo
