"""Autotuner for the filter of a stream: footprint radius and CTA tile shape.

* radius: the footprint is an integer disc of radius R over the frame bins,
  so a wide Gaussian is cut short when R is small next to its spatial width.
  From a pilot reconstruction the tuner reads the stream's spatial widths
  and takes the smallest R in the candidates with R >= k * (95th percentile of
  sigma_s); this changes results, so callers that compare against a
  reference run the reference at the chosen R.
* tile shape: the filter's CTA covers (2*tile_bx) x (64/tile_bx) pixels; the
  tuner times each candidate (CUDA events, after a warm-up) on the stream
  itself and keeps the fastest. This does not change results.
Choices are cached per (width, height, depth, colour type, radius).
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L
from .api import Reconstructor, set_tuning

RADII = (3, 4, 5)
TILES = (4, 8, 16)
_cache: dict = {}


def choose_radius(rec: Reconstructor, t_now: float = 1.0, params=None, radii=RADII, k: float = 1.5) -> int:
    rec.reconstruct(t_now, params)
    ss = rec.export_map(L.AFR_MAP_SIGMA_S)
    p95 = float(np.quantile(ss, 0.95))
    for r in radii:
        if r >= k * p95:
            return r
    return radii[-1]


def time_filter(rec: Reconstructor, t_now: float, params, reps: int = 3) -> float:
    out = torch.empty((rec.H, rec.W, 4), dtype=torch.float32, device=rec.device)
    rec.reconstruct(t_now, params, out=out)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    for _ in range(reps):
        rec.reconstruct(t_now, params, out=out, flags=L.AFR_RECON_KEEP_SIGMA)
    end.record()
    torch.cuda.synchronize()
    return start.elapsed_time(end) / reps


def tune(rec: Reconstructor, t_now: float = 1.0, params=None, radii=RADII, tiles=TILES) -> tuple[int, int]:
    """Chooses and applies (radius, tile_bx); needs gradients and frame view for t_now."""
    radius = choose_radius(rec, t_now, params, radii)
    key = (rec.W, rec.H, rec.b, rec.ct, radius)
    if key not in _cache:
        best, best_ms = tiles[0], float("inf")
        for tb in tiles:
            set_tuning(rec, radius, tb)
            ms = time_filter(rec, t_now, params)
            if ms < best_ms:
                best, best_ms = tb, ms
        _cache[key] = best
    set_tuning(rec, radius, _cache[key])
    return radius, _cache[key]
