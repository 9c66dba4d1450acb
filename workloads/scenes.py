"""Seeded synthetic scenes and sample streams for the reconstruction path.

This module only *generates inputs*: analytic scenes (a black/white checkerboard
background, optionally panning, under opaque moving discs), sample streams drawn
from them and dense ground-truth images.  It holds none of the reconstruction
method's arithmetic (no luminance, age weighting, gradients, reprojection or
filtering); both the CPU oracle and the CUDA path consume exactly the arrays it
returns.

The scenes stand in for the animated ray-traced test scenes of the paper's
evaluation (section 7), which are not available here.  Every scene, sample
position, time and colour is drawn from numpy's Philox generator keyed by
``(config key, seed)``.

Sample records follow the layout the library ingests:

* ``pos``    float32 [n, 4]  (x, y, t, depth), pixel units, t in window units
* ``color``  float32 [n, 4]  (r, g, b, 0)
* ``motion`` float32 [n, 2]  screen-space velocity in pixels per window

Samples are sorted by t (stable), so insertion order and time order agree.
"""
from __future__ import annotations

import dataclasses
import hashlib
import math

import numpy as np

__all__ = [
    "Scene", "SceneSpec", "CONFIGS", "make_scene", "eval_scene",
    "sample_stream", "ground_truth", "config_stream", "batched_specs",
]


def _rng(key: str, seed: int, stream: int = 0) -> np.random.Generator:
    digest = hashlib.sha256(f"{key}/{seed}/{stream}".encode()).digest()
    k = int.from_bytes(digest[:16], "little")
    return np.random.Generator(np.random.Philox(key=k))


@dataclasses.dataclass(frozen=True)
class SceneSpec:
    """Shape of one synthetic workload (the paper's sample-stream scenarios)."""
    key: str
    width: int
    height: int
    depth: int                    # ring depth b
    n_discs: int
    radius: tuple[float, float]   # disc radius range, pixels
    speed: float                  # disc velocity uniform in [-speed, speed]^2 px/window
    check: int                    # checker cell size, pixels
    pan: tuple[float, float] = (0.0, 0.0)   # background pan, px/window
    highlight: bool = False       # radial specular highlight on discs
    importance: bool = False      # 32x32-tile importance-sampled positions
    edge_fraction: float | None = None      # tune radii to this occlusion-edge fraction

    @property
    def n_samples(self) -> int:
        return self.width * self.height * self.depth


CONFIGS: dict[str, SceneSpec] = {
    # 128x128 image, 4-deep buffer, static scene (65,536 samples)
    "c1_128x128x4": SceneSpec("c1_128x128x4", 128, 128, 4, 8, (6.0, 20.0), 0.0, 8),
    # 1024x1024, 8-deep, 64 moving discs with highlights over a panning checker
    "c2_1024x1024x8": SceneSpec("c2_1024x1024x8", 1024, 1024, 8, 64, (16.0, 64.0), 32.0, 16,
                                pan=(8.0, 0.0), highlight=True, importance=True),
    # 1920x1080, 16-deep, 256 moving discs, ~10% of pixels on occlusion edges
    "c3_1920x1080x16": SceneSpec("c3_1920x1080x16", 1920, 1080, 16, 256, (8.0, 24.0), 64.0, 16,
                                 edge_fraction=0.10),
    # a quarter of the 1920x1080x16 scene (same sample, disc and edge densities),
    # for counter captures that must stay a few GB on the device
    "p3_960x540x16": SceneSpec("p3_960x540x16", 960, 540, 16, 64, (8.0, 24.0), 64.0, 16, edge_fraction=0.10),
    # 512x512, 8-deep, 32 moving discs (differentiation form)
    "c4_512x512x8": SceneSpec("c4_512x512x8", 512, 512, 8, 32, (12.0, 40.0), 32.0, 16),
}


@dataclasses.dataclass
class Scene:
    spec: SceneSpec
    cx: np.ndarray      # disc centre at t=0, float64 [k]
    cy: np.ndarray
    vx: np.ndarray      # disc velocity, px/window
    vy: np.ndarray
    r: np.ndarray       # disc radius
    rgb: np.ndarray     # [k, 3]
    depth: np.ndarray   # [k]

    @property
    def width(self) -> int:
        return self.spec.width

    @property
    def height(self) -> int:
        return self.spec.height


def _edge_fraction(scene: Scene, t: float, reach: int = 2) -> float:
    """Fraction of pixels lying on an occlusion edge at time t: pixels whose
    (2*reach+1)^2 pixel-centre neighbourhood sees more than one surface."""
    W, H = scene.width, scene.height
    ys, xs = np.mgrid[0:H, 0:W]
    sid = _eval(scene, xs.ravel() + 0.5, ys.ravel() + 0.5, t)[3].reshape(H, W)
    pad = np.pad(sid, reach, mode="edge")
    edge = np.zeros((H, W), bool)
    for dy in range(-reach, reach + 1):
        for dx in range(-reach, reach + 1):
            edge |= pad[reach + dy:reach + dy + H, reach + dx:reach + dx + W] != sid
    return float(edge.mean())


def make_scene(spec: SceneSpec | str, seed: int = 0) -> Scene:
    if isinstance(spec, str):
        spec = CONFIGS[spec]
    rng = _rng(spec.key, seed, 1)
    k = spec.n_discs
    W, H = spec.width, spec.height
    cx = rng.uniform(0.0, W, k)
    cy = rng.uniform(0.0, H, k)
    vx = rng.uniform(-spec.speed, spec.speed, k)
    vy = rng.uniform(-spec.speed, spec.speed, k)
    u = rng.uniform(0.0, 1.0, k)
    rgb = rng.uniform(0.0, 1.0, (k, 3))
    depth = rng.uniform(0.0, 1.0, k)
    lo, hi = spec.radius
    scene = Scene(spec, cx, cy, vx, vy, lo + (hi - lo) * u, rgb, depth)
    if spec.edge_fraction is not None:
        # scale all radii by one factor so that the edge-pixel fraction at t=1
        # lands on the target (bisection on a deterministic function)
        a, b = 0.25, 4.0
        for _ in range(12):
            m = math.sqrt(a * b)
            scene.r = (lo + (hi - lo) * u) * m
            if _edge_fraction(scene, 1.0) < spec.edge_fraction:
                a = m
            else:
                b = m
        scene.r = (lo + (hi - lo) * u) * math.sqrt(a * b)
    return scene


def _checker(scene: Scene, x, y, t):
    s = scene.spec.check
    px, py = scene.spec.pan
    cx = np.floor((x - px * t) / s).astype(np.int64)
    cy = np.floor((y - py * t) / s).astype(np.int64)
    return ((cx + cy) & 1) == 0


def eval_scene(scene: Scene, x, y, t):
    """Analytic point evaluation: colour [n,3], motion [n,2], depth [n] (float64).

    The nearest disc covering (x, y) at time t wins; otherwise the checker
    background (depth +inf) shows.
    """
    return _eval(scene, x, y, t)[:3]


def _eval(scene: Scene, x, y, t, cell: int = 64):
    """eval_scene plus the surface id (-1 background, else disc index); discs
    are culled with a coarse grid so large streams stay cheap."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    t = np.broadcast_to(np.asarray(t, np.float64), x.shape)
    n = x.shape[0]
    white = _checker(scene, x, y, t)
    rgb = np.where(white[:, None], 1.0, 0.0) * np.ones((1, 3))
    mo = np.empty((n, 2))
    mo[:, 0], mo[:, 1] = scene.spec.pan
    depth = np.full(n, np.inf)
    sid = np.full(n, -1, np.int64)
    if len(scene.r) == 0 or n == 0:
        return rgb, mo, depth, sid
    W, H = scene.width, scene.height
    ncx = max(1, math.ceil(W / cell))
    ncy = max(1, math.ceil(H / cell))
    gx = np.clip(np.floor(x / cell).astype(np.int64), 0, ncx - 1)
    gy = np.clip(np.floor(y / cell).astype(np.int64), 0, ncy - 1)
    cid = gy * ncx + gx
    order = np.argsort(cid, kind="stable")
    starts = np.searchsorted(cid[order], np.arange(ncx * ncy + 1))
    for i in range(len(scene.r)):
        r = scene.r[i]
        x0 = min(scene.cx[i], scene.cx[i] + scene.vx[i]) - r
        x1 = max(scene.cx[i], scene.cx[i] + scene.vx[i]) + r
        y0 = min(scene.cy[i], scene.cy[i] + scene.vy[i]) - r
        y1 = max(scene.cy[i], scene.cy[i] + scene.vy[i]) + r
        c0 = max(0, int(math.floor(x0 / cell)))
        c1 = min(ncx - 1, int(math.floor(x1 / cell)))
        r0 = max(0, int(math.floor(y0 / cell)))
        r1 = min(ncy - 1, int(math.floor(y1 / cell)))
        if c0 > c1 or r0 > r1:
            continue
        idx = np.concatenate([order[starts[row * ncx + c0]:starts[row * ncx + c1 + 1]]
                              for row in range(r0, r1 + 1)])
        if idx.size == 0:
            continue
        tt = t[idx]
        dx = x[idx] - (scene.cx[i] + scene.vx[i] * tt)
        dy = y[idx] - (scene.cy[i] + scene.vy[i] * tt)
        d2 = dx * dx + dy * dy
        hit = (d2 <= r * r) & (scene.depth[i] < depth[idx])
        sel = idx[hit]
        if sel.size == 0:
            continue
        col = np.broadcast_to(scene.rgb[i], (sel.size, 3)).copy()
        if scene.spec.highlight:
            col += np.exp(-d2[hit] / (0.1 * r) ** 2)[:, None]
        rgb[sel] = col
        mo[sel, 0] = scene.vx[i]
        mo[sel, 1] = scene.vy[i]
        depth[sel] = scene.depth[i]
        sid[sel] = i
    return rgb, mo, depth, sid


def _importance_tiles(scene: Scene, rng: np.random.Generator, tile: int = 32):
    """Tile probabilities proportional to the pilot colour variance at t=0.5,
    mixed with a 5% uniform floor."""
    W, H = scene.width, scene.height
    ys, xs = np.mgrid[0:H, 0:W]
    rgb, _, _ = eval_scene(scene, xs.ravel() + 0.5, ys.ravel() + 0.5, 0.5)
    img = rgb.reshape(H, W, 3)
    ntx, nty = math.ceil(W / tile), math.ceil(H / tile)
    var = np.zeros((nty, ntx))
    for j in range(nty):
        for i in range(ntx):
            blk = img[j * tile:(j + 1) * tile, i * tile:(i + 1) * tile].reshape(-1, 3)
            var[j, i] = blk.var(axis=0).mean()
    p = var.ravel()
    p = 0.95 * p / p.sum() + 0.05 / p.size if p.sum() > 0 else np.full(p.size, 1.0 / p.size)
    return p / p.sum(), ntx, nty


def sample_stream(scene: Scene, n: int, seed: int = 0, *, t_range=(0.0, 1.0), stream: int = 2):
    """Draw n samples: (x, y) uniform (or importance-sampled), t uniform in
    t_range and sorted ascending, colour and motion from the analytic scene."""
    spec = scene.spec
    rng = _rng(spec.key, seed, stream)
    W, H = spec.width, spec.height
    if spec.importance:
        p, ntx, nty = _importance_tiles(scene, rng)
        tiles = rng.choice(p.size, size=n, p=p)
        tx = (tiles % ntx) * 32
        ty = (tiles // ntx) * 32
        tw = np.minimum(32, W - tx)
        th = np.minimum(32, H - ty)
        x = tx + rng.uniform(0.0, 1.0, n) * tw
        y = ty + rng.uniform(0.0, 1.0, n) * th
    else:
        x = rng.uniform(0.0, W, n)
        y = rng.uniform(0.0, H, n)
    t = np.sort(rng.uniform(t_range[0], t_range[1], n))
    x32 = np.minimum(x.astype(np.float32), np.nextafter(np.float32(W), np.float32(0)))
    y32 = np.minimum(y.astype(np.float32), np.nextafter(np.float32(H), np.float32(0)))
    t32 = t.astype(np.float32)
    rgb, mo, depth = eval_scene(scene, x32.astype(np.float64), y32.astype(np.float64),
                                t32.astype(np.float64))
    pos = np.stack([x32, y32, t32, depth.astype(np.float32)], axis=1)
    color = np.zeros((n, 4), np.float32)
    color[:, :3] = rgb
    motion = mo.astype(np.float32)
    return {"pos": np.ascontiguousarray(pos), "color": color,
            "motion": np.ascontiguousarray(motion)}


def ground_truth(scene: Scene, t: float = 1.0, spp_side: int = 8, seed: int = 0):
    """Dense reference image at time t: spp_side^2 stratified jittered point
    evaluations per pixel, averaged (float64 [H, W, 3])."""
    W, H = scene.width, scene.height
    rng = _rng(scene.spec.key, seed, 3)
    acc = np.zeros((H * W, 3))
    ys, xs = np.mgrid[0:H, 0:W]
    xs = xs.ravel().astype(np.float64)
    ys = ys.ravel().astype(np.float64)
    for sj in range(spp_side):
        for si in range(spp_side):
            jx = rng.uniform(0.0, 1.0, H * W)
            jy = rng.uniform(0.0, 1.0, H * W)
            rgb, _, _ = eval_scene(scene, xs + (si + jx) / spp_side, ys + (sj + jy) / spp_side, t)
            acc += rgb
    return (acc / (spp_side * spp_side)).reshape(H, W, 3)


def config_stream(key: str, seed: int = 0):
    """Scene and its full sample stream for one named configuration."""
    scene = make_scene(key, seed)
    return scene, sample_stream(scene, scene.spec.n_samples, seed)


def batched_specs(n_streams: int = 48):
    """Viewer streams of the batched form: resolution from {256^2, 640x480,
    1280x720, 1920x1080}, depth from {4, 8, 16}, 16-256 moving discs; stream i
    uses seed i."""
    rng = _rng("c5_batched", 0, 0)
    res = [(256, 256), (640, 480), (1280, 720), (1920, 1080)]
    specs = []
    for i in range(n_streams):
        w, h = res[rng.integers(0, 4)]
        b = int((4, 8, 16)[rng.integers(0, 3)])
        k = int(rng.integers(16, 257))
        specs.append(SceneSpec(f"c5_stream{i}", w, h, b, k, (8.0, 32.0), 32.0, 16))
    return specs
