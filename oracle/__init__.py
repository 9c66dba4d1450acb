"""CPU oracle of the adaptive frameless reconstruction path (ctypes wrapper).

TEST INFRASTRUCTURE. The oracle is a plain, slow, double-precision C
restatement of the method (see afr_oracle.h); only the tests, the smoke check
and the benchmark's CPU-baseline leg may load it. It shares no code with the
CUDA library under paper_2510_15876_gb300/ and imports nothing from it.

Parity status of each function (what pins it, in tests/test_oracle_pins.py):

* ingest      -- pinned: a collections.deque(maxlen=b) model of the queues.
* gradients   -- pinned: constant scene, linear luminance ramps (with the Rec. 709
                 weight of each primary), linear-in-time colour, single samples.
* tile stats  -- pinned: two-valued tiles, hand-counted empty slots and u.
* reproject   -- pinned: a pure-Python float32 reprojection and a sort.
* sigma       -- pinned: the defining identities e_s^2 e_t = V_S and
                 e_s G_s = e_t G_t, closed-form volumes, clamps.
* filter      -- pinned: constant colour, partition of unity, one- and
                 two-sample closed forms, brute force, a numpy scatter sum.
* backward    -- pinned: central finite differences of the oracle's forward.
* camera      -- pinned: a float32 numpy projection model, the identity camera
                 (screen points map to themselves), a camera pan equal to a
                 screen shift, points behind the camera dropped.
* fifo        -- pinned: a collections.deque(maxlen=N) model; its frame view
                 against a float32 numpy reprojection of the deque.
* tile error  -- pinned: hand-computed shares, the partition identity
                 sum E / s = kappa + lambda + (1 - kappa - lambda), a constant-
                 age ramp scene for the gain control.
* coverage    -- pinned: hand-computed updates (growth, shrinkage, clamps,
                 border means), a numpy count of records per disc, hole
                 filling, and the per-pixel-radius filter against brute force
                 and against the fixed-radius filter.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NF, NR, NT, NP = 9, 6, 8, 6
DEFAULT_THETA = np.array([1.0, 0.0, 3.0, 1.0, 0.0, 1.0])


def build(force: bool = False) -> str:
    """Compile afr_oracle.c into liboracle.so (gcc, no contraction)."""
    src = os.path.join(_HERE, "afr_oracle.c")
    hdr = os.path.join(_HERE, "afr_oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-o", tmp, src, "-lm"]
    try:   # OpenMP over independent pixels, rows and tiles; results do not depend on it
        subprocess.check_call(cmd[:-1] + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i64, i32, u32, f32, f64 = (ctypes.c_int64, ctypes.c_int, ctypes.c_uint32,
                                       ctypes.c_float, ctypes.c_double)
            L.afo_set_threads.restype = None
            L.afo_set_threads.argtypes = [i32]
            L.afo_max_threads.restype = i32
            L.afo_max_threads.argtypes = []
            L.afo_ingest.restype = i64
            L.afo_ingest.argtypes = [i32, i32, i32, P, P, P, u32, i64, P, P, P]
            L.afo_gradients.restype = None
            L.afo_gradients.argtypes = [i32, i32, i32, P, P, P, f32, P, P, P, P]
            L.afo_tile_feedback.restype = None
            L.afo_tile_feedback.argtypes = [i32, i32, i32, i32, P, P, f32, P, P, P, f64, P]
            L.afo_reproject.restype = i64
            L.afo_reproject.argtypes = [i32, i32, i32, P, P, P, f32, P, P, P, i64, P]
            L.afo_sigma.restype = None
            L.afo_sigma.argtypes = [i32, i32, i32, i32, P, P, P, P, P, f64, f64, P, P]
            L.afo_filter.restype = None
            L.afo_filter.argtypes = [i32, i32, i32, P, P, f32, P, P, P, i64, P]
            L.afo_filter_brute.restype = None
            L.afo_filter_brute.argtypes = [i32, i32, i32, i64, P, f32, P, P, P]
            L.afo_reproject_camera.restype = i64
            L.afo_reproject_camera.argtypes = [i32, i32, i32, P, P, P, P, P, f32, P, P, P, i64, P]
            L.afo_fifo_insert.restype = i64
            L.afo_fifo_insert.argtypes = [i32, i32, i64, P, P, P, u32, i64, P, P, P]
            L.afo_tile_error.restype = None
            L.afo_tile_error.argtypes = [i32, i32, i32, i32, P, P, f32, P, P, f64, f64, f64, f64, P, P]
            L.afo_coverage_update.restype = None
            L.afo_coverage_update.argtypes = [i32, i32, P, P, f32, f32, P, P]
            L.afo_coverage_count.restype = None
            L.afo_coverage_count.argtypes = [i32, i32, P, P, P]
            L.afo_filter_var.restype = None
            L.afo_filter_var.argtypes = [i32, i32, P, P, P, f32, P, P, P, i64, P]
            L.afo_filter_brute_var.restype = None
            L.afo_filter_brute_var.argtypes = [i32, i32, P, i64, P, f32, P, P, P]
            L.afo_backward.restype = None
            L.afo_backward.argtypes = [i32, i32, i32, i32, i32, P, P, P, P, P, f64, f64,
                                       P, P, f32, P, P, P]
            _lib = L
    return _lib


def set_threads(n: int) -> None:
    """Threads of the oracle's loops over independent pixels, rows and tiles."""
    lib().afo_set_threads(int(n))


def max_threads() -> int:
    return int(lib().afo_max_threads())


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


class Ring:
    """Canonical deep buffer: per pixel, slots newest first."""

    def __init__(self, W: int, H: int, b: int):
        self.W, self.H, self.b = W, H, b
        P = W * H
        self.count = np.zeros(P, np.int32)
        self.slot = np.zeros((P, b, NF), np.float32)
        self.seq = np.zeros((P, b), np.uint32)
        self.total = 0
        self.rejected = 0

    def insert(self, pos, color, motion) -> int:
        pos = np.ascontiguousarray(pos, np.float32)
        color = np.ascontiguousarray(color, np.float32)
        motion = np.ascontiguousarray(motion, np.float32)
        n = pos.shape[0]
        rej = lib().afo_ingest(self.W, self.H, self.b, _p(self.count), _p(self.slot),
                               _p(self.seq), self.total & 0xFFFFFFFF, n, _p(pos), _p(color),
                               _p(motion))
        self.total += n
        self.rejected += rej
        return rej

    @property
    def resident(self) -> int:
        return int(self.count.sum())


def reproject_camera(ring: Ring, world_by_seq, view_proj, t_now: float = 1.0):
    """reproject() with the stored 3D hit points rendered by the row-major 4x4
    view_proj (section 6.2); world_by_seq[seq] = (X, Y, Z, -) of every sample
    inserted so far, indexed by sequence number."""
    P = ring.W * ring.H
    cap = max(1, ring.resident)
    off = np.zeros(P + 1, np.uint32)
    rec = np.zeros((cap, NR), np.float32)
    rseq = np.zeros(cap, np.uint32)
    dropped = ctypes.c_int64(0)
    world = np.ascontiguousarray(world_by_seq, np.float32).reshape(-1, 4)
    vp = np.ascontiguousarray(view_proj, np.float32).reshape(16)
    n = lib().afo_reproject_camera(ring.W, ring.H, ring.b, _p(ring.count), _p(ring.slot), _p(ring.seq),
                                   _p(world), _p(vp), t_now, _p(off), _p(rec), _p(rseq), cap,
                                   ctypes.addressof(dropped))
    assert n >= 0
    return off, rec[:n].copy(), rseq[:n].copy(), dropped.value


class Fifo:
    """The reconstructor's buffer of section 5.2: the N most recent accepted
    samples of the whole image, in one queue. Sequence numbers count every
    sample offered (accepted or not), as for the per-pixel queues."""

    def __init__(self, W: int, H: int, N: int):
        self.W, self.H, self.N = W, H, N
        self.q = np.zeros((N, NF), np.float32)
        self.seq = np.zeros(N, np.uint32)
        self.accepted = ctypes.c_int64(0)
        self.total = 0

    def insert(self, pos, color, motion) -> int:
        pos = np.ascontiguousarray(pos, np.float32)
        color = np.ascontiguousarray(color, np.float32)
        motion = np.ascontiguousarray(motion, np.float32)
        n = pos.shape[0]
        rej = lib().afo_fifo_insert(self.W, self.H, self.N, ctypes.addressof(self.accepted), _p(self.q),
                                    _p(self.seq), self.total & 0xFFFFFFFF, n, _p(pos), _p(color), _p(motion))
        self.total += n
        return rej

    @property
    def resident(self) -> int:
        return int(min(self.accepted.value, self.N))


def reproject_fifo(fifo: Fifo, t_now: float = 1.0):
    """reproject() over the FIFO's samples: the queue is handed to the same
    routine as one list (a single 'pixel' holding every sample); the frame
    view orders records by bin and sequence number, so storage order does
    not matter."""
    W, H, P, n = fifo.W, fifo.H, fifo.W * fifo.H, fifo.resident
    count = np.zeros(P, np.int32)
    count[0] = n
    cap = max(1, n)
    off = np.zeros(P + 1, np.uint32)
    rec = np.zeros((cap, NR), np.float32)
    rseq = np.zeros(cap, np.uint32)
    dropped = ctypes.c_int64(0)
    slot = np.ascontiguousarray(fifo.q[:max(n, 1)])
    seq = np.ascontiguousarray(fifo.seq[:max(n, 1)])
    m = lib().afo_reproject(W, H, max(n, 1), _p(count), _p(slot), _p(seq), t_now, _p(off), _p(rec), _p(rseq),
                            cap, ctypes.addressof(dropped))
    assert m >= 0
    return off, rec[:m].copy(), rseq[:m].copy(), dropped.value


def gradients(ring: Ring, t_now: float = 1.0):
    P = ring.W * ring.H
    L, gx, gy, gt = (np.empty(P) for _ in range(4))
    lib().afo_gradients(ring.W, ring.H, ring.b, _p(ring.count), _p(ring.slot), _p(ring.seq),
                        t_now, _p(L), _p(gx), _p(gy), _p(gt))
    return L, gx, gy, gt


def tile_feedback(ring: Ring, grads, S: int = 32, t_now: float = 1.0, m: float = 2.0):
    ntx, nty = -(-ring.W // S), -(-ring.H // S)
    out = np.empty((ntx * nty, NT))
    _, gx, gy, gt = grads
    lib().afo_tile_feedback(ring.W, ring.H, ring.b, S, _p(ring.count), _p(ring.slot), t_now,
                            _p(gx), _p(gy), _p(gt), m, _p(out))
    return out


def tile_error(ring: Ring, tiles, S: int = 32, t_now: float = 1.0, occluded=None, kappa: float = 0.5,
               lam: float = 0.5, importance: float = 1.0, eps: float = 1e-4):
    """Per-tile error E and gain control (dC/ds, dC/dt, T, S*, N*) from the
    records of tile_feedback (sections 6.1 and 4.1)."""
    tiles = np.ascontiguousarray(tiles, np.float64)
    E = np.zeros(tiles.shape[0])
    gain = np.zeros(5)
    occ = None if occluded is None else np.ascontiguousarray(occluded, np.float64)
    lib().afo_tile_error(ring.W, ring.H, ring.b, S, _p(ring.count), _p(ring.slot), t_now, _p(tiles),
                         None if occ is None else _p(occ), kappa, lam, importance, eps, _p(E), _p(gain))
    return E, gain


def reproject(ring: Ring, t_now: float = 1.0):
    P = ring.W * ring.H
    cap = max(1, ring.resident)
    off = np.zeros(P + 1, np.uint32)
    rec = np.zeros((cap, NR), np.float32)
    rseq = np.zeros(cap, np.uint32)
    dropped = ctypes.c_int64(0)
    n = lib().afo_reproject(ring.W, ring.H, ring.b, _p(ring.count), _p(ring.slot),
                            _p(ring.seq), t_now, _p(off), _p(rec), _p(rseq), cap,
                            ctypes.addressof(dropped))
    assert n >= 0
    return off, rec[:n].copy(), rseq[:n].copy(), dropped.value


def sigma(ring_count, W, H, grads, theta=DEFAULT_THETA, S: int = 32, window: float = 1.0,
          eps: float = 1e-4, b: int = 0):
    _, gx, gy, gt = grads
    th = np.ascontiguousarray(theta, np.float64)
    ss, st = np.empty(W * H), np.empty(W * H)
    cnt = np.ascontiguousarray(ring_count, np.int32)
    lib().afo_sigma(W, H, b, S, _p(cnt), _p(np.ascontiguousarray(gx)),
                    _p(np.ascontiguousarray(gy)), _p(np.ascontiguousarray(gt)), _p(th), window,
                    eps, _p(ss), _p(st))
    return ss, st


def filter_image(W, H, off, rec, sig_s, sig_t, R=4, t_now: float = 1.0, pixels=None):
    """R: one disc radius, or an array of W*H per-pixel radii."""
    out = np.zeros((W * H, 4))
    rec = np.ascontiguousarray(rec, np.float32)
    if rec.size == 0:
        rec = np.zeros((1, NR), np.float32)
    ss = np.ascontiguousarray(sig_s, np.float64)
    st = np.ascontiguousarray(sig_t, np.float64)
    if not np.isscalar(R):
        Rp = np.ascontiguousarray(R, np.int32).reshape(-1)
        assert Rp.size == W * H
        px = None if pixels is None else np.ascontiguousarray(pixels, np.int64)
        lib().afo_filter_var(W, H, _p(Rp), _p(off), _p(rec), t_now, _p(ss), _p(st),
                             None if px is None else _p(px), 0 if px is None else px.size, _p(out))
        return out
    if pixels is None:
        lib().afo_filter(W, H, R, _p(off), _p(rec), t_now, _p(ss), _p(st), None, 0, _p(out))
    else:
        px = np.ascontiguousarray(pixels, np.int64)
        lib().afo_filter(W, H, R, _p(off), _p(rec), t_now, _p(ss), _p(st), _p(px), px.size,
                         _p(out))
    return out


def filter_brute(W, H, rec, sig_s, sig_t, R=4, t_now: float = 1.0):
    """R: one disc radius, or an array of W*H per-pixel radii."""
    out = np.zeros((W * H, 4))
    rec = np.ascontiguousarray(rec, np.float32)
    n = rec.shape[0]
    if n == 0:
        rec = np.zeros((1, NR), np.float32)
    if not np.isscalar(R):
        Rp = np.ascontiguousarray(R, np.int32).reshape(-1)
        lib().afo_filter_brute_var(W, H, _p(Rp), n, _p(rec), t_now,
                                   _p(np.ascontiguousarray(sig_s, np.float64)),
                                   _p(np.ascontiguousarray(sig_t, np.float64)), _p(out))
        return out
    lib().afo_filter_brute(W, H, R, n, _p(rec), t_now,
                           _p(np.ascontiguousarray(sig_s, np.float64)),
                           _p(np.ascontiguousarray(sig_t, np.float64)), _p(out))
    return out


def backward(ring_count, W, H, grads, off, rec, grad_rgb, theta=DEFAULT_THETA, S: int = 32,
             R: int = 4, t_now: float = 1.0, window: float = 1.0, eps: float = 1e-4):
    _, gx, gy, gt = grads
    n = rec.shape[0]
    gcol = np.zeros((max(n, 1), 3))
    gth = np.zeros(NP)
    rec = np.ascontiguousarray(rec, np.float32) if n else np.zeros((1, NR), np.float32)
    lib().afo_backward(W, H, 0, S, R, _p(np.ascontiguousarray(ring_count, np.int32)),
                       _p(np.ascontiguousarray(gx)), _p(np.ascontiguousarray(gy)),
                       _p(np.ascontiguousarray(gt)),
                       _p(np.ascontiguousarray(theta, np.float64)), window, eps, _p(off),
                       _p(rec), t_now, _p(np.ascontiguousarray(grad_rgb, np.float64)),
                       _p(gcol), _p(gth))
    return gcol[:n], gth


def coverage_update(W, H, r_prev, n_prev, r_min: float = 0.5, r_max: float = 8.0):
    """Next footprint radii (float32 r, integer R) from the previous image's
    radii and sample counts (n_prev < 0: no information)."""
    rp = np.ascontiguousarray(r_prev, np.float32).reshape(-1)
    npv = np.ascontiguousarray(n_prev, np.int32).reshape(-1)
    r_next = np.zeros(W * H, np.float32)
    R_next = np.zeros(W * H, np.int32)
    lib().afo_coverage_update(W, H, _p(rp), _p(npv), r_min, r_max, _p(r_next), _p(R_next))
    return r_next, R_next


def coverage_count(W, H, Rp, off):
    n = np.zeros(W * H, np.int32)
    lib().afo_coverage_count(W, H, _p(np.ascontiguousarray(Rp, np.int32).reshape(-1)),
                             _p(np.ascontiguousarray(off, np.uint32)), _p(n))
    return n


def reconstruct_adaptive(ring: Ring, state: dict, t_now: float = 1.0, theta=DEFAULT_THETA, S: int = 32,
                         window: float = 1.0, eps: float = 1e-4, r_min: float = 0.5, r_max: float = 8.0,
                         pixels=None):
    """One image with footprints sized by the coverage of the previous one
    (section 6.2). state holds 'r' (float32 radii used last time) and 'n'
    (samples that reached each pixel, -1 if unknown); it is updated."""
    W, H = ring.W, ring.H
    grads = gradients(ring, t_now)
    off, rec, rseq, dropped = reproject(ring, t_now)
    ss, st = sigma(ring.count, W, H, grads, theta, S, window, eps)
    r, Rp = coverage_update(W, H, state["r"], state["n"], r_min, r_max)
    img = filter_image(W, H, off, rec, ss, st, Rp, t_now, pixels)
    state["r"], state["n"] = r, coverage_count(W, H, Rp, off)
    return {"off": off, "rec": rec, "sig_s": ss, "sig_t": st, "R": Rp, "image": img}


def reconstruct(ring: Ring, t_now: float = 1.0, theta=DEFAULT_THETA, S: int = 32, R: int = 4,
                window: float = 1.0, eps: float = 1e-4, m: float = 2.0, pixels=None):
    """The whole forward path on the oracle: gradients, tile statistics,
    reprojection, widths and the filter."""
    grads = gradients(ring, t_now)
    tiles = tile_feedback(ring, grads, S, t_now, m)
    off, rec, rseq, dropped = reproject(ring, t_now)
    ss, st = sigma(ring.count, ring.W, ring.H, grads, theta, S, window, eps)
    img = filter_image(ring.W, ring.H, off, rec, ss, st, R, t_now, pixels)
    return {"grads": grads, "tiles": tiles, "off": off, "rec": rec, "rseq": rseq,
            "dropped": dropped, "sig_s": ss, "sig_t": st, "image": img}
