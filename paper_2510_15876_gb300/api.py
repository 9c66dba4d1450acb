"""Python binding of the reconstruction library (argument marshalling only).

Every compute step runs in the CUDA kernels of libafr.so; torch only provides
device memory and the current stream. The names follow the C ABI
(include/afr.h), which cites the passage of the paper each call implements.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L

_COLOR_TYPES = {"f32": L.AFR_F32, "f16": L.AFR_F16, "bf16": L.AFR_BF16}
_COLOR_DTYPES = {L.AFR_F32: torch.float32, L.AFR_F16: torch.float16, L.AFR_BF16: torch.bfloat16}
DEFAULT_PARAMS = (1.0, 0.0, 3.0, 1.0, 0.0, 1.0)
TILE_FIELDS = ("n", "empty_slots", "mean_L", "var_L", "mean_Gx", "mean_Gy", "mean_Gt", "u")


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _params(p) -> L.AfrParams:
    if p is None:
        p = DEFAULT_PARAMS
    if isinstance(p, torch.Tensor):
        p = p.detach().to("cpu", torch.float64).tolist()
    return L.AfrParams(*[float(v) for v in p])


class Reconstructor:
    """One reconstruction context: the deep buffer of a width x height image
    with queues of depth `depth`, and everything derived from it."""

    def __init__(self, width: int, height: int, depth: int, *, tile: int = 32, radius: int = 4,
                 color_type: str = "f32", window: float = 1.0, eps_grad: float = 1e-4,
                 undersample_m: float = 2.0, fifo_capacity: int = 0, world_points: bool = False, device=None,
                 lib=None):
        """lib: the loaded library to use (default libafr.so; L.load_debug()
        gives the AFR_DEBUG build)."""
        self.lib = lib if lib is not None else L.load()
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.type != "cuda":
            raise ValueError("the reconstruction library runs on CUDA devices only")
        torch.cuda.set_device(self.device)
        self.W, self.H, self.b, self.S, self.R = width, height, depth, tile, radius
        self.ct = _COLOR_TYPES[color_type]
        self.color_dtype = _COLOR_DTYPES[self.ct]
        cfg = L.AfrConfig(width, height, depth, tile, radius, self.ct, window, eps_grad, undersample_m, fifo_capacity,
                          1 if world_points else 0)
        h = ctypes.c_void_p()
        st = self.lib.afr_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != L.AFR_OK:
            raise L.AfrError(st, "afr_create failed")
        self.h = h
        n = ctypes.c_uint32()
        self._check(self.lib.afr_num_tiles(self.h, ctypes.byref(n)))
        self.n_tiles = n.value
        self._side = None                 # refresh(): stream of the gradient branch
        self._fork, self._join = torch.cuda.Event(), torch.cuda.Event()

    # -- plumbing ------------------------------------------------------------------
    def _check(self, st: int):
        if st != L.AFR_OK:
            msg = self.lib.afr_last_error(self.h) if getattr(self, "h", None) else b""
            raise L.AfrError(st, (msg or b"").decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.afr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the path ------------------------------------------------------------------
    def reset(self, stream=None):
        self._check(self.lib.afr_reset(self.h, _stream(stream)))

    def reserve(self, n: int):
        self._check(self.lib.afr_reserve(self.h, n))

    def insert(self, pos: torch.Tensor, color: torch.Tensor, motion: torch.Tensor, world: torch.Tensor | None = None,
               stream=None, reset: bool = False, queues_free=None):
        """world: [n, 4] float32 hit points (X, Y, Z, -) for world_points contexts.
        reset: clear the queues first (as reset() then insert()). queues_free
        (a recorded torch.cuda.Event): the steps that touch the queues wait
        for it, the binning before them does not (afr_insert_samples_ex)."""
        n = pos.shape[0]
        arrays = [(pos, torch.float32, 4), (color, self.color_dtype, 4), (motion, torch.float32, 2)]
        if world is not None:
            arrays.append((world, torch.float32, 4))
        for t, dt, cols in arrays:
            if t.device != self.device or t.dtype != dt or not t.is_contiguous() or tuple(t.shape) != (n, cols):
                raise ValueError(f"batch tensor must be contiguous {dt} [{n}, {cols}] on {self.device}")
        batch = L.AfrSampleBatch(pos.data_ptr(), color.data_ptr(), motion.data_ptr(),
                                 None if world is None else world.data_ptr())
        if not reset and queues_free is None:
            self._check(self.lib.afr_insert_samples(self.h, ctypes.byref(batch), n, _stream(stream)))
            return
        ev = None if queues_free is None else ctypes.c_void_p(queues_free.cuda_event)
        self._check(self.lib.afr_insert_samples_ex(self.h, ctypes.byref(batch), n,
                                                   L.AFR_INSERT_RESET if reset else 0, ev, _stream(stream)))

    def estimate_gradients(self, t_now: float = 1.0, stream=None):
        self._check(self.lib.afr_estimate_gradients(self.h, t_now, _stream(stream)))

    def reproject(self, t_now: float = 1.0, stream=None):
        self._check(self.lib.afr_reproject(self.h, t_now, _stream(stream)))

    def reproject_camera(self, t_now: float, view_proj, stream=None):
        """Frame view from the stored hit points rendered by the row-major 4x4
        view_proj (section 6.2)."""
        m = (ctypes.c_float * 16)(*[float(v) for v in np.asarray(view_proj, np.float32).reshape(16)])
        self._check(self.lib.afr_reproject_camera(self.h, t_now, m, _stream(stream)))

    def reconstruct(self, t_now: float = 1.0, params=None, out: torch.Tensor | None = None, flags: int = 0,
                    stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.H, self.W, 4), dtype=torch.float32, device=self.device)
        prm = _params(params)
        self._check(self.lib.afr_reconstruct_ex(self.h, t_now, ctypes.byref(prm), flags, _ptr(out),
                                                _stream(stream)))
        return out

    def tile_feedback(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Raw AfrTileStats records as a [n_tiles, 8] float32 tensor (fields n
        and empty_slots hold uint32 bits; see decode_tiles)."""
        if out is None:
            out = torch.empty((self.n_tiles, 8), dtype=torch.float32, device=self.device)
        self._check(self.lib.afr_tile_feedback(self.h, _ptr(out), _stream(stream)))
        return out

    def refresh(self, t_now: float = 1.0, out: torch.Tensor | None = None, tiles: torch.Tensor | None = None,
                params=None, flags: int = 0, stream=None, side_stream=None, reads_done=None, view_proj=None):
        """One displayed image from the buffered samples: the gradients
        (sections 4, 4.1) and the tile statistics (sections 4.2, 6.1) on
        side_stream while the samples are reprojected (section 6.2) on
        stream, then the widths and the filter (sections 5.1, 5.2) on stream
        once both are done. The two branches read the sample buffers and
        write disjoint state. reads_done (a torch.cuda.Event), if given, is
        recorded on stream when both branches are done with the sample
        buffers, before the filter: an insert of the next batch on another
        stream that waits for it overlaps the filter (the filter reads no
        sample buffer). view_proj, if given, reprojects the stored hit points
        with that camera (reproject_camera) instead of the screen motion.
        Returns (image, tile statistics)."""
        main = stream if stream is not None else torch.cuda.current_stream(self.device)
        if side_stream is None:
            if self._side is None:
                self._side = torch.cuda.Stream(self.device, priority=-1)
            side_stream = self._side
        if tiles is None:
            tiles = torch.empty((self.n_tiles, 8), dtype=torch.float32, device=self.device)
        if out is None:
            out = torch.empty((self.H, self.W, 4), dtype=torch.float32, device=self.device)
        self._fork.record(main)
        side_stream.wait_event(self._fork)
        self.estimate_gradients(t_now, stream=side_stream)
        self.tile_feedback(out=tiles, stream=side_stream)
        self._join.record(side_stream)
        if view_proj is None:
            self.reproject(t_now, stream=main)
        else:
            self.reproject_camera(t_now, view_proj, stream=main)
        main.wait_event(self._join)
        if reads_done is not None:
            reads_done.record(main)
        self.reconstruct(t_now, params, out, flags, stream=main)
        return out, tiles

    GAIN_KEYS = ("dC_ds", "dC_dt", "mean_age", "tile_width", "tile_count")

    def tile_error(self, kappa: float = 0.5, lam: float = 0.5, importance: float = 1.0,
                   occluded: torch.Tensor | None = None, stream=None, out=None, gain_on_device: bool = False):
        """Per-tile error E (sections 6.1) as a [n_tiles] float32 tensor and the
        gain control (section 4.1) as a dict; with gain_on_device, the gain
        record stays on the device as a float32 tensor of the five
        GAIN_KEYS values and nothing waits for the stream. out = (E, gain)
        tensors to fill instead of new ones."""
        if out is not None:
            E, g = out
        else:
            E = torch.empty(self.n_tiles, dtype=torch.float32, device=self.device)
            g = torch.empty(5, dtype=torch.float32, device=self.device)
        occ = None
        if occluded is not None:
            occ = occluded.to(self.device, torch.int32).contiguous()
            if occ.numel() != self.n_tiles:
                raise ValueError(f"occluded needs {self.n_tiles} counts")
        self._check(self.lib.afr_tile_error(self.h, kappa, lam, importance, _ptr(occ), _ptr(E), _ptr(g),
                                            _stream(stream)))
        if gain_on_device:
            return E, g
        return E, dict(zip(self.GAIN_KEYS, g.cpu().tolist()))

    def backward(self, grad_rgbw: torch.Tensor, want_colors: bool = True, want_params: bool = True,
                 n_frame: int | None = None, stream=None):
        grad_rgbw = grad_rgbw.contiguous()
        gcol = gprm = None
        if want_colors:
            if n_frame is None:
                n_frame = self.query(stream)["frame"]
            gcol = torch.empty((max(n_frame, 1), 3), dtype=torch.float32, device=self.device)
        if want_params:
            gprm = torch.empty(6, dtype=torch.float32, device=self.device)
        self._check(self.lib.afr_reconstruct_backward(self.h, _ptr(grad_rgbw), _ptr(gcol), _ptr(gprm),
                                                      _stream(stream)))
        if gcol is not None:
            gcol = gcol[:n_frame]
        return gcol, gprm

    def set_frame_colors(self, rgb: torch.Tensor, stream=None):
        rgb = rgb.to(self.device, torch.float32).contiguous()
        self._check(self.lib.afr_set_frame_colors(self.h, _ptr(rgb), _stream(stream)))

    def profile_filter(self, enable: bool = True):
        """Start (or stop) recording the filter kernel's duration per reconstruct call."""
        self._check(self.lib.afr_profile_filter(self.h, 1 if enable else 0))

    def profile_read(self) -> list[float]:
        """Durations (ms) of the filter launches recorded since profile_filter(True)."""
        buf = (ctypes.c_float * L.AFR_PROFILE_MAX_LAUNCHES)()
        n = ctypes.c_int32()
        self._check(self.lib.afr_profile_read(self.h, buf, L.AFR_PROFILE_MAX_LAUNCHES, ctypes.byref(n)))
        return [buf[k] for k in range(min(n.value, L.AFR_PROFILE_MAX_LAUNCHES))]

    # -- inspection ----------------------------------------------------------------
    def status(self, stream=None) -> int:
        """afr_get_status: waits for the work issued on stream (default: the
        current stream) and returns the device status word's condition."""
        return self.lib.afr_get_status(self.h, _stream(stream))

    def query(self, stream=None) -> dict:
        info = L.AfrInfo()
        self._check(self.lib.afr_query(self.h, ctypes.byref(info), _stream(stream)))
        return {f: getattr(info, f) for f, _ in L.AfrInfo._fields_}

    def export_ring(self):
        P, b = self.W * self.H, self.b
        count = np.zeros(P, np.int32)
        slot = np.zeros((P, b, 9), np.float32)
        seq = np.zeros((P, b), np.uint32)
        self._check(self.lib.afr_export_ring(self.h, count.ctypes.data, slot.ctypes.data, seq.ctypes.data))
        return count, slot, seq

    def export_frame(self):
        info = self.query()
        n = max(int(info["frame"]), 1)
        off = np.zeros(self.W * self.H + 1, np.uint32)
        rec = np.zeros((n, 6), np.float32)
        seq = np.zeros(n, np.uint32)
        self._check(self.lib.afr_export_frame(self.h, off.ctypes.data, rec.ctypes.data, seq.ctypes.data, n))
        m = int(off[-1])
        return off, rec[:m], seq[:m]

    def export_map(self, which: int) -> np.ndarray:
        out = np.zeros(self.W * self.H, np.float32)
        self._check(self.lib.afr_export_map(self.h, which, out.ctypes.data))
        return out

    def import_map(self, which: int, arr):
        a = np.ascontiguousarray(arr, np.float32).reshape(-1)
        assert a.size == self.W * self.H
        self._check(self.lib.afr_import_map(self.h, which, a.ctypes.data))


def decode_tiles(raw: torch.Tensor) -> dict:
    r = raw.detach().cpu().contiguous()
    u = r.view(torch.int32)
    out = {"n": u[:, 0].numpy().astype(np.uint32), "empty_slots": u[:, 1].numpy().astype(np.uint32)}
    for k, f in enumerate(TILE_FIELDS[2:], start=2):
        out[f] = r[:, k].numpy()
    return out


def to_device_batch(batch: dict, device, color_dtype=torch.float32):
    """Upload a workload batch (numpy arrays pos/color/motion) as contiguous tensors."""
    pos = torch.from_numpy(np.ascontiguousarray(batch["pos"], np.float32)).to(device)
    col = torch.from_numpy(np.ascontiguousarray(batch["color"], np.float32)).to(device).to(color_dtype)
    mo = torch.from_numpy(np.ascontiguousarray(batch["motion"], np.float32)).to(device)
    return pos.contiguous(), col.contiguous(), mo.contiguous()


class BatchReconstructor:
    """Many Reconstructors of one colour type reconstructed in one persistent
    launch (afr_batch_reconstruct). The contexts must outlive the batch; their
    filter tile shapes are frozen at creation."""

    def __init__(self, recs: list[Reconstructor]):
        self.lib = L.load()
        self.recs = list(recs)
        arr = (ctypes.c_void_p * len(recs))(*[r.h.value for r in recs])
        h = ctypes.c_void_p()
        st = self.lib.afr_batch_create(arr, len(recs), ctypes.byref(h))
        if st != L.AFR_OK:
            raise L.AfrError(st, "afr_batch_create failed")
        self.h = h
        self.outs = [torch.empty((r.H, r.W, 4), dtype=torch.float32, device=r.device) for r in recs]
        self._ptrs = (ctypes.c_void_p * len(recs))(*[o.data_ptr() for o in self.outs])

    def run(self, t_now: float = 1.0, params=None, stream=None) -> list[torch.Tensor]:
        prm = _params(params)
        st = self.lib.afr_batch_reconstruct(self.h, t_now, ctypes.byref(prm), self._ptrs, _stream(stream))
        if st != L.AFR_OK:
            raise L.AfrError(st, "afr_batch_reconstruct failed")
        return self.outs

    def refresh(self, t_now: float = 1.0, params=None, stream=None) -> list[torch.Tensor]:
        """afr_batch_refresh: gradients, reprojection and filter of every
        context, spread over the batch's worker streams."""
        prm = _params(params)
        st = self.lib.afr_batch_refresh(self.h, t_now, ctypes.byref(prm), self._ptrs, _stream(stream))
        if st != L.AFR_OK:
            raise L.AfrError(st, "afr_batch_refresh failed")
        return self.outs

    def close(self):
        if getattr(self, "h", None):
            self.lib.afr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_alu_peaks() -> dict:
    """Measured FP32 rates of the current device (afr_measure_alu_peaks)."""
    lib = L.load()
    out = (ctypes.c_float * 4)()
    st = lib.afr_measure_alu_peaks(out)
    if st != L.AFR_OK:
        raise L.AfrError(st, "afr_measure_alu_peaks failed")
    return {"fma_tflops": out[0], "fma2_tflops": out[1], "ex2_tops": out[2], "sms": int(out[3])}


def set_tuning(rec: Reconstructor, radius: int, tile_bx: int):
    rec._check(rec.lib.afr_set_tuning(rec.h, radius, tile_bx))
    rec.R = radius
    rec.tile_bx = tile_bx
