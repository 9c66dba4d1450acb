"""GB300-native reconstruction path of adaptive frameless rendering.

Dayal, Woolley, Watson and Luebke, "Adaptive Frameless Rendering": samples
are binned into a temporally deep per-pixel buffer, space-time colour
gradients are estimated from it, buffered samples are reprojected to the
display time, and each pixel is filtered with a space-time Gaussian whose
widths adapt to the gradients and the local sample density; per-tile
statistics are returned to the sampler. All of it runs in the CUDA kernels of
libafr.so behind the C ABI of include/afr.h.
"""
from . import _lib  # noqa: F401

__all__ = ["Reconstructor", "reconstruct", "decode_tiles", "build"]


def build(force: bool = False):
    from .build import build as _build
    return _build(force=force)


def __getattr__(name):
    if name in ("Reconstructor", "decode_tiles", "to_device_batch"):
        from . import api
        return getattr(api, name)
    if name == "reconstruct":
        from .autograd import reconstruct
        return reconstruct
    raise AttributeError(name)
