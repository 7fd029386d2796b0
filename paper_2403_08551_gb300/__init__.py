"""GB300-native accumulated-summation rasterizer for 2D Gaussians
(GaussianImage, arXiv 2403.08551).

The compute path is libgi.so (CUDA kernels for sm_103a behind the C ABI in
include/gi.h); this package is its Python binding: per-stage calls, an
autograd Function and multi-image fitting contexts.
"""
from .api import (RENDER_SPLITS, Bins, Fit, GIRender, Renderer, alu_peaks, autotune, bin_tiles, codec_decode, codec_init,
                  device_errors, project, rasterize, render, render_backward, selftest_bounded_waits, tiles,
                  vq_decode)
from ._lib import GIError, load

__all__ = ["RENDER_SPLITS", "Bins", "Fit", "GIRender", "Renderer", "GIError", "alu_peaks", "autotune", "bin_tiles",
           "codec_decode", "codec_init",
           "device_errors", "load", "project", "rasterize", "render", "render_backward",
           "selftest_bounded_waits", "tiles", "vq_decode"]
