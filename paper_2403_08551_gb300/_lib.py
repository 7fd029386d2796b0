"""ctypes binding of libgi (include/gi.h): argument marshalling only.

Every function here forwards torch tensors (device memory) and the current
torch CUDA stream to the C ABI. No computation of the method happens in
Python; if libgi.so is missing, loading fails with an error (there is no CPU
fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# GI_LIB_VARIANT=check loads the bounds-checking build (see build.py).
LIB_PATH = os.path.join(HERE, "_build_check" if os.environ.get("GI_LIB_VARIANT") == "check" else "_build",
                        "libgi.so")

P = ctypes.c_void_p
i32, i64, f32, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
size_t = ctypes.c_size_t

GI_OK = 0
STATUS = {0: "GI_OK", 1: "GI_ERR_INVALID_ARG", 2: "GI_ERR_CUDA", 3: "GI_ERR_CAPACITY",
          4: "GI_ERR_TIMEOUT", 5: "GI_ERR_UNSUPPORTED", 6: "GI_ERR_NO_MEMORY"}
DEVERR_CAPACITY, DEVERR_TIMEOUT, DEVERR_BOUNDS = 1, 2, 4

(FIT_PARAMS, FIT_ADAM_M, FIT_ADAM_V, FIT_GRADS, FIT_OUT, FIT_LOSS, FIT_STEP, FIT_K, FIT_TARGET, FIT_ADAN_N,
 FIT_ADAN_GPREV, FIT_CODEC_GB, FIT_CODEBOOKS, FIT_EMA_COUNT, FIT_EMA_TOTAL, FIT_CODES, FIT_RVQ_IDX,
 FIT_CODEC_OUT, FIT_OPACITY, FIT_N_LAST, FIT_KEYS, FIT_IDS, FIT_RANGES, FIT_PAIR_OFF, FIT_RECT, FIT_CNT,
 FIT_MEANS16) = range(27)

# Every symbol include/gi.h declares, with (restype, argtypes).
SIGNATURES = {
    "gi_abi_version": (i32, []),
    "gi_last_error": (ctypes.c_char_p, []),
    "gi_status_string": (ctypes.c_char_p, [i32]),
    "gi_device_errors": (i32, [P, i32, P]),
    "gi_project": (i32, [P, P, P, i32, None, P, P, P, P]),
    "gi_bin_workspace_size": (i32, [i32, None, i64, P]),
    "gi_bin_tiles": (i32, [P, P, P, i32, None, i64, P, size_t, P, P, P, P, P, P, P]),
    "gi_bin_tiles_noalloc": (i32, [P, P, P, i32, None, i64, P, P, P, P, P, P, P]),
    "gi_render": (i32, [P, P, None, P, P, P, P, P]),
    "gi_backward_workspace_size": (i32, [i32, None, i64, P]),
    "gi_render_backward": (i32, [P, P, P, P, P, P, P, P, P, i32, None, i64, P, P, size_t, P, P, P, P, P]),
    "gi_vq_decode": (i32, [P, P, P, i32, i32, i32, P, P, P, P]),
    "gi_codec_decode": (i32, [P, P, P, P, P, i32, i32, i32, P, P, P, P]),
    "gi_fit_create": (i32, [P, P, P]),
    "gi_fit_step": (i32, [P, i32, P]),
    "gi_fit_render": (i32, [P, P]),
    "gi_fit_set_target_source": (i32, [P, P, P]),
    "gi_fit_pointer": (i32, [P, i32, P]),
    "gi_fit_count_pairs": (i32, [P, P, P]),
    "gi_fit_destroy": (i32, [P]),
    "gi_fit_stage_times": (i32, [P, P]),
    "gi_alu_peaks": (i32, [P, P]),
    "gi_selftest_bounded_waits": (i32, [P, i64, P]),
}


class GIImage(ctypes.Structure):
    _fields_ = [("width", i32), ("height", i32), ("tile", i32)]


class GIFitDesc(ctypes.Structure):
    _fields_ = [("n_images", i32), ("widths", P), ("heights", P), ("counts", P), ("targets", P),
                ("params", P), ("tile", i32), ("lr_means", f32), ("lr_chol", f32), ("lr_color", f32),
                ("beta1", f32), ("beta2", f32), ("eps", f32), ("capacity", i64), ("use_graph", i32),
                ("stage_events", i32), ("render_split", i32), ("param_mode", i32), ("optimizer", i32),
                ("beta3", f32), ("lr_halve_every", i32), ("cov_mode", i32), ("codec_bits", i32),
                ("codec_stages", i32), ("codec_size", i32), ("codebooks", P), ("lsq_gamma", f32 * 3),
                ("lsq_beta", f32 * 3), ("ema_decay", f32), ("ema_eps", f32), ("opacity_mode", i32),
                ("opacity_logits", P), ("tile_queue", i32)]


class GIError(RuntimeError):
    pass


_lock = threading.Lock()
_lib = None


def load():
    """Load libgi.so (built by ``paper_2403_08551_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise GIError(f"libgi.so not built ({LIB_PATH}); run __graft_entry__.build() first")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = [GIImage if a is None else a for a in args]
            _lib = lib
    return _lib


def check(status: int, what: str = ""):
    if status != GI_OK:
        msg = load().gi_last_error().decode(errors="replace")
        raise GIError(f"{what or 'libgi'}: {STATUS.get(status, status)}: {msg}")


def ptr(t):
    """Device (or host) address of a tensor, or None."""
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def stream_handle(device=None):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
