"""Python API over libgi: per-stage calls, an autograd Function and fitting
contexts. Torch supplies device memory and the current CUDA stream; every
step of the rasterizer runs in libgi's kernels.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import List, Optional, Sequence

import torch

from . import _lib as L

__all__ = ["project", "bin_tiles", "render", "render_backward", "vq_decode", "device_errors",
           "GIRender", "rasterize", "Fit", "Bins", "alu_peaks", "tiles", "autotune", "RENDER_SPLITS", "Renderer",
           "selftest_bounded_waits", "codec_init", "codec_decode", "ADAN_BETAS"]

# Render splits (lane groups sharing one tile's list) available per tile edge.
RENDER_SPLITS = {8: (2, 4), 16: (4, 8), 32: (1, 2)}


def tiles(W: int, H: int, T: int):
    return (W + T - 1) // T, (H + T - 1) // T


def _dev(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t.contiguous()


def _img(W, H, T):
    return L.GIImage(int(W), int(H), int(T))


def device_errors(clear: bool = True) -> int:
    bits = ctypes.c_uint32(0)
    L.check(L.load().gi_device_errors(ctypes.byref(bits), int(clear), L.stream_handle()), "gi_device_errors")
    return bits.value


def project(means, chol, color, W: int, H: int, tile: int = 16):
    """Formation (Eq. 1): returns rec [n,8], rect [n,4] int32, cnt [n] int32."""
    means = _dev(means, torch.float32, "means")
    chol = _dev(chol, torch.float32, "chol")
    color = _dev(color, torch.float32, "color")
    n = means.shape[0]
    rec = torch.empty((n, 8), dtype=torch.float32, device=means.device)
    rect = torch.empty((n, 4), dtype=torch.int32, device=means.device)
    cnt = torch.empty((n,), dtype=torch.int32, device=means.device)
    L.check(L.load().gi_project(L.ptr(means), L.ptr(chol), L.ptr(color), n, _img(W, H, tile), L.ptr(rec),
                                L.ptr(rect), L.ptr(cnt), L.stream_handle()), "gi_project")
    return rec, rect, cnt


@dataclass
class Bins:
    keys: torch.Tensor
    ids: torch.Tensor
    ranges: torch.Tensor
    rec_binned: Optional[torch.Tensor]
    pair_off: torch.Tensor
    k_dev: torch.Tensor
    K: int
    capacity: int


def bin_tiles(rect, cnt, rec, W: int, H: int, tile: int = 16, capacity: Optional[int] = None) -> Bins:
    """Tile binning. With ``capacity=None`` the pair count is read back and
    the call is repeated once with an exact capacity if the guess was short
    (one host synchronisation)."""
    lib = L.load()
    n = cnt.shape[0]
    dev = cnt.device
    rect = _dev(rect, torch.int32, "rect")
    cnt = _dev(cnt, torch.int32, "cnt")
    rec = None if rec is None else _dev(rec, torch.float32, "rec")
    tw, th = tiles(W, H, tile)
    auto = capacity is None
    cap = int(capacity) if capacity else max(4096, 8 * n)
    for _ in range(2):
        ws_bytes = ctypes.c_size_t(0)
        L.check(lib.gi_bin_workspace_size(n, _img(W, H, tile), cap, ctypes.byref(ws_bytes)), "gi_bin_workspace_size")
        ws = torch.empty((ws_bytes.value + 256,), dtype=torch.uint8, device=dev)
        keys = torch.empty((cap,), dtype=torch.int32, device=dev)
        ids = torch.empty((cap,), dtype=torch.int32, device=dev)
        ranges = torch.empty((tw * th, 2), dtype=torch.int32, device=dev)
        rec_binned = torch.empty((cap, 8), dtype=torch.float32, device=dev) if rec is not None else None
        pair_off = torch.empty((n + 1,), dtype=torch.int64, device=dev)
        k_dev = torch.empty((1,), dtype=torch.int64, device=dev)
        L.check(lib.gi_bin_tiles(L.ptr(rect) if n else None, L.ptr(cnt) if n else None, L.ptr(rec) if n else None,
                                 n, _img(W, H, tile), cap, L.ptr(ws), ws_bytes.value, L.ptr(keys), L.ptr(ids),
                                 L.ptr(ranges), L.ptr(rec_binned) if rec is not None else None, L.ptr(pair_off),
                                 L.ptr(k_dev), L.stream_handle()), "gi_bin_tiles")
        K = int(k_dev.item())
        if K <= cap:
            return Bins(keys, ids, ranges, rec_binned, pair_off, k_dev, K, cap)
        if not auto:
            raise L.GIError(f"gi_bin_tiles: {K} pairs exceed capacity {cap}")
        device_errors(clear=True)  # drop the capacity bit raised by the short guess
        cap = K
    raise L.GIError("gi_bin_tiles: capacity retry failed")


def render(bins: Bins, W: int, H: int, tile: int = 16, target=None, want_dl: bool = False):
    """Accumulated-summation render (Eq. 7); with a target also the L2 loss
    (mean over 3HW) and optionally dL/dC. Returns (out, dl or None, loss or None)."""
    dev = bins.ranges.device
    out = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    dl = loss = None
    if target is not None:
        target = _dev(target, torch.float32, "target")
        loss = torch.zeros((1,), dtype=torch.float64, device=dev)
        if want_dl:
            dl = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    L.check(L.load().gi_render(L.ptr(bins.rec_binned), L.ptr(bins.ranges), _img(W, H, tile), L.ptr(target),
                               L.ptr(out), L.ptr(dl), L.ptr(loss), L.stream_handle()), "gi_render")
    if loss is not None:
        loss = loss / (3.0 * W * H)
    return out, dl, loss


def render_backward(bins: Bins, rect, cnt, chol, dl_dout, W: int, H: int, tile: int = 16, want_conic=False):
    """Gradients (App. A.1, A.2): returns g_means [n,2], g_chol [n,3],
    g_color [n,3] and g_conic [n,3] (or None)."""
    lib = L.load()
    n = cnt.shape[0]
    dev = cnt.device
    chol = _dev(chol, torch.float32, "chol")
    dl_dout = _dev(dl_dout, torch.float32, "dl_dout")
    ws_bytes = ctypes.c_size_t(0)
    L.check(lib.gi_backward_workspace_size(n, _img(W, H, tile), bins.capacity, ctypes.byref(ws_bytes)),
            "gi_backward_workspace_size")
    ws = torch.empty((ws_bytes.value + 256,), dtype=torch.uint8, device=dev)
    gm = torch.empty((n, 2), dtype=torch.float32, device=dev)
    gl = torch.empty((n, 3), dtype=torch.float32, device=dev)
    gc = torch.empty((n, 3), dtype=torch.float32, device=dev)
    gq = torch.empty((n, 3), dtype=torch.float32, device=dev) if want_conic else None
    L.check(lib.gi_render_backward(L.ptr(bins.rec_binned), L.ptr(bins.keys), L.ptr(bins.ids), L.ptr(bins.ranges),
                                   L.ptr(rect), L.ptr(cnt), L.ptr(bins.pair_off), L.ptr(bins.k_dev), L.ptr(chol), n,
                                   _img(W, H, tile), bins.capacity, L.ptr(dl_dout), L.ptr(ws), ws_bytes.value,
                                   L.ptr(gm), L.ptr(gl), L.ptr(gc), L.ptr(gq), L.stream_handle()),
            "gi_render_backward")
    return gm, gl, gc, gq


def vq_decode(means16, idx, codebooks, out=None):
    """Codec decode (Sec. 3.3). means16 [n,2] float16 or int16/uint16 bits,
    idx [2,M,n] uint8, codebooks [2,M,B,3] float32. out: optional
    preallocated (means [n,2], chol [n,3], color [n,3]) float32 tensors."""
    lib = L.load()
    if means16.dtype == torch.float16:
        means16 = means16.view(torch.int16)
    means16 = means16.contiguous()
    idx = _dev(idx, torch.uint8, "idx")
    cb = _dev(codebooks, torch.float32, "codebooks")
    n = means16.shape[0]
    M, B = cb.shape[1], cb.shape[2]
    dev = means16.device
    if out is None:
        means = torch.empty((n, 2), dtype=torch.float32, device=dev)
        chol = torch.empty((n, 3), dtype=torch.float32, device=dev)
        color = torch.empty((n, 3), dtype=torch.float32, device=dev)
    else:
        means, chol, color = (_dev(t, torch.float32, "out") for t in out)
    L.check(lib.gi_vq_decode(L.ptr(means16), L.ptr(idx), L.ptr(cb), n, M, B, L.ptr(means), L.ptr(chol),
                             L.ptr(color), L.stream_handle()), "gi_vq_decode")
    return means, chol, color


def codec_decode(stream: dict):
    """Decode of the paper's codec stream (Sec. 3.3), as `Fit.encode` returns
    it: means16 [n,2] binary16 bits (int16/uint16 or float16), codes [n,4]
    uint8, gamma_beta (6 floats: gamma, beta), idx [M,n] uint8, codebooks
    [M,B,3] float32. Returns pixel-space means [n,2], Cholesky vectors [n,3]
    and colours [n,3] (float32, on the device of means16)."""
    lib = L.load()
    m16 = stream["means16"]
    if m16.dtype == torch.float16:
        m16 = m16.view(torch.int16)
    m16 = m16.contiguous()
    codes = _dev(stream["codes"], torch.uint8, "codes")
    idx = _dev(stream["idx"], torch.uint8, "idx")
    cb = _dev(stream["codebooks"], torch.float32, "codebooks")
    gb = (ctypes.c_float * 6)(*[float(x) for x in stream["gamma_beta"]])
    n = m16.shape[0]
    M, B = cb.shape[0], cb.shape[1]
    dev = m16.device
    means = torch.empty((n, 2), dtype=torch.float32, device=dev)
    chol = torch.empty((n, 3), dtype=torch.float32, device=dev)
    color = torch.empty((n, 3), dtype=torch.float32, device=dev)
    L.check(lib.gi_codec_decode(L.ptr(m16), L.ptr(codes), ctypes.cast(gb, ctypes.c_void_p), L.ptr(idx), L.ptr(cb), n,
                                M, B, L.ptr(means), L.ptr(chol), L.ptr(color), L.stream_handle()), "gi_codec_decode")
    return means, chol, color


class GIRender(torch.autograd.Function):
    """Differentiable render: forward runs formation, binning and Eq. 7;
    backward recomputes the weights per tile (no per-pixel state saved)."""

    @staticmethod
    def forward(ctx, means, chol, color, W: int, H: int, tile: int = 16):
        rec, rect, cnt = project(means, chol, color, W, H, tile)
        bins = bin_tiles(rect, cnt, rec, W, H, tile)
        out, _, _ = render(bins, W, H, tile)
        ctx.save_for_backward(chol.detach().contiguous(), rect, cnt)
        ctx.bins = bins
        ctx.meta = (W, H, tile)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        chol, rect, cnt = ctx.saved_tensors
        W, H, tile = ctx.meta
        gm, gl, gc, _ = render_backward(ctx.bins, rect, cnt, chol, grad_out.contiguous(), W, H, tile)
        return gm, gl, gc, None, None, None


def rasterize(means, chol, color, W: int, H: int, tile: int = 16):
    return GIRender.apply(means, chol, color, W, H, tile)


class _DevArray:
    """Zero-copy view of device memory owned by a Fit context."""

    def __init__(self, addr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (addr, False),
                                         "version": 3, "strides": None}


# Adan's decay factors of its three averages (Adan's 0.02, 0.08, 0.01).
ADAN_BETAS = (0.98, 0.92, 0.99)
# Table 3's forms: merged colour c' (the paper's), separate opacity with
# accumulated summation ("w/o M"), separate opacity with alpha-blending ("w/o AR").
OPACITY_MODES = {"merged": 0, "separate": 1, "blend": 2}
CODEC_EMA_DECAY = 0.99  # codebook EMA decay (the paper gives none; the common VQ-VAE value)
CODEC_EMA_EPS = 1e-5    # Laplace smoothing of the EMA counts


def codec_init(params, bits: int = 6, stages: int = 2, size: int = 8, iters: int = 5, seed: int = 0,
               param_mode: str = "pixel") -> dict:
    """Starting point of the codec fine-tuning (Sec. 3.3-3.4, the paper's b = 6,
    M = 2, B = 8, five K-means iterations), computed on the host once:
    gamma_i, beta_i span the fitted Cholesky components (beta = min,
    gamma = (max - min) / (2^b - 1)); each RVQ stage's codebook is K-means
    (Lloyd, FP64, centroids started at `size` distinct Gaussians drawn with
    `seed`, an empty cluster keeps its centroid) on the residual left by
    the stages before it. params [n,8] as the fit holds them."""
    import numpy as np
    p = params.detach().cpu().numpy().astype(np.float64).reshape(-1, 8)
    l = p[:, 2:5].copy()
    if param_mode == "paper":
        l[:, 0] += 0.5
        l[:, 2] += 0.5
    qp = 2 ** bits - 1
    lo, hi = l.min(axis=0), l.max(axis=0)
    gamma = np.where(hi > lo, (hi - lo) / qp, 1.0)
    r = p[:, 5:8].copy()
    gen = np.random.default_rng(seed)
    cbs = np.zeros((stages, size, 3))
    def nearest(x, c):  # index of the nearest centroid, in row blocks (bounded memory)
        return np.concatenate([np.argmin(((x[i:i + 8192, None, :] - c[None]) ** 2).sum(-1), axis=1)
                               for i in range(0, x.shape[0], 8192)]) if x.shape[0] else np.zeros(0, np.int64)

    for m in range(stages):
        cent = r[gen.permutation(r.shape[0])[:size]].copy()
        if cent.shape[0] < size:
            cent = np.concatenate([cent, np.zeros((size - cent.shape[0], 3))])
        for _ in range(iters):
            a = nearest(r, cent)
            for j in range(size):
                sel = a == j
                if sel.any():
                    cent[j] = r[sel].mean(axis=0)
        a = nearest(r, cent)
        r = r - cent[a]
        cbs[m] = cent
    return {"bits": bits, "codebooks": torch.from_numpy(cbs.astype(np.float32)).to(params.device),
            "gamma": gamma.astype(np.float32).tolist(), "beta": lo.astype(np.float32).tolist()}


class Fit:
    """Fitting context over one or more images (Sec. 3.4): each step is
    formation, binning, render + L2 loss, backward and Adam, replayed from a
    CUDA graph when ``use_graph``.

    targets: list of [H,W,3] float32 CUDA tensors; params: list of [n,8]
    float32 tensors (mx, my, l1, l2, l3, c'r, c'g, c'b) per image.

    Options (all validated by the library, which refuses combinations it
    does not support):
      lr            learning rates of (positions, covariance, colour)
      param_mode    "pixel" (parameters as above) or "paper" (App. C.1:
                    positions through tanh, +0.5 on the Cholesky diagonal
                    or on the scales)
      optimizer     "adam" (betas, eps) or "adan" (betas = three decays,
                    default ADAN_BETAS); lr_halve_every halves every rate
                    every that many steps (0 = never)
      cov           "cholesky" (l1, l2, l3) or "rs" (theta, s1, s2; Eq. 2-3)
      codec         codec_init(...) dict: quantisation-aware fine-tuning
                    (FP16 positions, b-bit Cholesky, RVQ colour; one image)
      opacity       "merged" (c', the paper's form), "separate" (colour and
                    a sigmoid opacity, accumulated summation) or "blend"
                    (sorted alpha-blending, tile 16); opacity_logits gives
                    the initial logits (default 0)
      render_split  lane groups per tile in the render (0 = chosen from the
                    first binning; see RENDER_SPLITS)
      tile_queue    render from a device queue of tiles ordered by
                    descending list length with persistent blocks (same
                    results as the default one block per tile)
      use_graph     replay each step from a captured CUDA graph
      stage_events  record CUDA events between the stages (stage_times)
    Methods: step, render, images, mse, stage_times, set_target_source,
    encode (codec), state_dict / load_state_dict, close."""

    def __init__(self, targets: Sequence[torch.Tensor], params: Sequence[torch.Tensor], tile: int = 16,
                 lr=(1e-3, 1e-2, 1e-2), betas=(0.9, 0.999), eps=1e-8, capacity: Optional[int] = None,
                 capacity_factor: float = 1.5, use_graph: bool = True, stage_events: bool = False,
                 render_split: int = 0, param_mode: str = "pixel", optimizer: str = "adam",
                 lr_halve_every: int = 0, cov: str = "cholesky", codec: Optional[dict] = None,
                 opacity: str = "merged", opacity_logits: Optional[Sequence[torch.Tensor]] = None,
                 tile_queue: bool = False):
        lib = L.load()
        assert len(targets) == len(params) and len(targets) >= 1
        self.shapes = [(int(t.shape[1]), int(t.shape[0])) for t in targets]
        self.counts = [int(p.shape[0]) for p in params]
        self.tile = tile
        dev = targets[0].device
        tgt = torch.cat([_dev(t, torch.float32, "target").reshape(-1) for t in targets])
        prm = torch.cat([_dev(p, torch.float32, "params").reshape(-1, 8) for p in params]).contiguous()
        if param_mode not in ("pixel", "paper") or optimizer not in ("adam", "adan") or cov not in ("cholesky", "rs"):
            raise ValueError("param_mode must be 'pixel' or 'paper', optimizer 'adam' or 'adan', cov 'cholesky' or 'rs'")
        self.param_mode, self.optimizer, self.cov = param_mode, optimizer, cov
        if optimizer == "adan" and len(betas) != 3:
            betas = ADAN_BETAS
        n_img = len(targets)
        self._w = (ctypes.c_int32 * n_img)(*[s[0] for s in self.shapes])
        self._h = (ctypes.c_int32 * n_img)(*[s[1] for s in self.shapes])
        self._n = (ctypes.c_int32 * n_img)(*self.counts)
        desc = L.GIFitDesc(n_img, ctypes.cast(self._w, ctypes.c_void_p), ctypes.cast(self._h, ctypes.c_void_p),
                           ctypes.cast(self._n, ctypes.c_void_p), tgt.data_ptr(), prm.data_ptr(), tile,
                           lr[0], lr[1], lr[2], betas[0], betas[1], eps, 1, int(use_graph),
                           int(stage_events), 0, int(param_mode == "paper"),
                           int(optimizer == "adan"), float(betas[2]) if optimizer == "adan" else 0.0,
                           int(lr_halve_every), int(cov == "rs"))
        if opacity not in OPACITY_MODES:
            raise ValueError(f"opacity must be one of {tuple(OPACITY_MODES)}")
        self.opacity_mode = opacity
        desc.opacity_mode = OPACITY_MODES[opacity]
        desc.tile_queue = int(bool(tile_queue))
        self.tile_queue = bool(tile_queue)
        if opacity != "merged" and opacity_logits is not None:
            lg = torch.cat([_dev(x, torch.float32, "opacity_logits").reshape(-1) for x in opacity_logits]).contiguous()
            assert lg.numel() == sum(self.counts)
            self._logits_init = lg
            desc.opacity_logits = lg.data_ptr()
        self.codec = None
        if codec is not None:
            cb = _dev(codec["codebooks"], torch.float32, "codebooks").contiguous()
            M, Bn = int(cb.shape[0]), int(cb.shape[1])
            desc.codec_bits, desc.codec_stages, desc.codec_size = int(codec.get("bits", 6)), M, Bn
            desc.codebooks = cb.data_ptr()
            desc.lsq_gamma[:] = [float(x) for x in codec["gamma"]]
            desc.lsq_beta[:] = [float(x) for x in codec["beta"]]
            desc.ema_decay = float(codec.get("ema_decay", CODEC_EMA_DECAY))
            desc.ema_eps = float(codec.get("ema_eps", CODEC_EMA_EPS))
            self.codec = {"bits": desc.codec_bits, "stages": M, "size": Bn, "ema_decay": desc.ema_decay,
                          "ema_eps": desc.ema_eps}
        K = None
        if capacity is None or (render_split == 0 and tile == 16):
            # pairs of the first step, counted by the library with this
            # context's own formation (parameterisation, covariance form, codec)
            K = ctypes.c_int64(0)
            L.check(lib.gi_fit_count_pairs(ctypes.byref(desc), L.stream_handle(), ctypes.byref(K)),
                    "gi_fit_count_pairs")
            K = K.value
        self.initial_pairs = K  # pairs of the first step, counted by the library (None when not needed)
        if capacity is None:
            capacity = max(4096, int(K * capacity_factor) + 1024)
        if render_split == 0 and tile == 16:
            # Short tile lists are rendered faster by fewer lane groups per tile
            # (measured on GB300: 97 pairs per tile, split 4 is 1.2x faster than
            # 8; 234 pairs per tile, split 8 is 1.06x faster than 4).
            n_tiles = sum(tiles(W, H, tile)[0] * tiles(W, H, tile)[1] for W, H in self.shapes)
            render_split = 8 if K >= 160 * n_tiles else 4
        self.render_split = int(render_split)
        self.capacity = int(capacity)
        desc.render_split = self.render_split
        desc.capacity = self.capacity
        h = ctypes.c_void_p()
        L.check(lib.gi_fit_create(ctypes.byref(desc), L.stream_handle(), ctypes.byref(h)), "gi_fit_create")
        self._h_fit = h
        self.device = dev
        N = sum(self.counts)
        npix = sum(W * H for W, H in self.shapes)
        self.params = self._view(L.FIT_PARAMS, (N, 8), "<f4")
        self.adam_m = self._view(L.FIT_ADAM_M, (N, 8), "<f4")
        self.adam_v = self._view(L.FIT_ADAM_V, (N, 8), "<f4")
        self.grads = self._view(L.FIT_GRADS, (N, 8), "<f4")
        self.out = self._view(L.FIT_OUT, (npix * 3,), "<f4")
        self.loss_sum = self._view(L.FIT_LOSS, (n_img,), "<f8")
        self.step_count = self._view(L.FIT_STEP, (1,), "<i4")
        self.k = self._view(L.FIT_K, (1,), "<i8")
        if optimizer == "adan":
            self.adan_n = self._view(L.FIT_ADAN_N, (N, 8), "<f4")
            self.adan_gprev = self._view(L.FIT_ADAN_GPREV, (N, 8), "<f4")
        self.targets = self._view(L.FIT_TARGET, (npix * 3,), "<f4")
        if self.codec is not None:
            M, Bn = self.codec["stages"], self.codec["size"]
            self.codec_gb = self._view(L.FIT_CODEC_GB, (5, 6), "<f4")  # gamma, beta; then m, v, n, g_prev
            self.codebooks = self._view(L.FIT_CODEBOOKS, (M, Bn, 3), "<f4")
            self.ema_count = self._view(L.FIT_EMA_COUNT, (M, Bn), "<f8")
            self.ema_total = self._view(L.FIT_EMA_TOTAL, (M, Bn, 3), "<f8")
            self.codes = self._view(L.FIT_CODES, (N, 4), "|u1")
            self.rvq_idx = self._view(L.FIT_RVQ_IDX, (M, N), "|u1")
            self.codec_out = self._view(L.FIT_CODEC_OUT, (7,), "<f8")
            self.means16 = self._view(L.FIT_MEANS16, (N, 2), "<i2")
        if self.opacity_mode != "merged":
            base = ctypes.c_void_p()
            L.check(L.load().gi_fit_pointer(self._h_fit, L.FIT_OPACITY, ctypes.byref(base)), "gi_fit_pointer")
            row = (N * 4 + 255) // 256 * 256
            rows = [torch.as_tensor(_DevArray(base.value + i * row, (N,), "<f4"), device=self.device) for i in range(7)]
            (self.opacity_logit, self.opacity, self.opacity_m, self.opacity_v, self.opacity_n, self.opacity_gprev,
             self.opacity_grad) = rows
            if self.opacity_mode == "blend":
                self.n_last = self._view(L.FIT_N_LAST, (npix,), "<i4")

    def _view(self, what, shape, typestr):
        p = ctypes.c_void_p()
        L.check(L.load().gi_fit_pointer(self._h_fit, what, ctypes.byref(p)), "gi_fit_pointer")
        return torch.as_tensor(_DevArray(p.value, shape, typestr), device=self.device)

    def step(self, n: int = 1):
        L.check(L.load().gi_fit_step(self._h_fit, int(n), L.stream_handle()), "gi_fit_step")

    def binning(self) -> dict:
        """The binning of the last step (or render), as the library holds it:
        keys and ids [K] (global tile and Gaussian ids, sorted by tile,
        ascending Gaussian id inside a tile), ranges [tiles, 2], pair_off
        [N + 1], rect [N, 4] and cnt [N] (device views; synchronises)."""
        N = sum(self.counts)
        n_tiles = sum(tiles(W, H, self.tile)[0] * tiles(W, H, self.tile)[1] for W, H in self.shapes)
        K = int(self.k.item())
        return {"K": K, "keys": self._view(L.FIT_KEYS, (self.capacity,), "<i4")[:K],
                "ids": self._view(L.FIT_IDS, (self.capacity,), "<i4")[:K],
                "ranges": self._view(L.FIT_RANGES, (n_tiles, 2), "<i4"),
                "pair_off": self._view(L.FIT_PAIR_OFF, (N + 1,), "<i8"),
                "rect": self._view(L.FIT_RECT, (N, 4), "<i4"), "cnt": self._view(L.FIT_CNT, (N,), "<i4")}

    def stage_times(self):
        """Device ms of the last step's stages: formation, binning, render,
        backward, update (needs stage_events=True)."""
        ms = (ctypes.c_float * 5)()
        L.check(L.load().gi_fit_stage_times(self._h_fit, ms), "gi_fit_stage_times")
        return list(ms)

    def render(self):
        L.check(L.load().gi_fit_render(self._h_fit, L.stream_handle()), "gi_fit_render")

    def encode(self) -> dict:
        """The codec stream of the current parameters (Sec. 3.3; a codec
        fine-tuning context only): renders once so that the codes and indices
        match the current parameters, gamma, beta and codebooks, and returns
        means16 (the pixel-space positions in FP16, as int16 bits), codes
        [N,4] uint8, gamma_beta, idx [M,N] uint8, codebooks [M,B,3] and the
        stream size in bits (positions 16 bits each, b bits per code,
        log2 B per index, gamma, beta and codebooks as FP32)."""
        import math
        if self.codec is None:
            raise ValueError("encode needs a codec fine-tuning context")
        self.render()
        M, Bn, b = self.codec["stages"], self.codec["size"], self.codec["bits"]
        N = sum(self.counts)
        bits = N * (2 * 16 + 3 * b + M * max(1, math.ceil(math.log2(Bn)))) + 6 * 32 + M * Bn * 3 * 32
        torch.cuda.current_stream().synchronize()
        return {"means16": self.means16.clone(), "codes": self.codes.clone(),
                "gamma_beta": self.codec_gb[0].cpu().tolist(), "idx": self.rvq_idx.clone(),
                "codebooks": self.codebooks.clone(), "bits": bits}

    def set_target_source(self, src: Optional[torch.Tensor] = None):
        """Train against `src` instead of the context's target copy: a CUDA
        tensor, or a pinned CPU tensor that every step's render reads over
        the host link (overlapped with its work, no separate copy); same
        layout as the concatenated targets (float32, HWC). None restores the
        context's own copy. `src` must stay alive while steps read it."""
        ptr = None
        if src is not None:
            if src.dtype != torch.float32 or not src.is_contiguous() or src.numel() != self.targets.numel():
                raise ValueError("target source must be a contiguous float32 tensor of the targets' size")
            if src.device.type == "cpu" and not src.is_pinned():
                raise ValueError("a CPU target source must be pinned")
            ptr = src.data_ptr()
        self._target_src = src
        L.check(L.load().gi_fit_set_target_source(self._h_fit, ptr, L.stream_handle()), "gi_fit_set_target_source")

    def images(self) -> List[torch.Tensor]:
        outs, o = [], 0
        for W, H in self.shapes:
            outs.append(self.out[o:o + W * H * 3].view(H, W, 3))
            o += W * H * 3
        return outs

    def mse(self) -> List[float]:
        """Per-image mean squared error of the last step's render."""
        s = self.loss_sum.cpu().tolist()
        return [v / (3.0 * W * H) for v, (W, H) in zip(s, self.shapes)]

    def state_dict(self) -> dict:
        """Checkpoint of the fit: parameters, Adam moments and the completed
        step count (copies on the context's device). The pipeline has no
        random state; everything else is recomputed every step."""
        torch.cuda.current_stream().synchronize()
        sd = {"params": self.params.clone(), "adam_m": self.adam_m.clone(), "adam_v": self.adam_v.clone(),
              "step": int(self.step_count.item()), "shapes": list(self.shapes), "counts": list(self.counts),
              "tile": self.tile, "param_mode": self.param_mode, "optimizer": self.optimizer, "cov": self.cov}
        if self.optimizer == "adan":
            sd["adan_n"] = self.adan_n.clone()
            sd["adan_gprev"] = self.adan_gprev.clone()
        sd["opacity"] = self.opacity_mode
        if self.opacity_mode != "merged":
            for k in ("opacity_logit", "opacity_m", "opacity_v", "opacity_n", "opacity_gprev"):
                sd[k] = getattr(self, k).clone()
        if self.codec is not None:
            sd["codec"] = dict(self.codec)
            for k in ("codec_gb", "codebooks", "ema_count", "ema_total"):
                sd[k] = getattr(self, k).clone()
        return sd

    def load_state_dict(self, sd: dict):
        """Restores a checkpoint of a fit with the same images, Gaussian
        counts and tile edge; the next steps continue bit-identically."""
        if list(sd["shapes"]) != list(self.shapes) or list(sd["counts"]) != list(self.counts) or \
                sd["tile"] != self.tile or sd.get("param_mode", "pixel") != self.param_mode or \
                sd.get("optimizer", "adam") != self.optimizer or sd.get("cov", "cholesky") != self.cov or \
                sd.get("codec") != self.codec or sd.get("opacity", "merged") != self.opacity_mode:
            raise ValueError("checkpoint of a different fit (images, Gaussian counts, tile edge, "
                             "parameterisation or optimiser)")
        self.params.copy_(sd["params"])
        self.adam_m.copy_(sd["adam_m"])
        self.adam_v.copy_(sd["adam_v"])
        if self.optimizer == "adan":
            self.adan_n.copy_(sd["adan_n"])
            self.adan_gprev.copy_(sd["adan_gprev"])
        if self.codec is not None:
            for k in ("codec_gb", "codebooks", "ema_count", "ema_total"):
                getattr(self, k).copy_(sd[k])
        if self.opacity_mode != "merged":
            for k in ("opacity_logit", "opacity_m", "opacity_v", "opacity_n", "opacity_gprev"):
                getattr(self, k).copy_(sd[k])
        self.step_count.fill_(int(sd["step"]))

    def close(self):
        if getattr(self, "_h_fit", None) is not None:
            L.load().gi_fit_destroy(self._h_fit)
            self._h_fit = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Renderer:
    """Forward-only pipeline with preallocated buffers for a fixed image size
    and Gaussian count: formation, binning and render (Eq. 7), enqueued on
    the current stream without host synchronisation. `capacity` bounds the
    pair count; overflow is reported by device_errors()."""

    def __init__(self, W: int, H: int, n: int, tile: int = 16, capacity: int = 1 << 20, device="cuda"):
        lib = L.load()
        self.W, self.H, self.n, self.tile, self.capacity = W, H, n, tile, int(capacity)
        tw, th = tiles(W, H, tile)
        f32, i32 = torch.float32, torch.int32
        self.rec = torch.empty((n, 8), dtype=f32, device=device)
        self.rect = torch.empty((n, 4), dtype=i32, device=device)
        self.cnt = torch.empty((n,), dtype=i32, device=device)
        nb = ctypes.c_size_t(0)
        L.check(lib.gi_bin_workspace_size(n, _img(W, H, tile), self.capacity, ctypes.byref(nb)), "gi_bin_workspace_size")
        self.ws_bytes = nb.value
        self.ws = torch.empty((nb.value,), dtype=torch.uint8, device=device)
        self.keys = torch.empty((self.capacity,), dtype=i32, device=device)
        self.ids = torch.empty((self.capacity,), dtype=i32, device=device)
        self.ranges = torch.empty((tw * th, 2), dtype=i32, device=device)
        self.rec_binned = torch.empty((self.capacity, 8), dtype=f32, device=device)
        self.pair_off = torch.empty((n + 1,), dtype=torch.int64, device=device)
        self.k_dev = torch.empty((1,), dtype=torch.int64, device=device)
        self.out = torch.empty((H, W, 3), dtype=f32, device=device)

    def __call__(self, means, chol, color):
        lib = L.load()
        img = _img(self.W, self.H, self.tile)
        s = L.stream_handle()
        L.check(lib.gi_project(L.ptr(means), L.ptr(chol), L.ptr(color), self.n, img, L.ptr(self.rec),
                               L.ptr(self.rect), L.ptr(self.cnt), s), "gi_project")
        L.check(lib.gi_bin_tiles(L.ptr(self.rect), L.ptr(self.cnt), L.ptr(self.rec), self.n, img, self.capacity,
                                 L.ptr(self.ws), self.ws_bytes, L.ptr(self.keys), L.ptr(self.ids), L.ptr(self.ranges),
                                 L.ptr(self.rec_binned), L.ptr(self.pair_off), L.ptr(self.k_dev), s), "gi_bin_tiles")
        L.check(lib.gi_render(L.ptr(self.rec_binned), L.ptr(self.ranges), img, None, L.ptr(self.out), None, None, s),
                "gi_render")
        return self.out


def autotune(targets, params, tiles=(8, 16, 32), splits=None, steps=10, warmup=3, lr=(1e-3, 1e-2, 1e-2)):
    """Chooses the tile edge and the render's warps-per-tile split for a fit
    of these images by timing `steps` graph-replayed fit steps of every
    candidate (CUDA events on the current stream) after `warmup` steps.
    Every candidate runs on fresh copies of the parameters, which are left
    untouched. Returns {"tile", "render_split", "ms_per_step": {(T, split): ms}}."""
    stream = torch.cuda.current_stream()
    times = {}
    for T in tiles:
        for sp in (splits or {}).get(T, RENDER_SPLITS[T]):
            f = Fit(targets, [p.clone() for p in params], tile=T, lr=lr, render_split=sp)
            f.step(warmup)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f.step(steps)
            e1.record(stream)
            e1.synchronize()
            times[(T, sp)] = e0.elapsed_time(e1) / steps
            f.close()
    best = min(times, key=times.get)
    return {"tile": best[0], "render_split": best[1], "ms_per_step": times}


def selftest_bounded_waits(limit_ns: int = 2_000_000) -> int:
    """Runs the bounded-wait self-test (gi_selftest_bounded_waits) and
    returns its status bits: 3 = both waits gave up after limit_ns."""
    bits = ctypes.c_uint32(0)
    L.check(L.load().gi_selftest_bounded_waits(ctypes.byref(bits), int(limit_ns), L.stream_handle()),
            "gi_selftest_bounded_waits")
    return int(bits.value)


def alu_peaks():
    r = (ctypes.c_double * 6)()
    L.check(L.load().gi_alu_peaks(r, L.stream_handle()), "gi_alu_peaks")
    return {"ffma_lane_ops_s": r[0], "ffma2_lane_ops_s": r[1], "ex2_s": r[2], "mix_elems_s": r[3],
            "sm_mhz": r[4], "sms": int(r[5])}
