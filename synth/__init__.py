"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the CUDA path's tests/bench and by the CPU oracle's
tests. It holds none of the method's arithmetic: it only draws images,
initial Gaussian parameters, codebooks and upstream gradients from seeded
numpy PCG64 generators.

The paper evaluates on Kodak (24 images, 768x512) and DIV2K (x2 down-scaled,
sides 408-1020 px) (Sec. 4.1). Neither dataset is available here, so these
synthetic images stand in for them. Recipe (all constants fixed here):

* base level 0.3 on all channels;
* ``n_blobs`` anisotropic Gaussian blobs: centre uniform over the image,
  major std log-uniform in [2, min(W,H)/8] px, aspect uniform [1,4], angle
  uniform, per-channel amplitude uniform [-0.3, 0.5], truncated at 3.5 major
  std;
* 3 sinusoids: per-channel amplitude 0.1, at most 3 cycles per image width,
  random direction and phase;
* ``n_lines`` line segments: length uniform [10, 200] px, Gaussian cross
  profile with std 1 px, per-channel amplitude uniform [-0.3, 0.3];
* clamp to [0, 1], float32, HWC layout.

Gaussian initialisation (pixel-space parameters, the boundary's convention):
mean uniform over [0,W)x[0,H); Cholesky diagonal l1, l3 log-uniform in
[1, 8] px; off-diagonal l2 uniform in [-2, 2]; weighted colour c' uniform in
[0, 0.2] per channel.

Seeds follow ``seed = 1000 * config + image_index``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "rng",
    "image",
    "init_gaussians",
    "skewed_means",
    "workload",
    "batch_workload",
    "batch_sizes",
    "batch_gaussian_count",
    "codebooks",
    "Workload",
    "CONFIGS",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _add_blobs(img: np.ndarray, g: np.random.Generator, n_blobs: int) -> None:
    H, W, _ = img.shape
    smax = max(2.0, min(W, H) / 8.0)
    for _ in range(n_blobs):
        cx = g.uniform(0, W)
        cy = g.uniform(0, H)
        s_major = math.exp(g.uniform(math.log(2.0), math.log(smax)))
        aspect = g.uniform(1.0, 4.0)
        s_minor = s_major / aspect
        ang = g.uniform(0, math.pi)
        amp = g.uniform(-0.3, 0.5, size=3).astype(np.float32)
        r = 3.5 * s_major
        x0, x1 = max(0, int(cx - r)), min(W, int(cx + r) + 1)
        y0, y1 = max(0, int(cy - r)), min(H, int(cy + r) + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        xs = np.arange(x0, x1, dtype=np.float32) + 0.5 - cx
        ys = np.arange(y0, y1, dtype=np.float32) + 0.5 - cy
        X, Y = np.meshgrid(xs, ys)
        ca, sa = math.cos(ang), math.sin(ang)
        u = ca * X + sa * Y
        v = -sa * X + ca * Y
        w = np.exp(-0.5 * ((u / s_major) ** 2 + (v / s_minor) ** 2)).astype(np.float32)
        img[y0:y1, x0:x1, :] += w[:, :, None] * amp[None, None, :]


def _add_sinusoids(img: np.ndarray, g: np.random.Generator) -> None:
    H, W, _ = img.shape
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float32)
    for _ in range(3):
        f = g.uniform(0.2, 3.0) / W  # cycles per pixel, at most 3 per width
        th = g.uniform(0, 2 * math.pi)
        ph = g.uniform(0, 2 * math.pi, size=3)
        arg = 2 * math.pi * f * (math.cos(th) * xs + math.sin(th) * ys)
        for c in range(3):
            img[:, :, c] += (0.1 * np.sin(arg + ph[c])).astype(np.float32)


def _add_lines(img: np.ndarray, g: np.random.Generator, n_lines: int) -> None:
    H, W, _ = img.shape
    for _ in range(n_lines):
        x0, y0 = g.uniform(0, W), g.uniform(0, H)
        length = g.uniform(10, 200)
        ang = g.uniform(0, 2 * math.pi)
        x1, y1 = x0 + length * math.cos(ang), y0 + length * math.sin(ang)
        amp = g.uniform(-0.3, 0.3, size=3).astype(np.float32)
        m = 4.0
        bx0 = max(0, int(min(x0, x1) - m))
        bx1 = min(W, int(max(x0, x1) + m) + 1)
        by0 = max(0, int(min(y0, y1) - m))
        by1 = min(H, int(max(y0, y1) + m) + 1)
        if bx0 >= bx1 or by0 >= by1:
            continue
        X, Y = np.meshgrid(np.arange(bx0, bx1, dtype=np.float32) + 0.5,
                           np.arange(by0, by1, dtype=np.float32) + 0.5)
        dx, dy = x1 - x0, y1 - y0
        tpar = np.clip(((X - x0) * dx + (Y - y0) * dy) / (dx * dx + dy * dy), 0.0, 1.0)
        d2 = (X - (x0 + tpar * dx)) ** 2 + (Y - (y0 + tpar * dy)) ** 2
        w = np.exp(-0.5 * d2).astype(np.float32)
        img[by0:by1, bx0:bx1, :] += w[:, :, None] * amp[None, None, :]


def image(W: int, H: int, seed: int, n_blobs: int = 40, n_lines: int = 0) -> np.ndarray:
    """Synthetic RGB target image, float32 HWC in [0, 1]."""
    g = rng(seed)
    img = np.full((H, W, 3), 0.3, dtype=np.float32)
    _add_blobs(img, g, n_blobs)
    _add_sinusoids(img, g)
    if n_lines:
        _add_lines(img, g, n_lines)
    np.clip(img, 0.0, 1.0, out=img)
    return np.ascontiguousarray(img, dtype=np.float32)


def init_gaussians(n: int, W: int, H: int, seed: int):
    """Initial pixel-space parameters: means [n,2], chol [n,3] (l1,l2,l3), color [n,3]."""
    g = rng(seed + 500)
    means = np.empty((n, 2), np.float32)
    means[:, 0] = g.uniform(0, W, size=n)
    means[:, 1] = g.uniform(0, H, size=n)
    chol = np.empty((n, 3), np.float32)
    chol[:, 0] = np.exp(g.uniform(0.0, math.log(8.0), size=n))
    chol[:, 1] = g.uniform(-2.0, 2.0, size=n)
    chol[:, 2] = np.exp(g.uniform(0.0, math.log(8.0), size=n))
    color = g.uniform(0.0, 0.2, size=(n, 3)).astype(np.float32)
    # uniform(0, W) can round up to W in float32; keep means inside [0, W).
    np.minimum(means[:, 0], np.nextafter(np.float32(W), np.float32(0)), out=means[:, 0])
    np.minimum(means[:, 1], np.nextafter(np.float32(H), np.float32(0)), out=means[:, 1])
    return means, chol, color


def init_gaussians_rs(n: int, W: int, H: int, seed: int):
    """Initial pixel-space parameters in the rotation-scaling form: means
    [n,2], rs [n,3] (theta uniform in [-pi, pi), scales s1, s2 log-uniform
    in [1, 8] like the Cholesky diagonal of init_gaussians), color [n,3]."""
    means, _, color = init_gaussians(n, W, H, seed)
    g = rng(seed + 700)
    rs = np.empty((n, 3), np.float32)
    rs[:, 0] = g.uniform(-math.pi, math.pi, size=n)
    rs[:, 1] = np.exp(g.uniform(0.0, math.log(8.0), size=n))
    rs[:, 2] = np.exp(g.uniform(0.0, math.log(8.0), size=n))
    return means, rs, color


def skewed_means(means: np.ndarray, W: int, H: int, seed: int, frac: float = 0.3,
                 area: float = 0.1) -> np.ndarray:
    """Move ``frac`` of the means uniformly into a seeded axis-aligned rectangle
    covering ``area`` of the image (sqrt(area)*W x sqrt(area)*H)."""
    g = rng(seed + 900)
    m = means.copy()
    n = m.shape[0]
    k = int(round(frac * n))
    rw, rh = math.sqrt(area) * W, math.sqrt(area) * H
    x0 = g.uniform(0, W - rw)
    y0 = g.uniform(0, H - rh)
    sel = g.permutation(n)[:k]
    m[sel, 0] = (x0 + g.uniform(0, rw, size=k)).astype(np.float32)
    m[sel, 1] = (y0 + g.uniform(0, rh, size=k)).astype(np.float32)
    return m


def upstream_grad(W: int, H: int, seed: int, scale: float = 1e-3) -> np.ndarray:
    """A seeded upstream gradient dL/dC [H,W,3] (for backward-only tests)."""
    g = rng(seed + 700)
    return (g.standard_normal((H, W, 3)) * scale).astype(np.float32)


@dataclass
class Workload:
    W: int
    H: int
    n: int
    target: np.ndarray
    means: np.ndarray
    chol: np.ndarray
    color: np.ndarray
    name: str = ""


# Named single-image workloads (sizes from the paper's settings: Kodak-sized
# 768x512 and DIV2K-sized 2040x1356 images).
CONFIGS = {
    # 256x256, 2,000 Gaussians, 40 blobs: the small parity case.
    "c0_256x256_2k": dict(W=256, H=256, n=2000, blobs=40, lines=0, config=0, skew=False),
    # 768x512 (Kodak shape), 70,000 Gaussians (560K params), 400 blobs + 200 lines.
    "c1_768x512_70k": dict(W=768, H=512, n=70000, blobs=400, lines=200, config=1, skew=False),
    # 2040x1356 (DIV2K full-res shape), 100k / 200k Gaussians, skewed means.
    "c2_2040x1356_100k": dict(W=2040, H=1356, n=100000, blobs=1500, lines=0, config=2, skew=True),
    "c2_2040x1356_200k": dict(W=2040, H=1356, n=200000, blobs=1500, lines=0, config=2, skew=True),
    # Codec decode path: 768x512, 50,000 Gaussians.
    "c4_768x512_50k": dict(W=768, H=512, n=50000, blobs=400, lines=200, config=4, skew=False),
}


def workload(name: str, index: int = 0) -> Workload:
    c = CONFIGS[name]
    seed = 1000 * c["config"] + index
    W, H, n = c["W"], c["H"], c["n"]
    tgt = image(W, H, seed, n_blobs=c["blobs"], n_lines=c["lines"])
    means, chol, color = init_gaussians(n, W, H, seed)
    if c["skew"]:
        means = skewed_means(means, W, H, seed)
    return Workload(W, H, n, tgt, means, chol, color, name)


BATCH_SHAPES = [(256, 256), (512, 384), (768, 512), (1024, 768)]


def batch_gaussian_count(W: int, H: int) -> int:
    """Gaussians proportional to pixel count: 70,000 at 1024x768, at least 5,000."""
    return max(5000, int(round(70000 * W * H / 786432)))


def batch_sizes(n_images: int, seed: int = 3000):
    g = rng(seed)
    idx = g.integers(0, len(BATCH_SHAPES), size=n_images)
    return [BATCH_SHAPES[i] for i in idx]


def batch_workload(n_images: int = 64, config: int = 3):
    """Uneven batch: sizes uniform over BATCH_SHAPES, blobs/lines scaled by area."""
    out = []
    for i, (W, H) in enumerate(batch_sizes(n_images, seed=1000 * config)):
        seed = 1000 * config + i
        area = W * H / (768 * 512)
        tgt = image(W, H, seed, n_blobs=max(20, int(round(400 * area))),
                    n_lines=int(round(200 * area)))
        n = batch_gaussian_count(W, H)
        means, chol, color = init_gaussians(n, W, H, seed)
        out.append(Workload(W, H, n, tgt, means, chol, color, f"batch{i}_{W}x{H}"))
    return out


def codebooks(seed: int, size: int = 256, stages: int = 2):
    """Seeded RVQ codebooks [2 attr][stages][size][3] float32.

    attr 0 = Cholesky (l1, l2, l3), attr 1 = weighted colour. Stage 0 is
    uniform over the initialisation ranges; later stages are uniform within
    +-10% of the stage-0 range."""
    g = rng(seed + 800)
    lo = np.array([[1.0, -2.0, 1.0], [0.0, 0.0, 0.0]], np.float64)
    hi = np.array([[8.0, 2.0, 8.0], [0.2, 0.2, 0.2]], np.float64)
    cb = np.empty((2, stages, size, 3), np.float32)
    for a in range(2):
        cb[a, 0] = g.uniform(lo[a], hi[a], size=(size, 3))
        for s in range(1, stages):
            r = 0.1 * (hi[a] - lo[a])
            cb[a, s] = g.uniform(-r, r, size=(size, 3))
    return cb


def vq_indices(n: int, seed: int, size: int = 256, stages: int = 2) -> np.ndarray:
    """Seeded uniform uint8 indices [2 attr][stages][n] (bench input)."""
    g = rng(seed + 850)
    return g.integers(0, size, size=(2, stages, n), dtype=np.uint8)
