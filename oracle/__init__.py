"""FP64 CPU oracle for the GaussianImage accumulated-summation rasterizer.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``. The product path (the
``paper_2403_08551_gb300`` package and its CUDA library) never imports, links
or runs anything here, and nothing here imports the product.

The heavy loops (support rule, binning, render, backward) are plain C in
``gi_oracle.c`` (FP64 arithmetic, FP32 only for the support rule); the
per-Gaussian steps with no loops worth compiling (Adam, vector-quantisation
decode/encode, PSNR) are numpy in FP64 here. Every function cites the passage
of the paper it follows.

Parity status per function (pins live in ``tests/test_oracle_*.py``):
  rect_rule ... pinned (3-sigma ellipse extents, brute-force tile test)
  bin ......... pinned (numpy brute force per tile)
  render ...... pinned (isotropic closed form, linearity, permutation,
                union additivity, brute force bit-exact)
  backward .... pinned (central finite differences, isotropic closed form)
  adam ........ pinned (closed-form first step, torch.optim.Adam)
  paper_formation / paper_forward_backward ... pinned (finite differences
                in theta and the raw Cholesky vector; inverse of atanh init)
  rs_to_chol / rs_chain / rs_forward_backward ... pinned (Sigma rebuilt from
                R S against L L^T; finite differences in theta, s1, s2)
  adan ........ pinned (closed-form first step, constant-gradient steps,
                reduction to Adam's direction when b2 = 0)
  vq_decode ... pinned (IEEE float32 addition, zero residual codebook)
  rvq_encode .. pinned (exhaustive per-stage argmin)
  sigmoid_opacity / opacity_forward_backward / blend_render /
  blend_backward / blend_forward_backward ... pinned (per-pixel brute force
                over all Gaussians; closed forms of one and two Gaussians;
                the accumulated sum as the small-opacity limit; central
                finite differences in every parameter, opacity included)
  fp16_round / lsq_fake_quant / lsq_ste_grads / rvq_assign_f32 /
  commitment_loss / ema_codebook_update / codec_forward_backward ... pinned
                (struct half packing; brute-force nearest grid point;
                finite differences of the straight-through surrogate;
                brute-force nearest entry; zero-residual closed form;
                cluster means at decay 0; identity quantisers)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gi_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

LOG2E = 1.4426950408889634


def build(force: bool = False) -> str:
    """Compile gi_oracle.c with gcc (OpenMP when available)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", _SRC, "-lm"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-o", tmp],
                       capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base + ["-o", tmp], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int32
            lib.gio_rect_rule.argtypes = [P, P, P, i64, i32, i32, i32, P, P]
            lib.gio_rect_rule.restype = None
            lib.gio_bin.argtypes = [P, P, i64, i32, i32, i64, P, P, P]
            lib.gio_bin.restype = i64
            lib.gio_conic.argtypes = [P, i64, P]
            lib.gio_conic.restype = None
            lib.gio_render.argtypes = [P, P, P, P, P, i32, i32, i32, P]
            lib.gio_render.restype = None
            lib.gio_render_brute.argtypes = [P, P, P, P, P, i64, i32, i32, i32, i32, P]
            lib.gio_render_brute.restype = None
            lib.gio_loss.argtypes = [P, P, i32, i32, P]
            lib.gio_loss.restype = ctypes.c_double
            lib.gio_backward.argtypes = [P, P, P, P, P, i64, i32, i32, i32, P, P, P, P, P, P]
            lib.gio_backward.restype = None
            d = ctypes.c_double
            lib.gio_render_blend.argtypes = [P, P, P, P, P, P, i32, i32, i32, d, d, d, d, P, P, P, P]
            lib.gio_render_blend.restype = None
            lib.gio_backward_blend.argtypes = [P, P, P, P, P, P, i64, i32, i32, i32, d, d] + [P] * 10
            lib.gio_backward_blend.restype = None
            lib.gio_num_threads.restype = ctypes.c_int
            lib.gio_set_num_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def num_threads() -> int:
    return _load().gio_num_threads()


def set_num_threads(n: int) -> None:
    _load().gio_set_num_threads(int(n))


def tiles(W: int, H: int, T: int):
    return (W + T - 1) // T, (H + T - 1) // T


def rect_rule(means, chol, color, W, H, T):
    """Tile rectangles [n,4] (tx0, ty0, tx1, ty1) and counts [n] by the FP32
    3-sigma support rule (reading of Sec. 3.2; see gi_oracle.c)."""
    means, chol, color = _f32(means), _f32(chol), _f32(color)
    n = means.shape[0]
    rect = np.zeros((n, 4), np.int32)
    cnt = np.zeros(n, np.int32)
    _load().gio_rect_rule(_p(means), _p(chol), _p(color), n, W, H, T, _p(rect), _p(cnt))
    return rect, cnt


def bin_tiles(rect, cnt, W, H, T):
    """Per-tile Gaussian lists by definition (ascending g within a tile).
    Returns ids [K] uint32, ranges [T_img,2] int32, pair_off [n+1] int64."""
    rect = np.ascontiguousarray(rect, np.int32)
    cnt = np.ascontiguousarray(cnt, np.int32)
    n = cnt.shape[0]
    tw, th = tiles(W, H, T)
    K = int(cnt.astype(np.int64).sum())
    ids = np.zeros(max(K, 1), np.uint32)
    ranges = np.zeros((tw * th, 2), np.int32)
    pair_off = np.zeros(n + 1, np.int64)
    k = _load().gio_bin(_p(rect), _p(cnt), n, tw, th, ids.shape[0], _p(ids), _p(ranges), _p(pair_off))
    assert k == K
    return ids[:K], ranges, pair_off


def conic(chol):
    """Sigma^-1 = [[A, B], [B, C]] of Sigma = L L^T (Eq. 1), FP64 [n,3]."""
    chol = _f32(chol)
    q = np.zeros((chol.shape[0], 3), np.float64)
    _load().gio_conic(_p(chol), chol.shape[0], _p(q))
    return q


def render(means, chol, color, ids, ranges, W, H, T):
    """Binned accumulated-summation render (Eq. 7), FP64 [H,W,3]."""
    means, chol, color = _f32(means), _f32(chol), _f32(color)
    ids = np.ascontiguousarray(ids, np.uint32)
    if ids.size == 0:
        ids = np.zeros(1, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.int32)
    out = np.zeros((H, W, 3), np.float64)
    _load().gio_render(_p(means), _p(chol), _p(color), _p(ids), _p(ranges), W, H, T, _p(out))
    return out


def render_brute(means, chol, color, rect, cnt, W, H, T, use_support=True):
    """Every Gaussian at every pixel (Eq. 7); with ``use_support`` the same
    tile-granular support as the binned form, else untruncated."""
    means, chol, color = _f32(means), _f32(chol), _f32(color)
    rect = np.ascontiguousarray(rect, np.int32)
    cnt = np.ascontiguousarray(cnt, np.int32)
    out = np.zeros((H, W, 3), np.float64)
    _load().gio_render_brute(_p(means), _p(chol), _p(color), _p(rect), _p(cnt),
                             means.shape[0], W, H, T, int(bool(use_support)), _p(out))
    return out


def loss(out, target):
    """L2 loss read as the mean over 3HW (Sec. 3.4); returns (L, dL/dC)."""
    out = np.ascontiguousarray(out, np.float64)
    target = _f32(target)
    H, W, _ = out.shape
    d = np.zeros_like(out)
    L = _load().gio_loss(_p(out), _p(target), W, H, _p(d))
    return L, d


def backward(means, chol, color, rect, cnt, W, H, T, dldc):
    """Analytic gradients (App. A.1, A.2 with the errata noted in
    gi_oracle.c). Returns dict of FP64 arrays: means [n,2], chol [n,3],
    color [n,3], conic [n,3], and "abs": per parameter the sum over pixels of
    |that pixel's contribution| (the condition magnitude of the sum)."""
    means, chol, color = _f32(means), _f32(chol), _f32(color)
    rect = np.ascontiguousarray(rect, np.int32)
    cnt = np.ascontiguousarray(cnt, np.int32)
    dldc = np.ascontiguousarray(dldc, np.float64)
    n = means.shape[0]
    gm = np.zeros((n, 2)); gl = np.zeros((n, 3)); gc = np.zeros((n, 3)); gq = np.zeros((n, 3))
    ga = np.zeros((n, 8))
    _load().gio_backward(_p(means), _p(chol), _p(color), _p(rect), _p(cnt), n, W, H, T,
                         _p(dldc), _p(gm), _p(gl), _p(gc), _p(gq), _p(ga))
    return {"means": gm, "chol": gl, "color": gc, "conic": gq,
            "abs": {"means": ga[:, 0:2], "chol": ga[:, 2:5], "color": ga[:, 5:8]}}


def forward_backward(means, chol, color, target, T):
    """One full pass: support rule, binning, render, L2 loss, gradients."""
    H, W, _ = target.shape
    rect, cnt = rect_rule(means, chol, color, W, H, T)
    ids, ranges, pair_off = bin_tiles(rect, cnt, W, H, T)
    out = render(means, chol, color, ids, ranges, W, H, T)
    L, d = loss(out, target)
    grads = backward(means, chol, color, rect, cnt, W, H, T, d)
    return dict(rect=rect, cnt=cnt, ids=ids, ranges=ranges, pair_off=pair_off,
                out=out, loss=L, dldc=d, grads=grads)


ADAM_BETAS = (0.9, 0.999)
ADAM_EPS = 1e-8


def adam(param, grad, m, v, step, lr, betas=ADAM_BETAS, eps=ADAM_EPS):
    """One Adam step (Kingma & Ba, bias-corrected), FP64. ``step`` is the
    1-based step count after this update. Returns (param, m, v)."""
    b1, b2 = betas
    p = np.asarray(param, np.float64)
    g = np.asarray(grad, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** step)
    vhat = v / (1.0 - b2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ---------------------------------------------------------------------------
# The paper's own parameterisation and optimiser (App. C.1, Sec. 4.1).
# ---------------------------------------------------------------------------

def paper_formation(theta, chol_raw, W, H):
    """Raw parameters -> pixel-space ones (App. C.1): positions pass through
    tanh into (-1, 1), read as mu = (tanh(theta) + 1) / 2 * (W, H); the
    Cholesky diagonal gets +0.5 (l1' = l1 + 0.5, l3' = l3 + 0.5). Returns
    FP32 means and Cholesky vectors (tanh in FP64, each result rounded once)
    and the FP64 Jacobian d mu / d theta = (1 - tanh^2) / 2 * (W, H)."""
    th = np.asarray(theta, np.float64)
    t = np.tanh(th)
    scale = np.array([W, H], np.float64)
    means = ((t + 1.0) * 0.5 * scale).astype(np.float32)
    c = np.asarray(chol_raw, np.float32).copy()
    c[:, 0] = c[:, 0] + np.float32(0.5)
    c[:, 2] = c[:, 2] + np.float32(0.5)
    dmu = (1.0 - t) * (1.0 + t) * 0.5 * scale
    return means, c, dmu


def paper_forward_backward(theta, chol_raw, color, target, T):
    """forward_backward on the raw parameters of App. C.1: gradients with
    respect to theta (chained through tanh) and to the raw Cholesky vector
    (the +0.5 shift has unit derivative)."""
    H, W, _ = target.shape
    means, chol, dmu = paper_formation(theta, chol_raw, W, H)
    r = forward_backward(means, chol, color, target, T)
    g = r["grads"]
    r["grads_raw"] = {"theta": g["means"] * dmu, "chol": g["chol"], "color": g["color"],
                      "abs_theta": g["abs"]["means"] * np.abs(dmu)}
    return r


def rs_to_chol(rs):
    """Rotation-scaling form (Sec. 3.1, Eq. 2-3): Sigma = (R S)(R S)^T with R
    the rotation by theta and S = diag(s1, s2); returns the lower-triangular
    Cholesky vector of the same Sigma (FP64, each entry rounded once to FP32):
      Sigma11 = c^2 s1^2 + s^2 s2^2, Sigma12 = c s (s1^2 - s2^2),
      Sigma22 = s^2 s1^2 + c^2 s2^2,
      l1 = sqrt(Sigma11), l2 = Sigma12 / l1, l3 = |s1 s2| / l1
    (det Sigma = (s1 s2)^2 = (l1 l3)^2)."""
    rs = np.asarray(rs, np.float64)
    th, s1, s2 = rs[:, 0], rs[:, 1], rs[:, 2]
    c, s = np.cos(th), np.sin(th)
    S11 = c * c * s1 * s1 + s * s * s2 * s2
    S12 = c * s * (s1 * s1 - s2 * s2)
    with np.errstate(divide="ignore", invalid="ignore"):
        l1 = np.sqrt(S11)
        l2 = S12 / l1
        l3 = np.abs(s1 * s2) / l1
    return np.stack([l1, l2, l3], axis=1).astype(np.float32)


def rs_chain(rs, g_sigma):
    """dL/d(theta, s1, s2) from dL/dSigma = [[g1, g2], [g2, g3]] (Sigma12 and
    Sigma21 as separate entries, App. A.2's convention), FP64:
    dL/dx = g1 dSigma11/dx + 2 g2 dSigma12/dx + g3 dSigma22/dx."""
    rs = np.asarray(rs, np.float64)
    th, s1, s2 = rs[:, 0], rs[:, 1], rs[:, 2]
    c, s = np.cos(th), np.sin(th)
    g1, g2, g3 = (np.asarray(g_sigma, np.float64)[:, i] for i in range(3))
    d_th = g1 * 2 * c * s * (s2 * s2 - s1 * s1) + 2 * g2 * (c * c - s * s) * (s1 * s1 - s2 * s2) \
        + g3 * 2 * c * s * (s1 * s1 - s2 * s2)
    d_s1 = g1 * 2 * c * c * s1 + 2 * g2 * 2 * c * s * s1 + g3 * 2 * s * s * s1
    d_s2 = g1 * 2 * s * s * s2 - 2 * g2 * 2 * c * s * s2 + g3 * 2 * c * c * s2
    return np.stack([d_th, d_s1, d_s2], axis=1)


def chol_to_sigma_grad(chol, g_chol):
    """dL/dSigma (entries g1, g2, g3, App. A.2's convention) recovered from
    dL/dl: the Cholesky chain dL/dl1 = 2 g1 l1 + 2 g2 l2, dL/dl2 = 2 g2 l1 +
    2 g3 l2, dL/dl3 = 2 g3 l3 solved for (g1, g2, g3)."""
    l = np.asarray(chol, np.float64)
    gl = np.asarray(g_chol, np.float64)
    g3 = gl[:, 2] / (2 * l[:, 2])
    g2 = (gl[:, 1] - 2 * g3 * l[:, 1]) / (2 * l[:, 0])
    g1 = (gl[:, 0] - 2 * g2 * l[:, 1]) / (2 * l[:, 0])
    return np.stack([g1, g2, g3], axis=1)


def rs_forward_backward(means, rs, color, target, T, shift=0.0):
    """forward_backward for the rotation-scaling form (shift = 0.5 adds App.
    C.1's +0.5 to s1, s2): Sigma's Cholesky vector from rs_to_chol, the
    usual pass, then dL/dl -> dL/dSigma -> dL/d(theta, s1, s2)."""
    r_ = np.asarray(rs, np.float64).copy()
    r_[:, 1] += shift
    r_[:, 2] += shift
    chol = rs_to_chol(r_)
    r = forward_backward(means, chol, color, target, T)
    gs = chol_to_sigma_grad(chol, r["grads"]["chol"])
    live = (r["cnt"] > 0)[:, None]
    r["grads_rs"] = np.where(live, rs_chain(r_, np.nan_to_num(gs)), 0.0)
    return r


ADAN_BETAS = (0.98, 0.92, 0.99)  # decay factors of the three averages (Adan's 0.02, 0.08, 0.01)


def adan(param, grad, state, step, lr, betas=ADAN_BETAS, eps=ADAM_EPS):
    """One Adan step (Xie et al. 2022, Adaptive Nesterov momentum), FP64,
    without weight decay, with bias correction of the three averages.
    state = (m, v, n, g_prev); on the first step (step == 1) the previous
    gradient is taken equal to the current one, so the difference is 0.
      m = b1 m + (1 - b1) g                       (gradient average)
      v = b2 v + (1 - b2) (g - g_prev)            (gradient-difference average)
      n = b3 n + (1 - b3) (g + b2 (g - g_prev))^2 (second moment of the
                                                   Nesterov-corrected gradient)
      p -= lr (m^ + b2 v^) / (sqrt(n^) + eps),  x^ = x / (1 - b^step)
    Returns (param, (m, v, n, g))."""
    b1, b2, b3 = betas
    p = np.asarray(param, np.float64)
    g = np.asarray(grad, np.float64)
    m, v, n, gp = (np.asarray(x, np.float64) for x in state)
    if step == 1:
        gp = g
    d = g - gp
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * d
    n = b3 * n + (1.0 - b3) * (g + b2 * d) ** 2
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    nh = n / (1.0 - b3 ** step)
    return p - lr * (mh + b2 * vh) / (np.sqrt(nh) + eps), (m, v, n, g)


def lr_at(lr, step, halve_every):
    """Learning rate of 1-based step `step`: halved every `halve_every`
    steps (Sec. 4.1: 1e-3, halved every 20000); 0 = constant."""
    if not halve_every:
        return lr
    return lr * 0.5 ** ((step - 1) // halve_every)


def vq_decode(means16, idx, codebooks):
    """Codec decode (Sec. 3.3): positions from FP16; Cholesky and colour as
    the sum over RVQ stages of codebook rows (hat c^M = sum_k C^k[i^k]),
    evaluated in FP64 in stage order and rounded once to FP32.

    means16 [n,2] float16 (or its uint16 bits), idx [2][M][n] uint8,
    codebooks [2][M][B][3] float32 (attr 0 = Cholesky, 1 = colour)."""
    m16 = np.asarray(means16)
    if m16.dtype == np.uint16:
        m16 = m16.view(np.float16)
    means = m16.astype(np.float64).astype(np.float32)
    idx = np.asarray(idx)
    cb = np.asarray(codebooks, np.float32)
    outs = []
    for a in range(2):
        acc = np.zeros((idx.shape[2], 3), np.float64)
        for s in range(idx.shape[1]):
            acc = acc + cb[a, s][idx[a, s].astype(np.int64)].astype(np.float64)
        outs.append(acc.astype(np.float32))
    return means, outs[0], outs[1]


def rvq_encode(x, codebooks_attr):
    """Greedy residual VQ (Sec. 3.3): stage m picks
    argmin_k || C^m[k] - (x - hat x^{m-1}) ||^2 (lowest k on ties), FP64.
    x [n,3], codebooks_attr [M][B][3] -> idx [M][n] uint8."""
    x = np.asarray(x, np.float64)
    cb = np.asarray(codebooks_attr, np.float32).astype(np.float64)
    M = cb.shape[0]
    idx = np.zeros((M, x.shape[0]), np.uint8)
    recon = np.zeros_like(x)
    for m in range(M):
        res = x - recon
        d2 = ((res[:, None, :] - cb[m][None, :, :]) ** 2).sum(-1)
        k = np.argmin(d2, axis=1)  # first minimum = lowest index
        idx[m] = k.astype(np.uint8)
        recon = recon + cb[m][k]
    return idx


def psnr(out, target):
    """PSNR = 10 log10(1 / MSE) on the output clamped to [0, 1] (Sec. 4.1)."""
    o = np.clip(np.asarray(out, np.float64), 0.0, 1.0)
    mse = np.mean((o - np.asarray(target, np.float64)) ** 2)
    return float(10.0 * np.log10(1.0 / mse)) if mse > 0 else float("inf")


# ---------------------------------------------------------------------------
# Codec fine-tuning (Sec. 3.3 attribute quantisation-aware fine-tuning,
# Sec. 3.4 total loss). Every decision that yields an integer (a half-precision
# rounding, a quantiser code, an RVQ index) is taken in FP32 with one rounding
# per operation, the precision the GPU takes it in; sums are FP64.
# ---------------------------------------------------------------------------

def fp16_round(x):
    """Positions stored at 16-bit float precision (Sec. 3.3): FP32 -> FP16
    (round to nearest even) -> FP32."""
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float32)


def lsq_fake_quant(l, gamma, beta, bits):
    """b-bit asymmetric quantiser of the Cholesky vector (Sec. 3.3, the LSQ+
    form): x = (l_i - beta_i) / gamma_i, code = round(clamp(x, 0, 2^b - 1))
    (half to even), l_bar = code * gamma_i + beta_i; gamma, beta are shared
    by all Gaussians, one pair per component i.
    l [n,3]; gamma, beta [3]. Returns (l_bar f32 [n,3], x f32 [n,3],
    code f32 [n,3]); a non-finite x gives a non-finite l_bar and code."""
    l = np.asarray(l, np.float32)
    g = np.asarray(gamma, np.float32)
    b = np.asarray(beta, np.float32)
    qp = np.float32(2 ** bits - 1)
    with np.errstate(all="ignore"):
        x = (l - b) / g
        xc = np.where(x < 0, np.float32(0), np.where(x > qp, qp, x)).astype(np.float32)
        q = np.rint(xc).astype(np.float32)
        lbar = (q * g + b).astype(np.float32)
    return lbar, x.astype(np.float32), q


def lsq_ste_grads(g_lbar, x, q, bits):
    """Gradients of the quantiser with the straight-through estimator
    (d round(x)/dx taken as 1, the LSQ+ convention): inside the clamp range
    dl_bar/dl = 1, dl_bar/dgamma = code - x, dl_bar/dbeta = 0; below it
    l_bar = beta (0, 0, 1); above it l_bar = (2^b - 1) gamma + beta
    (0, 2^b - 1, 1). Returns (dL/dl [n,3], dL/dgamma [3], dL/dbeta [3]),
    FP64; a non-finite x contributes nothing."""
    g = np.asarray(g_lbar, np.float64)
    x = np.asarray(x, np.float64)
    q = np.asarray(q, np.float64)
    qp = float(2 ** bits - 1)
    inside = (x >= 0) & (x <= qp)
    below = x < 0
    above = x > qp
    g_l = np.where(inside, g, 0.0)
    g_gamma = np.where(inside, g * (q - np.where(inside, x, 0.0)), np.where(above, g * qp, 0.0)).sum(axis=0)
    g_beta = np.where(below | above, g, 0.0).sum(axis=0)
    return g_l, g_gamma, g_beta


def rvq_assign_f32(c, codebooks):
    """Greedy residual VQ of the colour coefficients (Sec. 3.3, Eq. 10) with
    FP32 decisions: r^0 = c'; stage m takes the entry j minimising
    ((C_j0 - r_0)^2 + (C_j1 - r_1)^2) + (C_j2 - r_2)^2 (each operation
    rounded to FP32), scanning j upward and moving only on a strictly smaller
    distance (lowest index on ties; a NaN distance never wins, so an
    all-NaN stage picks 0); r^m = r^{m-1} - C^m[i^m] in FP32.
    c [n,3], codebooks [M][B][3]. Returns (idx [M][n] int64, c_hat f32 [n,3]
    = sum over stages of the chosen entries in FP64 rounded once,
    r_in f32 [M][n][3] = the residual each stage quantised)."""
    c = np.asarray(c, np.float32)
    cb = np.asarray(codebooks, np.float32)
    M, Bn = cb.shape[0], cb.shape[1]
    n = c.shape[0]
    r = c.copy()
    idx = np.zeros((M, n), np.int64)
    r_in = np.zeros((M, n, 3), np.float32)
    with np.errstate(all="ignore"):
        for m in range(M):
            r_in[m] = r
            best = np.zeros(n, np.int64)
            bd = None
            for j in range(Bn):
                e = (cb[m, j][None, :] - r).astype(np.float32)
                d = ((e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1]) + e[:, 2] * e[:, 2]).astype(np.float32)
                if bd is None:
                    bd = d
                    continue
                take = d < bd
                best = np.where(take, j, best)
                bd = np.where(take, d, bd)
            idx[m] = best
            r = (r - cb[m][best]).astype(np.float32)
    chat = np.zeros((n, 3), np.float64)
    for m in range(M):
        chat = chat + cb[m][idx[m]].astype(np.float64)
    return idx, chat.astype(np.float32), r_in


def commitment_loss(r_in, codebooks, idx):
    """Commitment loss (Sec. 3.3, Eq. 11): L_c = 1/(N B) sum over stages m
    and Gaussians n of || r_n^{m-1} - C^m[i_n^m] ||^2, r^{m-1} = c' minus the
    first m-1 stages' entries (the stop-gradient operand). FP64."""
    r_in = np.asarray(r_in, np.float64)
    cb = np.asarray(codebooks, np.float32).astype(np.float64)
    M, Bn = cb.shape[0], cb.shape[1]
    n = r_in.shape[1]
    if n == 0:
        return 0.0
    tot = 0.0
    for m in range(M):
        tot += float(((r_in[m] - cb[m][np.asarray(idx[m])]) ** 2).sum())
    return tot / (n * Bn)


def ema_codebook_update(count, total, idx, r_in, decay, eps):
    """Exponential-moving-average codebook update (Sec. 3.4): per stage m and
    entry j, with n_j Gaussians assigned and s_j the sum of their residuals
    r^{m-1}: count_j <- d count_j + (1 - d) n_j, total_j <- d total_j +
    (1 - d) s_j; the count is Laplace-smoothed, N_j = (count_j + eps) /
    (sum count + B eps) * sum count, and C_j = total_j / N_j.
    count [M][B], total [M][B][3], idx [M][n], r_in [M][n][3]. Returns
    (count, total, codebooks), FP64."""
    count = np.asarray(count, np.float64).copy()
    total = np.asarray(total, np.float64).copy()
    r_in = np.asarray(r_in, np.float64)
    M, Bn = count.shape
    cb = np.zeros((M, Bn, 3))
    for m in range(M):
        n_j = np.bincount(np.asarray(idx[m]), minlength=Bn).astype(np.float64)
        s_j = np.zeros((Bn, 3))
        np.add.at(s_j, np.asarray(idx[m]), r_in[m])
        count[m] = decay * count[m] + (1.0 - decay) * n_j
        total[m] = decay * total[m] + (1.0 - decay) * s_j
        tot = count[m].sum()
        smoothed = (count[m] + eps) / (tot + Bn * eps) * tot
        with np.errstate(all="ignore"):
            cb[m] = total[m] / smoothed[:, None]
    return count, total, cb


def codec_forward_backward(means, chol, color, gamma, beta, codebooks, bits, target, T):
    """One fine-tuning pass (Sec. 3.3): the render sees FP16 positions, the
    quantised Cholesky vector and the RVQ colour; gradients pass straight
    through the FP16 rounding and the RVQ (dL/dc' = dL/dc_hat) and through
    the quantiser as lsq_ste_grads. means, chol are the pixel-space values
    the quantisers act on. Returns forward_backward's dict plus "codec":
    means16, chol_q, codes (uint8 [n,3]), x, idx, color_q, r_in, commit (L_c)
    and grads {means, chol, color, gamma, beta}."""
    mq = fp16_round(means)
    lbar, x, q = lsq_fake_quant(chol, gamma, beta, bits)
    idx, chat, r_in = rvq_assign_f32(color, codebooks)
    r = forward_backward(mq, lbar, chat, target, T)
    g = r["grads"]
    g_l, g_gamma, g_beta = lsq_ste_grads(g["chol"], x, q, bits)
    codes = np.where(np.isfinite(q), q, 0).astype(np.uint8)
    r["codec"] = {"means16": mq, "chol_q": lbar, "codes": codes, "x": x, "idx": idx, "color_q": chat,
                  "r_in": r_in, "commit": commitment_loss(r_in, codebooks, idx),
                  "grads": {"means": g["means"], "chol": g_l, "color": g["color"], "gamma": g_gamma,
                            "beta": g_beta}}
    return r


# ---------------------------------------------------------------------------
# The ablations of Table 3: colour and opacity kept apart ("w/o M", 9
# parameters, Sec. 3.1's basic 2D Gaussian) and sorted alpha-blending in
# place of the accumulated sum ("w/o AR", Eq. 3-4).
# ---------------------------------------------------------------------------

BLEND_THRESHOLDS = (1.0 / 255.0, 0.99, 1e-4)  # alpha skip, alpha clamp, transmittance stop (3D GS)
# A decision within this relative distance of its threshold is flagged: an
# FP32 evaluation (alpha to a few 1e-7, the transmittance, a product of up to a
# few hundred factors, to about 2e-5) may take it the other way.
BLEND_AMBIGUITY = 3e-5


def sigmoid_opacity(logit):
    """Opacity o = 1 / (1 + exp(-logit)) in FP64, rounded once to FP32 (the
    activation 3D GS applies to its opacity; the paper names none)."""
    z = np.asarray(logit, np.float64)
    return (1.0 / (1.0 + np.exp(-z))).astype(np.float32)


def opacity_forward_backward(means, chol, color, logit, target, T):
    """Accumulated summation with separate colour and opacity (Eq. 5,
    C_i = sum c_n o_n exp(-sigma_n)): the plain pass on c' = c o (one FP32
    rounding), then dL/dc = dL/dc' o and dL/dlogit = (dL/dc' . c) o (1 - o)."""
    o = sigmoid_opacity(logit)
    c = np.asarray(color, np.float32)
    cp = (c * o[:, None]).astype(np.float32)
    r = forward_backward(means, chol, cp, target, T)
    g = r["grads"]
    o64 = o.astype(np.float64)
    r["grads_opacity"] = {"color": g["color"] * o64[:, None],
                          "logit": (g["color"] * c.astype(np.float64)).sum(axis=1) * o64 * (1.0 - o64),
                          "abs_color": g["abs"]["color"] * o64[:, None],
                          "abs_logit": (g["abs"]["color"] * np.abs(c)).sum(axis=1) * o64 * (1.0 - o64)}
    return r


def blend_render(means, chol, color, opac, ids, ranges, W, H, T, thresholds=BLEND_THRESHOLDS, amb=BLEND_AMBIGUITY):
    """Sorted alpha-blending (Eq. 3-4) over the binned lists, front to back in
    ascending g with 3D GS's thresholds (gi_oracle.c). Returns (out [H,W,3]
    FP64, t_final [H,W], n_last [H,W] int32, ambiguous [H,W] bool)."""
    means, chol, color, opac = _f32(means), _f32(chol), _f32(color), _f32(opac)
    ids = np.ascontiguousarray(ids, np.uint32)
    if ids.size == 0:
        ids = np.zeros(1, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.int32)
    out = np.zeros((H, W, 3), np.float64)
    tf = np.zeros((H, W), np.float64)
    nl = np.zeros((H, W), np.int32)
    flags = np.zeros((H, W), np.uint8)
    a_min, a_max, t_min = thresholds
    _load().gio_render_blend(_p(means), _p(chol), _p(color), _p(opac), _p(ids), _p(ranges), W, H, T,
                             a_min, a_max, t_min, amb, _p(out), _p(tf), _p(nl), _p(flags))
    return out, tf, nl, flags.astype(bool)


def blend_backward(means, chol, color, opac, ids, ranges, W, H, T, out, n_last, dldc, thresholds=BLEND_THRESHOLDS,
                   ambiguous=None):
    """Analytic gradients of blend_render (gi_oracle.c): dict of FP64 means
    [n,2], chol [n,3], color [n,3], opac [n] (dL/do), abs [n,9] and
    abs_ambiguous [n,9] (magnitudes over the flagged pixels)."""
    means, chol, color, opac = _f32(means), _f32(chol), _f32(color), _f32(opac)
    ids = np.ascontiguousarray(ids, np.uint32)
    if ids.size == 0:
        ids = np.zeros(1, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.int32)
    out = np.ascontiguousarray(out, np.float64)
    n_last = np.ascontiguousarray(n_last, np.int32)
    dldc = np.ascontiguousarray(dldc, np.float64)
    n = means.shape[0]
    gm = np.zeros((n, 2)); gl = np.zeros((n, 3)); gc = np.zeros((n, 3)); go = np.zeros(n); ga = np.zeros((n, 9))
    gaa = np.zeros((n, 9))
    amb = np.ascontiguousarray(np.zeros((H, W), np.uint8) if ambiguous is None else ambiguous, np.uint8)
    a_min, a_max, _ = thresholds
    _load().gio_backward_blend(_p(means), _p(chol), _p(color), _p(opac), _p(ids), _p(ranges), n, W, H, T,
                               a_min, a_max, _p(out), _p(n_last), _p(amb), _p(dldc), _p(gm), _p(gl), _p(gc), _p(go),
                               _p(ga), _p(gaa))
    return {"means": gm, "chol": gl, "color": gc, "opac": go, "abs": ga, "abs_ambiguous": gaa}


def blend_forward_backward(means, chol, color, logit, target, T, thresholds=BLEND_THRESHOLDS):
    """One alpha-blending pass with opacity o = sigmoid_opacity(logit): the
    support rule and binning of the accumulated form (3-sigma rect, ascending
    g per tile), blend_render, the L2 loss, blend_backward, and
    dL/dlogit = dL/do o (1 - o)."""
    H, W, _ = target.shape
    o = sigmoid_opacity(logit)
    rect, cnt = rect_rule(means, chol, color, W, H, T)
    ids, ranges, pair_off = bin_tiles(rect, cnt, W, H, T)
    out, tf, nl, amb = blend_render(means, chol, color, o, ids, ranges, W, H, T, thresholds)
    L, d = loss(out, target)
    g = blend_backward(means, chol, color, o, ids, ranges, W, H, T, out, nl, d, thresholds, amb)
    o64 = o.astype(np.float64)
    g["logit"] = g["opac"] * o64 * (1.0 - o64)
    g["abs_logit"] = g["abs"][:, 8] * o64 * (1.0 - o64)
    g["abs_ambiguous_logit"] = g["abs_ambiguous"][:, 8] * o64 * (1.0 - o64)
    return dict(rect=rect, cnt=cnt, ids=ids, ranges=ranges, out=out, t_final=tf, n_last=nl, ambiguous=amb,
                loss=L, dldc=d, grads=g, opac=o)


def codec_decode(means16, codes, gamma, beta, idx, codebooks):
    """Decode of the codec stream (Sec. 3.3): FP16 positions to FP32; the
    Cholesky vector from its b-bit codes, l_bar_i = code_i gamma_i + beta_i
    (Eq. 9, FP32 product and sum); the colour as the sum of the chosen RVQ
    entries in stage order (Eq. 10) in FP64, rounded once. means16 [n,2]
    float16 (or uint16 bits), codes [n,>=3] uint8, gamma/beta [3],
    idx [M][n], codebooks [M][B][3]."""
    m16 = np.asarray(means16)
    if m16.dtype in (np.uint16, np.int16):
        m16 = m16.view(np.float16)
    means = m16.astype(np.float32)
    q = np.asarray(codes)[:, :3].astype(np.float32)
    g = np.asarray(gamma, np.float32)
    b = np.asarray(beta, np.float32)
    chol = ((q * g).astype(np.float32) + b).astype(np.float32)
    cb = np.asarray(codebooks, np.float32)
    idx = np.asarray(idx).astype(np.int64)
    acc = np.zeros((means.shape[0], 3), np.float64)
    for m in range(cb.shape[0]):
        acc = acc + cb[m][idx[m]].astype(np.float64)
    return means, chol, acc.astype(np.float32)
