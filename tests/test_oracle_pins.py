"""Pins of the FP64 oracle against facts the paper and mathematics fix.

Each test pins one oracle function to something other than itself: a closed
form, an invariant the paper states, a brute-force evaluation, or a library
routine. CPU only.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _tiny(n=50, W=64, H=48, seed=7):
    means, chol, color = synth.init_gaussians(n, W, H, seed)
    return means, chol, color


# --------------------------------------------------------------------------
# Render (Eq. 7)
# --------------------------------------------------------------------------

def test_isotropic_closed_form():
    """One isotropic Gaussian (l1 = l3 = s, l2 = 0) has Sigma^-1 = I/s^2, so
    C(p) = c' exp(-|p - mu|^2 / (2 s^2)) at every supported pixel."""
    W, H, T = 64, 64, 32
    s = 2.5
    mu = np.array([[30.3, 33.7]], np.float32)
    chol = np.array([[s, 0.0, s]], np.float32)
    col = np.array([[0.7, -0.2, 1.3]], np.float32)
    rect, cnt = oracle.rect_rule(mu, chol, col, W, H, T)
    ids, ranges, _ = oracle.bin_tiles(rect, cnt, W, H, T)
    out = oracle.render(mu, chol, col, ids, ranges, W, H, T)
    ys, xs = np.mgrid[0:H, 0:W]
    d2 = (xs + 0.5 - float(mu[0, 0])) ** 2 + (ys + 0.5 - float(mu[0, 1])) ** 2
    w = np.exp(-d2 / (2 * s * s))
    ref = w[:, :, None] * col[0].astype(np.float64)[None, None, :]
    # rect covers all four tiles here (rx = ry = 7.5)
    assert cnt[0] == 4
    # exp(-sigma) turns a relative error e of sigma into sigma*e: scale by sigma.
    sigma = d2 / (2 * s * s)
    tol = 8 * np.finfo(np.float64).eps * (1.0 + sigma)[:, :, None] * np.abs(ref)
    assert np.all(np.abs(out - ref) <= tol)


def test_linear_in_colour():
    """C_i is linear in the weighted colours c' (Eq. 7): scaling by a power of
    two is exact, and colours on a coarse grid add exactly in FP32."""
    W, H, T = 64, 48, 8
    means, chol, _ = _tiny()
    g = np.random.default_rng(8)
    c1 = (g.integers(0, 256, (50, 3)) / 1024.0).astype(np.float32)
    c2 = (g.integers(-256, 256, (50, 3)) / 1024.0).astype(np.float32)
    rect, cnt = oracle.rect_rule(means, chol, c1, W, H, T)
    ids, ranges, _ = oracle.bin_tiles(rect, cnt, W, H, T)
    a = oracle.render(means, chol, c1, ids, ranges, W, H, T)
    b = oracle.render(means, chol, c2, ids, ranges, W, H, T)
    half = oracle.render(means, chol, (c1 * np.float32(0.5)), ids, ranges, W, H, T)
    np.testing.assert_array_equal(half, 0.5 * a)
    s = oracle.render(means, chol, c1 + c2, ids, ranges, W, H, T)
    np.testing.assert_allclose(s, a + b, rtol=1e-13, atol=1e-15)


def test_permutation_invariance():
    """The sum has no order (Sec. 3.2): permuting the Gaussians changes only
    the rounding order."""
    W, H, T = 64, 48, 8
    means, chol, col = _tiny()
    rect, cnt = oracle.rect_rule(means, chol, col, W, H, T)
    ids, ranges, _ = oracle.bin_tiles(rect, cnt, W, H, T)
    a = oracle.render(means, chol, col, ids, ranges, W, H, T)
    perm = np.random.default_rng(3).permutation(means.shape[0])
    m2, l2, c2 = means[perm], chol[perm], col[perm]
    r2, n2 = oracle.rect_rule(m2, l2, c2, W, H, T)
    i2, g2, _ = oracle.bin_tiles(r2, n2, W, H, T)
    b = oracle.render(m2, l2, c2, i2, g2, W, H, T)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-15)


def test_union_additivity():
    """render(A u B) = render(A) + render(B)."""
    W, H, T = 64, 48, 8
    means, chol, col = _tiny()
    out = {}
    for name, sl in (("all", slice(None)), ("a", slice(0, 20)), ("b", slice(20, None))):
        m, l, c = means[sl], chol[sl], col[sl]
        r, n = oracle.rect_rule(m, l, c, W, H, T)
        i, g, _ = oracle.bin_tiles(r, n, W, H, T)
        out[name] = oracle.render(m, l, c, i, g, W, H, T)
    np.testing.assert_allclose(out["all"], out["a"] + out["b"], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("W,H,T", [(64, 48, 8), (61, 45, 8), (40, 33, 16)])
def test_binned_equals_brute_force(W, H, T):
    """Binned render == brute force over every (pixel, Gaussian) with the same
    support predicate, bit for bit (same FP64 operations, same order)."""
    means, chol, col = synth.init_gaussians(50, W, H, 11)
    rect, cnt = oracle.rect_rule(means, chol, col, W, H, T)
    ids, ranges, _ = oracle.bin_tiles(rect, cnt, W, H, T)
    a = oracle.render(means, chol, col, ids, ranges, W, H, T)
    b = oracle.render_brute(means, chol, col, rect, cnt, W, H, T, use_support=True)
    np.testing.assert_array_equal(a, b)
    # The untruncated sum differs only by the 3-sigma truncation.
    u = oracle.render_brute(means, chol, col, rect, cnt, W, H, T, use_support=False)
    assert np.all(u >= a - 1e-12)


# --------------------------------------------------------------------------
# Support rule and binning
# --------------------------------------------------------------------------

def test_rect_matches_ellipse_extent():
    """rx = 3|l1|, ry = 3 sqrt(l2^2 + l3^2) are the half-extents of the
    3-sigma ellipse {d : d^T Sigma^-1 d <= 9}: its boundary is d = 3 L u."""
    g = np.random.default_rng(5)
    th = np.linspace(0, 2 * np.pi, 20001)
    u = np.stack([np.cos(th), np.sin(th)])
    for _ in range(50):
        l1, l3 = np.exp(g.uniform(-1, 3, 2))
        l2 = g.uniform(-4, 4)
        L = np.array([[l1, 0.0], [l2, l3]])
        d = 3.0 * L @ u
        # boundary really is the 3-sigma contour
        Sinv = np.linalg.inv(L @ L.T)
        q = np.einsum("in,ij,jn->n", d, Sinv, d)
        np.testing.assert_allclose(q, 9.0, rtol=1e-10)
        rx, ry = 3 * abs(l1), 3 * math.sqrt(l2 * l2 + l3 * l3)
        assert np.abs(d[0]).max() <= rx * (1 + 1e-12)
        assert np.abs(d[1]).max() <= ry * (1 + 1e-12)
        assert np.abs(d[0]).max() >= rx * (1 - 1e-6)
        assert np.abs(d[1]).max() >= ry * (1 - 1e-6)


def test_rect_tiles_brute_force():
    """The tile rect is exactly the set of tiles whose half-open square meets
    the closed box [mu - r, mu + r], clipped to the image (FP64 check away
    from ties)."""
    W, H, T = 200, 130, 16
    means, chol, col = synth.init_gaussians(400, W, H, 21)
    means = means.copy()
    means[:40] -= 20.0  # some partly off-screen
    rect, cnt = oracle.rect_rule(means, chol, col, W, H, T)
    tw, th = oracle.tiles(W, H, T)
    for g in range(means.shape[0]):
        mx, my = float(means[g, 0]), float(means[g, 1])
        l1, l2, l3 = (float(v) for v in chol[g])
        rx, ry = 3 * abs(l1), 3 * math.sqrt(l2 * l2 + l3 * l3)
        xs = [tx for tx in range(tw) if tx * T <= mx + rx and (tx + 1) * T > mx - rx]
        ys = [ty for ty in range(th) if ty * T <= my + ry and (ty + 1) * T > my - ry]
        near_tie = any(abs(v / T - round(v / T)) < 1e-5 for v in (mx - rx, mx + rx, my - ry, my + ry))
        if near_tie:
            continue
        if not xs or not ys:
            assert cnt[g] == 0 and tuple(rect[g]) == (0, 0, 0, 0)
        else:
            assert tuple(rect[g]) == (xs[0], ys[0], xs[-1] + 1, ys[-1] + 1), g
            assert cnt[g] == len(xs) * len(ys)


def test_rect_culling():
    W, H, T = 64, 64, 16
    means = np.array([[8, 8], [np.nan, 3], [10, 10], [500, 500], [10, 10], [-40, 10]], np.float32)
    chol = np.array([[2, 0, 2], [2, 0, 2], [0, 1, 2], [2, 0, 2], [2, 0, 2], [2, 0, 2]], np.float32)
    col = np.array([[.1, .1, .1], [.1, .1, .1], [.1, .1, .1], [.1, .1, .1], [np.inf, 0, 0], [.1, .1, .1]],
                   np.float32)
    rect, cnt = oracle.rect_rule(means, chol, col, W, H, T)
    assert cnt[0] == 1 and tuple(rect[0]) == (0, 0, 1, 1)
    assert list(cnt[1:]) == [0, 0, 0, 0, 0]
    assert np.all(rect[1:] == 0)


def test_culling_rule_covers_a_finite_record_factor():
    """The support rule culls on the FP32 inverse covariance (Eq. 5 needs a
    finite Sigma^-1). A renderer that evaluates sigma through the scaled
    inverse Cholesky factor k L^-1 (k = sqrt(log2(e)/2), m11 = k/l1,
    m21 = -(l2 m11)/l3, m22 = k/l3 in FP32) needs no cull of its own. With
    F = FLT_MAX, a finite S22 = l2^2 + l3^2 and finite
    A = S22/(l1 l3)^2 >= 1/l1^2, C = 1/l3^2 give |l1|, |l3| >= 1/sqrt(F) and
    |l2/l1| <= sqrt(F) |l2 l3| / sqrt(l2^2 + l3^2) <= F/2, so |m11|, |m22|
    <= k sqrt(F) and the largest intermediate, |l2 m11|, stays below k F/2:
    a margin of 2.4x that rounding cannot close. Checked on the oracle's
    own cull over random magnitudes across the whole FP32 range and a dense
    sample at that extreme (l2 = l3 near sqrt(F/2), l1 near sqrt(2/F))."""
    W, H, T = 64, 64, 16
    g = np.random.default_rng(17)
    n = 400000
    mag = lambda lo, hi, k: (10.0 ** g.uniform(lo, hi, k)) * g.choice([-1.0, 1.0], k)
    l1 = np.concatenate([mag(-46, 39, n), 10.0 ** g.uniform(np.log10(7.0e-20), np.log10(1.0e-19), n)])
    l2 = np.concatenate([mag(-46, 39, n), mag(np.log10(1.1e19), np.log10(1.4e19), n)])
    l3 = np.concatenate([mag(-46, 39, n), mag(np.log10(1.1e19), np.log10(1.4e19), n)])
    with np.errstate(over="ignore"):  # magnitudes above FLT_MAX become infinities (culled)
        chol = np.stack([l1, l2, l3], axis=1).astype(np.float32)
    m = len(chol)
    means = np.full((m, 2), 20.0, np.float32)
    col = np.full((m, 3), 0.1, np.float32)
    with np.errstate(all="ignore"):
        rect, cnt = oracle.rect_rule(means, chol, col, W, H, T)
        f1, f2, f3 = chol[:, 0], chol[:, 1], chol[:, 2]
        k = np.float32(0.84932180028801904272)
        m11 = k / f1
        m22 = k / f3
        m21 = -((f2 * m11) / f3)
    kept = cnt > 0
    assert kept[:n].sum() > 20000 and (~kept[:n]).sum() > 20000 and kept[n:].sum() > 20000
    assert np.all(np.isfinite(m11[kept]) & np.isfinite(m21[kept]) & np.isfinite(m22[kept]))
    with np.errstate(all="ignore"):
        assert np.max(np.abs(f2[kept] * m11[kept])) <= 0.5 * np.finfo(np.float32).max


@pytest.mark.parametrize("W,H,T", [(64, 48, 8), (61, 45, 8), (100, 70, 16), (130, 99, 32)])
def test_binning_brute_force(W, H, T):
    """Per-tile lists = every g whose rect holds the tile, ascending g."""
    means, chol, col = synth.init_gaussians(120, W, H, 31)
    rect, cnt = oracle.rect_rule(means, chol, col, W, H, T)
    ids, ranges, pair_off = oracle.bin_tiles(rect, cnt, W, H, T)
    tw, th = oracle.tiles(W, H, T)
    pos = 0
    for t in range(tw * th):
        tx, ty = t % tw, t // tw
        lst = [g for g in range(120) if cnt[g] and rect[g, 0] <= tx < rect[g, 2] and rect[g, 1] <= ty < rect[g, 3]]
        if lst:
            assert tuple(ranges[t]) == (pos, pos + len(lst))
            assert list(ids[pos:pos + len(lst)]) == lst
            pos += len(lst)
        else:
            assert tuple(ranges[t]) == (0, 0)
    assert pos == ids.shape[0]
    np.testing.assert_array_equal(pair_off, np.concatenate([[0], np.cumsum(cnt.astype(np.int64))]))


def test_empty_inputs():
    W, H, T = 32, 32, 16
    z = np.zeros((0, 2), np.float32), np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32)
    rect, cnt = oracle.rect_rule(*z, W, H, T)
    ids, ranges, pair_off = oracle.bin_tiles(rect, cnt, W, H, T)
    assert ids.shape[0] == 0 and np.all(ranges == 0) and pair_off.tolist() == [0]
    out = oracle.render(*z, ids, ranges, W, H, T)
    assert np.all(out == 0)


# --------------------------------------------------------------------------
# Loss and gradients (Sec. 3.4, App. A)
# --------------------------------------------------------------------------

def test_loss_is_mse():
    g = np.random.default_rng(1)
    out = g.uniform(0, 1, (9, 7, 3))
    tgt = g.uniform(0, 1, (9, 7, 3)).astype(np.float32)
    L, d = oracle.loss(out, tgt)
    r = out - tgt.astype(np.float64)
    assert L == pytest.approx(np.mean(r ** 2), rel=1e-14)
    np.testing.assert_allclose(d, 2 * r / r.size, rtol=1e-14)


def _loss_fixed_support(means, chol, col, ids, ranges, W, H, T, target, G=None):
    out = oracle.render(means, chol, col, ids, ranges, W, H, T)
    if G is None:
        return oracle.loss(out, target)[0]
    return float((out * G).sum())


@pytest.mark.parametrize("which", ["mse", "linear"])
def test_gradients_match_finite_differences(which):
    """Central finite differences of the FP64 loss (support held fixed)
    against the analytic App. A gradients, every parameter of every
    Gaussian. Catches a dropped c' in dC/dsigma, a sign error in d, and the
    l2 term of dL/dl2."""
    W, H, T = 24, 20, 8
    n = 6
    means, chol, col = synth.init_gaussians(n, W, H, 41)
    chol = chol.copy()
    chol[:, 1] = np.array([1.5, -1.7, 0.8, -0.4, 1.9, -1.1], np.float32)  # l2 far from 0
    target = synth.image(W, H, 41, n_blobs=5)
    rect, cnt = oracle.rect_rule(means, chol, col, W, H, T)
    ids, ranges, _ = oracle.bin_tiles(rect, cnt, W, H, T)
    out = oracle.render(means, chol, col, ids, ranges, W, H, T)
    G = None
    if which == "mse":
        _, d = oracle.loss(out, target)
    else:
        G = np.random.default_rng(2).standard_normal((H, W, 3))
        d = G
    gr = oracle.backward(means, chol, col, rect, cnt, W, H, T, d)
    params = {"means": means, "chol": chol, "color": col}
    for name, arr in params.items():
        ana = gr[name]
        num = np.zeros_like(ana)
        for idx in np.ndindex(arr.shape):
            v = float(arr[idx])
            # power-of-two steps keep v +- h exact in FP32; Richardson
            # extrapolation of two central differences removes the h^2 term.
            h = 2.0 ** (math.floor(math.log2(abs(v))) - 8) if v != 0 else 2.0 ** -12

            def central(hh):
                ap, am = arr.copy(), arr.copy()
                ap[idx] = np.float32(v + hh)
                am[idx] = np.float32(v - hh)
                assert float(ap[idx]) - float(am[idx]) == 2 * hh
                pp = dict(params, **{name: ap})
                pm = dict(params, **{name: am})
                Lp = _loss_fixed_support(pp["means"], pp["chol"], pp["color"], ids, ranges, W, H, T, target, G)
                Lm = _loss_fixed_support(pm["means"], pm["chol"], pm["color"], ids, ranges, W, H, T, target, G)
                return (Lp - Lm) / (2 * hh)

            num[idx] = (4.0 * central(h / 2) - central(h)) / 3.0
        scale = np.abs(ana).max()
        np.testing.assert_allclose(ana, num, rtol=1e-6, atol=1e-8 * scale, err_msg=name)


def test_isotropic_gradient_closed_form():
    """One isotropic Gaussian, upstream gradient 1 at one pixel of channel 0:
    dL/dc'_0 = w, dL/dmu = c'_0 w (p - mu)/s^2, dL/dl1 = c'_0 w dx^2/l1^3,
    dL/dl3 = c'_0 w dy^2/l3^3, dL/dl2 = c'_0 w dx dy/(l1 l3^2) at l2 = 0."""
    W, H, T = 32, 32, 32
    s = 3.0
    mu = np.array([[14.2, 17.9]], np.float32)
    chol = np.array([[s, 0.0, s]], np.float32)
    col = np.array([[0.6, 0.3, 0.1]], np.float32)
    rect, cnt = oracle.rect_rule(mu, chol, col, W, H, T)
    px, py = 19, 12
    G = np.zeros((H, W, 3))
    G[py, px, 0] = 1.0
    gr = oracle.backward(mu, chol, col, rect, cnt, W, H, T, G)
    dx, dy = px + 0.5 - float(mu[0, 0]), py + 0.5 - float(mu[0, 1])
    w = math.exp(-(dx * dx + dy * dy) / (2 * s * s))
    c0 = float(col[0, 0])
    assert gr["color"][0, 0] == pytest.approx(w, rel=1e-13)
    assert gr["color"][0, 1] == 0.0
    np.testing.assert_allclose(gr["means"][0], [c0 * w * dx / s ** 2, c0 * w * dy / s ** 2], rtol=1e-12)
    np.testing.assert_allclose(gr["chol"][0], [c0 * w * dx * dx / s ** 3, c0 * w * dx * dy / s ** 3,
                                               c0 * w * dy * dy / s ** 3], rtol=1e-12)


# --------------------------------------------------------------------------
# Adam, codec decode/encode
# --------------------------------------------------------------------------

def test_adam_first_step_closed_form():
    """From zero state, m_hat = g and v_hat = g^2, so the step is
    -lr g / (|g| + eps)."""
    g = np.random.default_rng(4).standard_normal(100)
    p0 = np.random.default_rng(5).standard_normal(100)
    p1, m, v = oracle.adam(p0, g, np.zeros(100), np.zeros(100), 1, 1e-2)
    np.testing.assert_allclose(p1, p0 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-14, atol=1e-16)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    gen = np.random.default_rng(6)
    p = gen.standard_normal(64)
    t = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(64); v = np.zeros(64)
    for step in range(1, 8):
        g = gen.standard_normal(64)
        t.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        p, m, v = oracle.adam(p, g, m, v, step, 3e-3)
        np.testing.assert_allclose(p, t.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_vq_decode_is_float32_sum():
    """One FP32 addition per stage in FP64 then rounded equals IEEE float32
    addition (double rounding is innocuous for +: 53 >= 2*24 + 2)."""
    cb = synth.codebooks(4000)
    n = 5000
    idx = synth.vq_indices(n, 4000)
    means = synth.init_gaussians(n, 768, 512, 4000)[0]
    m16 = means.astype(np.float16)
    dm, dl, dc = oracle.vq_decode(m16, idx, cb)
    np.testing.assert_array_equal(dm, m16.astype(np.float32))
    ref_l = cb[0, 0][idx[0, 0]] + cb[0, 1][idx[0, 1]]  # numpy float32 add
    ref_c = cb[1, 0][idx[1, 0]] + cb[1, 1][idx[1, 1]]
    assert ref_l.dtype == np.float32
    np.testing.assert_array_equal(dl.view(np.uint32), ref_l.view(np.uint32))
    np.testing.assert_array_equal(dc.view(np.uint32), ref_c.view(np.uint32))
    cb0 = cb.copy()
    cb0[:, 1] = 0.0
    _, dl0, dc0 = oracle.vq_decode(m16, idx, cb0)
    np.testing.assert_array_equal(dl0, cb[0, 0][idx[0, 0]])
    np.testing.assert_array_equal(dc0, cb[1, 0][idx[1, 0]])


def test_rvq_encode_greedy_argmin():
    cb = synth.codebooks(4100)
    x = synth.init_gaussians(300, 64, 64, 4100)[2]
    idx = oracle.rvq_encode(x, cb[1])
    res = x.astype(np.float64)
    for m in range(cb.shape[1]):
        c = cb[1, m].astype(np.float64)
        for i in range(x.shape[0]):
            d2 = ((c - res[i]) ** 2).sum(-1)
            k = int(idx[m, i])
            assert d2[k] == d2.min() and k == int(np.flatnonzero(d2 == d2.min())[0])
        res = res - c[idx[m].astype(int)]


def test_gradient_abs_sums():
    """The condition magnitudes bound the gradients (triangle inequality); for
    an axis-aligned Gaussian (l2 = 0, so B = 0) and a single contributing
    pixel nothing cancels and they equal |gradient|."""
    W, H, T, n = 40, 32, 8, 30
    means, chol, color = synth.init_gaussians(n, W, H, 51)
    rect, cnt = oracle.rect_rule(means, chol, color, W, H, T)
    G = np.random.default_rng(9).standard_normal((H, W, 3))
    gr = oracle.backward(means, chol, color, rect, cnt, W, H, T, G)
    for k in ("means", "chol", "color"):
        assert np.all(gr["abs"][k] >= np.abs(gr[k]) * (1 - 1e-12))
    chol1 = chol.copy()
    chol1[:, 1] = 0.0
    G1 = np.zeros((H, W, 3))
    G1[17, 21, :] = [0.3, -0.2, 0.7]
    gr1 = oracle.backward(means, chol1, color, rect, cnt, W, H, T, G1)
    for k in ("means", "chol", "color"):
        np.testing.assert_allclose(gr1["abs"][k], np.abs(gr1[k]), rtol=1e-12, atol=1e-300)
