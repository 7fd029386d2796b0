"""Pins of the alpha-blending and opacity oracle (Eq. 3-5, Table 3's "w/o AR"
and "w/o M"): a per-pixel brute force written separately, closed forms of
one and two Gaussians, the accumulated sum as the small-opacity limit, and
central finite differences of the FP64 loss in every parameter."""
import numpy as np
import pytest

import oracle
import synth

A_MIN, A_MAX, T_MIN = oracle.BLEND_THRESHOLDS


def brute_blend(means, chol, color, opac, rect, cnt, W, H, T, th=oracle.BLEND_THRESHOLDS):
    """Every Gaussian in ascending index whose rect covers the pixel's tile,
    Sigma^-1 by numpy's matrix inverse of L L^T; 3D GS's rules in FP64."""
    a_min, a_max, t_min = th
    out = np.zeros((H, W, 3))
    inv = []
    for g in range(means.shape[0]):
        L = np.array([[chol[g, 0], 0.0], [chol[g, 1], chol[g, 2]]], np.float64)
        inv.append(np.linalg.inv(L @ L.T))
    for y in range(H):
        for x in range(W):
            tx, ty = x // T, y // T
            Tr, c = 1.0, np.zeros(3)
            for g in range(means.shape[0]):
                r = rect[g]
                if cnt[g] == 0 or not (r[0] <= tx < r[2] and r[1] <= ty < r[3]):
                    continue
                d = np.array([x + 0.5, y + 0.5]) - means[g].astype(np.float64)
                a = float(opac[g]) * np.exp(-0.5 * d @ inv[g] @ d)
                if a < a_min:
                    continue
                a = min(a, a_max)
                if Tr * (1 - a) < t_min:
                    break
                c += color[g].astype(np.float64) * a * Tr
                Tr *= 1 - a
            out[y, x] = c
    return out


def small_case(seed, n=14, W=24, H=20, T=8):
    means, chol, color = synth.init_gaussians(n, W, H, seed)
    logit = np.random.default_rng(seed).normal(0.5, 1.5, n)
    return means, chol, color, logit, W, H, T


def test_blend_render_matches_brute_force():
    for seed in (1, 2, 3):
        means, chol, color, logit, W, H, T = small_case(seed)
        o = oracle.sigmoid_opacity(logit)
        rect, cnt = oracle.rect_rule(means, chol, color, W, H, T)
        ids, ranges, _ = oracle.bin_tiles(rect, cnt, W, H, T)
        out, tf, nl, amb = oracle.blend_render(means, chol, color, o, ids, ranges, W, H, T)
        ref = brute_blend(means, chol, color, o, rect, cnt, W, H, T)
        ok = ~amb
        np.testing.assert_allclose(out[ok], ref[ok], rtol=1e-12, atol=1e-14)
        assert np.all(tf >= T_MIN) and np.all(tf <= 1.0)


def test_blend_one_and_two_gaussians_closed_forms():
    W, H, T = 16, 16, 16
    means = np.array([[8.0, 8.0], [8.0, 8.0]], np.float32)
    chol = np.array([[3.0, 0.0, 3.0], [3.0, 0.0, 3.0]], np.float32)
    color = np.array([[0.6, 0.2, 0.1], [0.1, 0.5, 0.9]], np.float32)
    opac = np.array([0.7, 0.4], np.float32)
    rect, cnt = oracle.rect_rule(means, chol, color, W, H, T)
    ids, ranges, _ = oracle.bin_tiles(rect, cnt, W, H, T)
    # one Gaussian: C = c o w
    out1, tf1, _, _ = oracle.blend_render(means[:1], chol[:1], color[:1], opac[:1], ids[ids == 0], np.array(
        [[0, 1]], np.int32), W, H, T)
    d2 = ((np.arange(W) + 0.5 - 8.0)[None, :] ** 2 + (np.arange(H) + 0.5 - 8.0)[:, None] ** 2)
    w = np.exp(-0.5 * d2 / 9.0)
    a1 = 0.7 * w
    keep = a1 >= A_MIN
    np.testing.assert_allclose(out1, np.where(keep, a1, 0.0)[..., None] * color[0].astype(np.float64),
                               rtol=1e-6)
    # two: C = c1 a1 + c2 a2 (1 - a1)
    out2, tf2, _, _ = oracle.blend_render(means, chol, color, opac, ids, ranges, W, H, T)
    a2 = 0.4 * w
    ref = (np.where(keep, a1, 0)[..., None] * color[0].astype(np.float64)
           + np.where(a2 >= A_MIN, a2 * (1 - np.where(keep, a1, 0)), 0)[..., None] * color[1].astype(np.float64))
    np.testing.assert_allclose(out2, ref, rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(tf2, (1 - np.where(keep, a1, 0)) * (1 - np.where(a2 >= A_MIN, a2, 0)), rtol=1e-6)


def test_blend_small_opacity_approaches_the_accumulated_sum():
    """Without thresholds and with opacities ~1e-3 the blended image differs
    from the accumulated sum sum c o w by at most sum_n |c_n| a_n sum_{m<n} a_m
    (first order in alpha) at every pixel."""
    W, H, T, n = 32, 32, 16, 40
    means, chol, color = synth.init_gaussians(n, W, H, 9)
    opac = np.full(n, 1e-3, np.float32)
    rect, cnt = oracle.rect_rule(means, chol, color, W, H, T)
    ids, ranges, _ = oracle.bin_tiles(rect, cnt, W, H, T)
    out, _, _, _ = oracle.blend_render(means, chol, color, opac, ids, ranges, W, H, T, thresholds=(0.0, 1.0, 0.0))
    acc = oracle.render(means, chol, (color * opac[:, None]).astype(np.float32), ids, ranges, W, H, T)
    # bound: a_n <= 1e-3, sum over at most n Gaussians
    bound = np.abs(color).max() * 1e-3 * 1e-3 * n * n
    assert np.abs(out - acc).max() <= bound
    assert np.abs(out - acc).max() > 0.0


def fd_check(loss_at, params, analytic, idxs, h):
    """Richardson-extrapolated central differences (steps h and h/2)."""
    for idx in idxs:
        def central(s):
            a, b = params.copy(), params.copy()
            a[idx] += s
            b[idx] -= s
            return (loss_at(a) - loss_at(b)) / (2 * s)
        num = (4 * central(h / 2) - central(h)) / 3
        assert num == pytest.approx(analytic[idx], rel=2e-4, abs=2e-9), idx


@pytest.mark.parametrize("thresholds", [(0.0, 0.99, 0.0), oracle.BLEND_THRESHOLDS])
def test_blend_gradients_match_finite_differences(thresholds):
    """Central differences of the FP64 loss with the tile lists frozen, in
    the position, Cholesky vector, colour and opacity logit of several
    Gaussians. The skip and stop thresholds make the loss jump where a
    decision flips, so the geometric and opacity differences run without
    them (the 0.99 clamp only bends the loss); with 3D GS's thresholds the
    colour, which decides nothing, is differenced."""
    means, chol, color, logit, W, H, T = small_case(5, n=10, W=20, H=16, T=8)
    target = synth.image(W, H, 5, n_blobs=3)
    r = oracle.blend_forward_backward(means, chol, color, logit, target, T, thresholds)
    ids, ranges = r["ids"], r["ranges"]
    g = r["grads"]
    live = np.nonzero(r["cnt"] > 0)[0][:6]

    def loss_of(m, l, c, lg):
        o = 1.0 / (1.0 + np.exp(-np.asarray(lg, np.float64)))
        out, _, _, _ = oracle.blend_render(m, l, c, np.asarray(o, np.float32), ids, ranges, W, H, T, thresholds)
        return float(((out - target.astype(np.float64)) ** 2).mean())

    if thresholds == oracle.BLEND_THRESHOLDS:
        assert r["n_last"].min() < r["n_last"].max()
        fd_check(lambda p: loss_of(means, chol, p.astype(np.float32), logit), color.astype(np.float64),
                 g["color"], [(i, k) for i in live for k in range(3)], 2.0 ** -6)
        return

    # means, chol, colour are FP32 in the render: power-of-two steps keep the
    # perturbed inputs exact
    fd_check(lambda p: loss_of(p.astype(np.float32), chol, color, logit), means.astype(np.float64), g["means"],
             [(i, k) for i in live for k in range(2)], 2.0 ** -6)
    fd_check(lambda p: loss_of(means, p.astype(np.float32), color, logit), chol.astype(np.float64), g["chol"],
             [(i, k) for i in live for k in range(3)], 2.0 ** -6)
    fd_check(lambda p: loss_of(means, chol, p.astype(np.float32), logit), color.astype(np.float64), g["color"],
             [(i, k) for i in live for k in range(3)], 2.0 ** -6)
    fd_check(lambda p: loss_of(means, chol, color, p), logit.astype(np.float64), g["logit"],
             [(i,) for i in live], 1e-2)


def test_opacity_form_gradients_match_finite_differences():
    """Accumulated summation with separate opacity: central differences in
    colour and opacity logit."""
    means, chol, color, logit, W, H, T = small_case(6, n=10, W=20, H=16, T=8)
    target = synth.image(W, H, 6, n_blobs=3)
    r = oracle.opacity_forward_backward(means, chol, color, logit, target, T)
    ids, ranges = r["ids"], r["ranges"]
    live = np.nonzero(r["cnt"] > 0)[0][:6]

    def loss_of(c, lg):
        o = 1.0 / (1.0 + np.exp(-np.asarray(lg, np.float64)))
        cp = (np.asarray(c, np.float64) * o[:, None]).astype(np.float32)
        out = oracle.render(means, chol, cp, ids, ranges, W, H, T)
        return float(((out - target.astype(np.float64)) ** 2).mean())

    go = r["grads_opacity"]
    fd_check(lambda p: loss_of(p, logit), color.astype(np.float64), go["color"],
             [(i, k) for i in live for k in range(3)], 1e-3)
    fd_check(lambda p: loss_of(color, p), logit.astype(np.float64), go["logit"], [(i,) for i in live], 2e-2)
