"""Pins of the codec fine-tuning oracle (Sec. 3.3, Sec. 3.4) against
definitions computed another way: struct's half-precision packing, brute
force over the quantiser grid and the codebook, finite differences of the
straight-through surrogate, closed forms of the EMA update."""
import struct

import numpy as np
import pytest

import oracle
import synth


def test_fp16_round_matches_struct_half_packing():
    gen = np.random.default_rng(1)
    x = np.concatenate([gen.uniform(0, 2048, 500), gen.uniform(-3, 3, 500), [0.5, 1024.5, 2049.0, 4097.0]])
    x = x.astype(np.float32)
    ref = np.array([struct.unpack("<e", struct.pack("<e", float(v)))[0] for v in x], np.float32)
    np.testing.assert_array_equal(oracle.fp16_round(x), ref)


def test_lsq_is_the_nearest_grid_point():
    """l_bar is the grid point beta + k gamma (k = 0 .. 2^b - 1) nearest to
    l, found by brute force in FP64 (points within 1e-4 of a midpoint are
    skipped: there FP32 rounding of x decides); outside the range the end
    points; codes are k."""
    bits = 6
    gen = np.random.default_rng(2)
    gamma = np.array([0.11, 0.07, 0.13], np.float32)
    beta = np.array([0.5, -2.0, 0.4], np.float32)
    l = np.stack([gen.uniform(-1, 9, 4000), gen.uniform(-4, 4, 4000), gen.uniform(-1, 10, 4000)], axis=1)
    l = l.astype(np.float32)
    lbar, x, q = oracle.lsq_fake_quant(l, gamma, beta, bits)
    k = np.arange(2 ** bits, dtype=np.float64)
    for i in range(3):
        grid = beta[i].astype(np.float64) + k * gamma[i].astype(np.float64)
        dist = np.abs(l[:, i].astype(np.float64)[:, None] - grid[None, :])
        kk = np.argmin(dist, axis=1)
        srt = np.sort(dist, axis=1)
        clear = (srt[:, 1] - srt[:, 0]) > 1e-4 * gamma[i]
        assert clear.mean() > 0.99
        np.testing.assert_array_equal(q[clear, i], kk[clear].astype(np.float32))
        np.testing.assert_allclose(lbar[clear, i], grid[kk[clear]], rtol=0, atol=4e-7 * np.abs(grid).max())
        lo = l[:, i] < beta[i]
        hi = l[:, i] > beta[i] + (2 ** bits - 1) * gamma[i] * 1.0001
        assert lo.any() and hi.any()
        np.testing.assert_array_equal(q[lo, i], 0.0)
        np.testing.assert_array_equal(q[hi, i], float(2 ** bits - 1))


def test_lsq_grid_points_are_fixed_points():
    gamma = np.array([0.25, 0.125, 0.5], np.float32)  # powers of two: the grid is exact in FP32
    beta = np.array([0.5, -4.0, 1.0], np.float32)
    k = np.arange(64, dtype=np.float32)
    l = np.stack([beta[i] + k * gamma[i] for i in range(3)], axis=1).astype(np.float32)
    lbar, x, q = oracle.lsq_fake_quant(l, gamma, beta, 6)
    np.testing.assert_array_equal(lbar, l)
    np.testing.assert_array_equal(q, np.stack([k] * 3, axis=1))
    np.testing.assert_array_equal(x, q)


def test_lsq_ste_gradients_are_the_surrogates_derivatives():
    """With the rounding offset delta = code - clamp(x) frozen, the surrogate
    f(l, gamma, beta) = gamma (clamp((l - beta)/gamma, 0, 2^b - 1) + delta)
    + beta is smooth; central differences of sum g f in FP64 equal
    lsq_ste_grads, inside, below and above the range."""
    bits = 6
    qp = 2 ** bits - 1
    gen = np.random.default_rng(3)
    n = 40
    gamma = np.array([0.1, 0.05, 0.2])
    beta = np.array([0.3, -1.0, 0.2])
    l = np.stack([gen.uniform(-0.5, 7.5, n), gen.uniform(-2, 2.5, n), gen.uniform(-0.5, 14, n)], axis=1)
    g = gen.normal(size=(n, 3))
    lbar, x, q = oracle.lsq_fake_quant(l, gamma, beta, bits)
    x64 = (l - beta) / gamma
    delta = q.astype(np.float64) - np.clip(x64, 0, qp)

    def F(l_, gm, bt):
        return float((g * (gm * (np.clip((l_ - bt) / gm, 0, qp) + delta) + bt)).sum())

    g_l, g_gamma, g_beta = oracle.lsq_ste_grads(g, x, q, bits)
    h = 1e-7
    assert ((x < 0).any() and (x > qp).any() and ((x > 0) & (x < qp)).any())
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        num_g = (F(l, gamma + e, beta) - F(l, gamma - e, beta)) / (2 * h)
        num_b = (F(l, gamma, beta + e) - F(l, gamma, beta - e)) / (2 * h)
        assert num_g == pytest.approx(g_gamma[i], rel=1e-5, abs=1e-6)
        assert num_b == pytest.approx(g_beta[i], rel=1e-5, abs=1e-6)
    far = np.abs(x64 - np.clip(x64, 0, qp)) > 1e-3
    far |= (x64 > 1e-3) & (x64 < qp - 1e-3)
    for idx in zip(*np.nonzero(far)):
        dl = np.zeros_like(l)
        dl[idx] = h
        num = (F(l + dl, gamma, beta) - F(l - dl, gamma, beta)) / (2 * h)
        assert num == pytest.approx(g_l[idx], rel=1e-5, abs=1e-6)


def test_rvq_assign_is_the_nearest_entry():
    """Stage 1 picks the brute-force nearest codebook entry (FP64 distances,
    clear margins); stage 2 quantises the FP32 residual c' - C^1[i^1]; the
    result agrees with the FP64 greedy encoder away from near-ties."""
    gen = np.random.default_rng(4)
    cb = synth.codebooks(4, size=8, stages=2)[1]
    c = gen.uniform(-0.3, 0.6, size=(3000, 3)).astype(np.float32)
    idx, chat, r_in = oracle.rvq_assign_f32(c, cb)
    d1 = ((c.astype(np.float64)[:, None, :] - cb[0].astype(np.float64)[None]) ** 2).sum(-1)
    srt = np.sort(d1, axis=1)
    clear = srt[:, 1] - srt[:, 0] > 1e-5
    np.testing.assert_array_equal(idx[0][clear], np.argmin(d1, axis=1)[clear])
    np.testing.assert_array_equal(r_in[0], c)
    np.testing.assert_array_equal(r_in[1], (c - cb[0][idx[0]]).astype(np.float32))
    ref = oracle.rvq_encode(c, cb)
    assert (ref == idx).all(axis=0).mean() > 0.99
    np.testing.assert_allclose(chat, cb[0][idx[0]].astype(np.float64) + cb[1][idx[1]], rtol=0, atol=1e-7)


def test_rvq_ties_take_the_lowest_index():
    cb = np.zeros((1, 8, 3), np.float32)
    cb[0, 3] = [1, 0, 0]
    cb[0, 5] = [1, 0, 0]
    cb[0, 6] = [0, 1, 0]
    c = np.array([[1, 0, 0], [0.5, 0.5, 0], [0, 0, 0]], np.float32)
    idx, _, _ = oracle.rvq_assign_f32(c, cb)
    np.testing.assert_array_equal(idx[0], [3, 0, 0])


def test_commitment_loss_closed_forms():
    """Colours that are stage-1 entries, with a zero vector in the stage-2
    codebook, give L_c = 0; one Gaussian against a one-entry-per-stage
    codebook gives the hand-computed value."""
    gen = np.random.default_rng(5)
    cb = gen.uniform(-1, 1, size=(2, 8, 3)).astype(np.float32)
    cb[1, 4] = 0.0
    c = cb[0][gen.integers(0, 8, 50)]
    idx, chat, r_in = oracle.rvq_assign_f32(c, cb)
    assert oracle.commitment_loss(r_in, cb, idx) == 0.0
    np.testing.assert_array_equal(chat, c)
    cb1 = np.zeros((2, 1, 3), np.float32)
    cb1[0, 0] = [1, 2, 3]
    cb1[1, 0] = [0.5, 0.5, 0.5]
    c1 = np.array([[2, 2, 2]], np.float32)
    idx1, _, r1 = oracle.rvq_assign_f32(c1, cb1)
    # stage 1: (2,2,2) - (1,2,3) = (1,0,-1), |.|^2 = 2; stage 2: (1,0,-1) - 0.5 -> 0.25 + 0.25 + 2.25
    assert oracle.commitment_loss(r1, cb1, idx1) == pytest.approx((2.0 + 2.75) / 1.0)


def test_ema_update_closed_forms():
    """decay 0, eps 0: every entry with assignments becomes the mean of its
    residuals (brute force per entry); Laplace smoothing keeps the total
    count; an entry with no assignments keeps its vector at eps 0; repeated
    updates on the same assignment converge to the cluster means."""
    gen = np.random.default_rng(6)
    M, Bn, n = 2, 8, 500
    idx = np.stack([gen.integers(0, Bn - 1, n), gen.integers(0, Bn, n)])  # stage-1 entry 7 unused
    r_in = gen.normal(size=(M, n, 3))
    count0 = np.ones((M, Bn))
    total0 = gen.normal(size=(M, Bn, 3))
    cnt, tot, cb = oracle.ema_codebook_update(count0, total0, idx, r_in, 0.0, 0.0)
    for m in range(M):
        for j in range(Bn):
            sel = idx[m] == j
            if sel.any():
                np.testing.assert_allclose(cb[m, j], r_in[m][sel].mean(axis=0), rtol=1e-12, atol=1e-12)
    cnt, tot, cb = oracle.ema_codebook_update(count0, total0, idx, r_in, 0.9, 0.0)
    np.testing.assert_allclose(cb[0, 7], total0[0, 7] / count0[0, 7], rtol=1e-12)
    cnt, tot, cb = oracle.ema_codebook_update(count0, total0, idx, r_in, 0.9, 1e-3)
    np.testing.assert_allclose(cnt.sum(axis=1), 0.9 * count0.sum(axis=1) + 0.1 * n, rtol=1e-12)
    c, t = count0, total0
    for _ in range(400):
        c, t, cb = oracle.ema_codebook_update(c, t, idx, r_in, 0.95, 1e-5)
    for m in range(M):
        for j in range(Bn):
            sel = idx[m] == j
            if sel.any():
                np.testing.assert_allclose(cb[m, j], r_in[m][sel].mean(axis=0), rtol=1e-3, atol=1e-6)


def test_codec_pass_with_identity_quantisers_is_the_plain_pass():
    """Positions representable in FP16, Cholesky entries on the quantiser
    grid and colours equal to stage-1 entries (zero stage-2 entry): the
    fine-tuning pass renders and differentiates exactly like the plain one,
    and the quantiser gradients vanish (on the grid, code - x = 0, and
    nothing is clamped)."""
    W, H, T, n = 40, 32, 8, 30
    gen = np.random.default_rng(7)
    means = (gen.integers(0, 4 * W, size=(n, 2)) / 4.0).astype(np.float32)
    means[:, 1] = np.minimum(means[:, 1], H - 0.25)
    gamma = np.array([0.125, 0.0625, 0.125], np.float32)
    beta = np.array([1.0, -2.0, 1.0], np.float32)
    k = gen.integers(0, 64, size=(n, 3))
    chol = (beta + k * gamma).astype(np.float32)
    cb = gen.uniform(0, 0.2, size=(2, 8, 3)).astype(np.float32)
    cb[1, 2] = 0.0
    color = cb[0][gen.integers(0, 8, n)]
    target = synth.image(W, H, 7, n_blobs=4)
    r = oracle.codec_forward_backward(means, chol, color, gamma, beta, cb, 6, target, T)
    p = oracle.forward_backward(means, chol, color, target, T)
    np.testing.assert_array_equal(r["out"], p["out"])
    for key in ("means", "color"):
        np.testing.assert_array_equal(r["codec"]["grads"][key], p["grads"][key])
    np.testing.assert_array_equal(r["codec"]["grads"]["chol"], p["grads"]["chol"])
    np.testing.assert_array_equal(r["codec"]["codes"], k.astype(np.uint8))
    assert r["codec"]["commit"] == 0.0
    np.testing.assert_array_equal(r["codec"]["grads"]["gamma"], 0.0)
    np.testing.assert_array_equal(r["codec"]["grads"]["beta"], 0.0)


def test_codec_gamma_beta_gradients_match_finite_differences():
    """Central differences of the render's FP64 loss in gamma and beta with
    the rounding offsets and the tile support frozen, against the chained
    gradients of codec_forward_backward."""
    W, H, T, n = 24, 20, 8, 8
    means, chol, color = synth.init_gaussians(n, W, H, 8)
    gamma = np.array([0.12, 0.06, 0.12], np.float32)
    beta = np.array([0.9, -1.9, 0.9], np.float32)
    cb = synth.codebooks(8, size=8, stages=2)[1]
    target = synth.image(W, H, 8, n_blobs=3)
    r = oracle.codec_forward_backward(means, chol, color, gamma, beta, cb, 6, target, T)
    cdc = r["codec"]
    x64 = (chol.astype(np.float64) - beta.astype(np.float64)) / gamma.astype(np.float64)
    delta = cdc["codes"].astype(np.float64) - np.clip(x64, 0, 63)
    ids, ranges = r["ids"], r["ranges"]

    def loss_at(gm, bt):
        lq = gm * (np.clip((chol - bt) / gm, 0, 63) + delta) + bt
        out = oracle.render(cdc["means16"], lq.astype(np.float32), cdc["color_q"], ids, ranges, W, H, T)
        return oracle.loss(out, target)[0]

    g64, b64 = gamma.astype(np.float64), beta.astype(np.float64)
    for i in range(3):
        e = np.zeros(3)
        e[i] = 1e-3

        def central(h, which):
            d = e * h / 1e-3
            if which == "g":
                return (loss_at(g64 + d, b64) - loss_at(g64 - d, b64)) / (2 * h)
            return (loss_at(g64, b64 + d) - loss_at(g64, b64 - d)) / (2 * h)
        for which, ana in (("g", cdc["grads"]["gamma"][i]), ("b", cdc["grads"]["beta"][i])):
            num = (4 * central(5e-4, which) - central(1e-3, which)) / 3
            assert num == pytest.approx(ana, rel=2e-3, abs=1e-5 * max(1.0, abs(ana)))


def test_codec_decode_reproduces_what_the_quantisers_render():
    """Decoding the codes, indices and FP16 positions that the quantisers
    produce gives back exactly the positions, Cholesky vectors and colours
    they handed to the render (Eq. 9's reconstruction, Eq. 10's sum)."""
    gen = np.random.default_rng(9)
    n = 500
    means = gen.uniform(0, 700, size=(n, 2)).astype(np.float32)
    chol = np.stack([gen.uniform(0.5, 9, n), gen.uniform(-3, 3, n), gen.uniform(0.5, 9, n)], axis=1).astype(np.float32)
    color = gen.uniform(-0.1, 0.6, size=(n, 3)).astype(np.float32)
    gamma = np.array([0.13, 0.09, 0.14], np.float32)
    beta = np.array([0.5, -3.0, 0.5], np.float32)
    cb = synth.codebooks(9, size=8, stages=2)[1]
    lbar, x, q = oracle.lsq_fake_quant(chol, gamma, beta, 6)
    idx, chat, _ = oracle.rvq_assign_f32(color, cb)
    m16 = means.astype(np.float16)
    codes = np.zeros((n, 4), np.uint8)
    codes[:, :3] = q.astype(np.uint8)
    dm, dl, dc = oracle.codec_decode(m16.view(np.uint16), codes, gamma, beta, idx, cb)
    np.testing.assert_array_equal(dm, oracle.fp16_round(means))
    np.testing.assert_array_equal(dl, lbar)
    np.testing.assert_array_equal(dc, chat)
