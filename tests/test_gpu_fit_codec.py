"""GPU codec fine-tuning (Sec. 3.3-3.4) against the oracle. At every step
the oracle is evaluated at the GPU's own state (parameters, gamma, beta,
codebooks, EMA sums, optimiser moments), so each step is checked exactly:
quantiser codes and RVQ indices bit for bit (both sides decide in FP32),
loss, straight-through gradients, dL/dgamma, dL/dbeta, the commitment loss,
the EMA codebook update and the optimiser updates within tolerance."""
import numpy as np
import pytest

import oracle
import synth
import tolerances

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BITS = 6


@pytest.fixture(scope="module")
def gi():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_08551_gb300 as m
    m.load()
    return m


def check_grads(g_gpu, g_ref, g_abs, t):
    return tolerances.check_grads(g_gpu, g_ref, g_abs, f"step {t}")


def oracle_step(pg, gb, cb, target, T, paper):
    """Oracle pass at the GPU's state; returns the codec dict, loss, the
    gradients in the fit's parameter space and their condition magnitudes."""
    H, W, _ = target.shape
    if paper:
        means, chol, dmu = oracle.paper_formation(pg[:, 0:2], pg[:, 2:5].astype(np.float32), W, H)
    else:
        means, chol, dmu = pg[:, 0:2].astype(np.float32), pg[:, 2:5].astype(np.float32), np.ones((pg.shape[0], 2))
    r = oracle.codec_forward_backward(means, chol, pg[:, 5:8].astype(np.float32), gb[0:3], gb[3:6], cb, BITS,
                                      target, T)
    c = r["codec"]
    g = c["grads"]
    g_ref = np.concatenate([g["means"] * dmu, g["chol"], g["color"]], axis=1)
    a = r["grads"]["abs"]
    g_abs = np.concatenate([a["means"] * np.abs(dmu), a["chol"], a["color"]], axis=1)
    c["g_lbar"] = r["grads"]["chol"]  # dL/d(quantised Cholesky), before the straight-through mask
    return c, r["loss"], g_ref, g_abs


def run_codec(gi, target, p0, T, steps, paper, optimizer, lr, decay=0.9, size=8, stages=2):
    H, W, _ = target.shape
    n = p0.shape[0]
    pt = torch.from_numpy(p0).cuda()
    spec = gi.codec_init(pt, bits=BITS, stages=stages, size=size, param_mode="paper" if paper else "pixel")
    spec["ema_decay"] = decay
    fit = gi.Fit([torch.from_numpy(target).cuda()], [pt], tile=T, lr=lr, param_mode="paper" if paper else "pixel",
                 optimizer=optimizer, codec=spec)
    lrv = np.tile(np.array([lr[0]] * 2 + [lr[1]] * 3 + [lr[2]] * 3), (n, 1))
    adan = optimizer == "adan"
    for t in range(1, steps + 1):
        pg = fit.params.cpu().numpy().astype(np.float64)
        views = (fit.adam_m, fit.adam_v) + ((fit.adan_n, fit.adan_gprev) if adan else ())
        state = tuple(x.cpu().numpy().astype(np.float64) for x in views)
        gbs = fit.codec_gb.cpu().numpy().astype(np.float64)
        cb = fit.codebooks.cpu().numpy()
        cnt0 = fit.ema_count.cpu().numpy()
        tot0 = fit.ema_total.cpu().numpy()
        c, loss, g_ref, g_abs = oracle_step(pg, gbs[0].astype(np.float32), cb, target, T, paper)
        fit.step(1)
        torch.cuda.synchronize()
        # integer decisions: bit for bit
        np.testing.assert_array_equal(fit.codes.cpu().numpy()[:, :3], c["codes"])
        np.testing.assert_array_equal(fit.rvq_idx.cpu().numpy().astype(np.int64), c["idx"])
        assert fit.mse()[0] == pytest.approx(loss, rel=1e-5)
        tol_g = check_grads(fit.grads.cpu().numpy().astype(np.float64), g_ref, g_abs, t)
        out = fit.codec_out.cpu().numpy()
        assert out[0] == pytest.approx(c["commit"], rel=1e-5)
        # dL/dgamma, dL/dbeta: each term's gradient is within tol_g, summed
        x, q = c["x"].astype(np.float64), c["codes"].astype(np.float64)
        qp = 2 ** BITS - 1
        inside = (x >= 0) & (x <= qp)
        w_g = np.where(inside, np.abs(q - np.where(inside, x, 0)), np.where(x > qp, qp, 0.0))
        w_b = np.where(inside, 0.0, 1.0)
        g_full = c["g_lbar"]
        for i in range(3):
            tg = (tol_g[:, 2 + i] * w_g[:, i]).sum() + 1e-6 * np.abs(g_full[:, i] * w_g[:, i]).sum() + 1e-12
            tb = (tol_g[:, 2 + i] * w_b[:, i]).sum() + 1e-6 * np.abs(g_full[:, i] * w_b[:, i]).sum() + 1e-12
            assert abs(out[1 + i] - c["grads"]["gamma"][i]) <= tg, f"step {t}: dL/dgamma_{i}"
            assert abs(out[4 + i] - c["grads"]["beta"][i]) <= tb, f"step {t}: dL/dbeta_{i}"
        # EMA codebook update from the GPU's previous sums and this step's indices
        # the decay and eps the context holds (FP32 values)
        cnt, tot, cb_ref = oracle.ema_codebook_update(cnt0, tot0, c["idx"], c["r_in"], fit.codec["ema_decay"],
                                                      fit.codec["ema_eps"])
        np.testing.assert_allclose(fit.ema_count.cpu().numpy(), cnt, rtol=1e-9)
        scale = np.abs(tot).max()
        np.testing.assert_allclose(fit.ema_total.cpu().numpy(), tot, rtol=1e-5, atol=1e-6 * scale)
        np.testing.assert_allclose(fit.codebooks.cpu().numpy(), cb_ref, rtol=1e-5, atol=1e-6 * np.abs(cb_ref).max())
        # optimiser updates of the Gaussians and of gamma, beta
        lr_c = np.full(6, lr[1])
        g_gb = np.concatenate([out[1:4], out[4:7]])
        if adan:
            p_ref, _ = oracle.adan(pg, g_ref, state, t, lrv)
            gb_ref, _ = oracle.adan(gbs[0], g_gb, (gbs[1], gbs[2], gbs[3], gbs[4]), t, lr_c)
        else:
            p_ref, _, _ = oracle.adam(pg, g_ref, state[0], state[1], t, lrv)
            gb_ref, _, _ = oracle.adam(gbs[0], g_gb, gbs[1], gbs[2], t, lr_c)
        p_new = fit.params.cpu().numpy().astype(np.float64)
        close = np.abs(p_new - p_ref) <= 1e-5 * np.maximum(np.abs(p_ref), 1.0) + 1e-3 * lrv
        assert close.mean() > 0.999, f"step {t}: {np.sum(~close)} parameters off the oracle's update"
        bound = (4 if adan else 2) * lrv
        assert np.all(np.abs(p_new - p_ref) <= bound + 1e-5 * np.maximum(np.abs(p_ref), 1.0))
        gb_new = fit.codec_gb.cpu().numpy()[0].astype(np.float64)
        np.testing.assert_allclose(gb_new, gb_ref, rtol=1e-5, atol=1e-3 * lr[1])
    assert int(fit.step_count.item()) == steps
    return fit


@pytest.mark.parametrize("T", [8, 16, 32])
def test_codec_pixel_adam_steps_track_oracle(gi, T):
    W, H, n = 128, 96, 800
    target = synth.image(W, H, 41, n_blobs=20)
    p0 = np.concatenate(synth.init_gaussians(n, W, H, 41), axis=1).astype(np.float32)
    run_codec(gi, target, p0, T, 5, paper=False, optimizer="adam", lr=(1e-3, 1e-2, 1e-2)).close()


@pytest.mark.parametrize("stages,size", [(2, 256), (3, 64)])
def test_codec_large_codebooks_track_oracle(gi, stages, size):
    """Codebooks beyond the paper's 8 entries (the sums of every entry go
    through the reduction's dynamic shared memory): 2 x 256 and 3 x 64."""
    W, H, T, n = 128, 96, 16, 2000
    target = synth.image(W, H, 45, n_blobs=20)
    p0 = np.concatenate(synth.init_gaussians(n, W, H, 45), axis=1).astype(np.float32)
    run_codec(gi, target, p0, T, 3, paper=False, optimizer="adam", lr=(1e-3, 1e-2, 1e-2), size=size,
              stages=stages).close()


def paper_params(means, chol, color, W, H):
    theta = np.arctanh(np.clip(means.astype(np.float64) / [W, H] * 2 - 1, -0.999, 0.999))
    c = chol.astype(np.float32).copy()
    c[:, 0] -= 0.5
    c[:, 2] -= 0.5
    return np.concatenate([theta, c, color], axis=1).astype(np.float32)


def test_codec_paper_adan_steps_track_oracle(gi):
    W, H, T, n = 160, 112, 16, 1200
    target = synth.image(W, H, 42, n_blobs=24)
    p0 = paper_params(*synth.init_gaussians(n, W, H, 42), W, H)
    run_codec(gi, target, p0, T, 5, paper=True, optimizer="adan", lr=(1e-3, 1e-3, 1e-3)).close()


@pytest.mark.slow
def test_codec_paper_adan_full_size(gi):
    """The 768x512, 70k-Gaussian workload fine-tuned with the paper's codec
    (b = 6, M = 2, B = 8) and optimiser, first five steps."""
    w = synth.workload("c1_768x512_70k")
    p0 = paper_params(w.means, w.chol, w.color, w.W, w.H)
    run_codec(gi, w.target, p0, 16, 5, paper=True, optimizer="adan", lr=(1e-3, 1e-3, 1e-3)).close()


def test_codec_render_is_the_decoded_image(gi):
    """fit.render() in codec mode renders what the codes decode to: the
    plain renderer on FP16 positions, code * gamma + beta and the summed
    codebook entries gives the same image bit for bit."""
    W, H, T, n = 96, 64, 16, 500
    target = synth.image(W, H, 43, n_blobs=10)
    p0 = np.concatenate(synth.init_gaussians(n, W, H, 43), axis=1).astype(np.float32)
    pt = torch.from_numpy(p0).cuda()
    spec = gi.codec_init(pt)
    fit = gi.Fit([torch.from_numpy(target).cuda()], [pt], tile=T, codec=spec, render_split=8)
    fit.step(3)
    fit.render()
    torch.cuda.synchronize()
    codes = fit.codes.cpu().numpy()[:, :3].astype(np.float32)
    gbv = fit.codec_gb.cpu().numpy()[0]
    chol = (codes * gbv[0:3] + gbv[3:6]).astype(np.float32)
    idx = fit.rvq_idx.cpu().numpy().astype(np.int64)
    cb = fit.codebooks.cpu().numpy()
    # the codebooks moved after the last step's assignment; re-render with the
    # indices the render pass itself chose
    color = (cb[0][idx[0]].astype(np.float64) + cb[1][idx[1]]).astype(np.float32)
    means = oracle.fp16_round(fit.params.cpu().numpy()[:, 0:2])
    img = gi.rasterize(torch.from_numpy(means).cuda(), torch.from_numpy(chol).cuda(),
                       torch.from_numpy(color).cuda(), W, H, T)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(fit.images()[0].cpu().numpy(), img.cpu().numpy())
    fit.close()


def test_codec_arguments_are_validated(gi):
    W, H, n = 64, 64, 100
    target = torch.from_numpy(synth.image(W, H, 44, n_blobs=4)).cuda()
    p0 = torch.from_numpy(np.concatenate(synth.init_gaussians(n, W, H, 44), axis=1).astype(np.float32)).cuda()
    spec = gi.codec_init(p0)
    for bad in ({"bits": 9}, {"gamma": [0.0, 1.0, 1.0]}, {"ema_decay": 1.0}):
        s = dict(spec)
        s.update(bad)
        with pytest.raises(gi.GIError):
            gi.Fit([target], [p0], tile=16, codec=s)
    with pytest.raises(gi.GIError):
        gi.Fit([target], [p0], tile=16, codec=spec, cov="rs")


def test_codec_decode_bit_exact(gi):
    """gi_codec_decode against the oracle on random streams (two and three
    stages), including the bounds check of an index outside the codebook."""
    gen = np.random.default_rng(45)
    for n, M, Bn in ((5000, 2, 8), (3000, 3, 16)):
        m16 = gen.uniform(0, 2000, size=(n, 2)).astype(np.float16)
        codes = gen.integers(0, 64, size=(n, 4)).astype(np.uint8)
        gb = [0.13, 0.07, 0.11, 0.6, -2.5, 0.4]
        idx = gen.integers(0, Bn, size=(M, n)).astype(np.uint8)
        cb = gen.uniform(-0.3, 0.5, size=(M, Bn, 3)).astype(np.float32)
        stream = {"means16": torch.from_numpy(m16.view(np.int16)).cuda(), "codes": torch.from_numpy(codes).cuda(),
                  "gamma_beta": gb, "idx": torch.from_numpy(idx).cuda(), "codebooks": torch.from_numpy(cb).cuda()}
        means, chol, color = gi.codec_decode(stream)
        torch.cuda.synchronize()
        rm, rl, rc = oracle.codec_decode(m16, codes, gb[0:3], gb[3:6], idx, cb)
        np.testing.assert_array_equal(means.cpu().numpy(), rm)
        np.testing.assert_array_equal(chol.cpu().numpy(), rl)
        np.testing.assert_array_equal(color.cpu().numpy(), rc)
        assert gi.device_errors(clear=True) == 0
    bad = dict(stream)
    bad_idx = idx.copy()
    bad_idx[0, 7] = Bn  # one index past the codebook
    bad["idx"] = torch.from_numpy(bad_idx).cuda()
    gi.codec_decode(bad)
    assert gi.device_errors(clear=True) & 4  # GI_DEVERR_BOUNDS


@pytest.mark.parametrize("paper", [False, True])
def test_codec_encode_decode_renders_the_fit_image(gi, paper):
    """The stream a fine-tuning context encodes decodes (gi_codec_decode) to
    the Gaussians its render used: rendering them with the plain renderer
    gives the context's image bit for bit."""
    W, H, T, n = 128, 96, 16, 900
    target = synth.image(W, H, 46, n_blobs=12)
    means, chol, color = synth.init_gaussians(n, W, H, 46)
    p0 = paper_params(means, chol, color, W, H) if paper else np.concatenate([means, chol, color], axis=1)
    pt = torch.from_numpy(p0.astype(np.float32)).cuda()
    spec = gi.codec_init(pt, param_mode="paper" if paper else "pixel")
    fit = gi.Fit([torch.from_numpy(target).cuda()], [pt], tile=T, codec=spec, render_split=8,
                 param_mode="paper" if paper else "pixel", optimizer="adan" if paper else "adam")
    fit.step(4)
    stream = fit.encode()
    img = fit.images()[0].clone()
    m, l, c = gi.codec_decode(stream)
    ref = gi.rasterize(m, l, c, W, H, T)
    torch.cuda.synchronize()
    assert torch.equal(ref, img)
    assert stream["bits"] == n * (32 + 18 + 2 * 3) + 6 * 32 + 2 * 8 * 3 * 32
    fit.close()


def test_codec_checkpoint_resume_is_bit_identical(gi, tmp_path):
    """A codec fine-tuning context (paper parameters, Adan) saved after 4
    steps and restored into a fresh context continues exactly like the
    uninterrupted one: parameters, Adan state, gamma/beta, codebooks, EMA."""
    W, H, T, n = 128, 96, 16, 700
    target = torch.from_numpy(synth.image(W, H, 47, n_blobs=12)).cuda()
    p0 = torch.from_numpy(paper_params(*synth.init_gaussians(n, W, H, 47), W, H)).cuda()
    spec = gi.codec_init(p0, param_mode="paper")
    kw = dict(tile=T, lr=(1e-3, 1e-3, 1e-3), codec=spec, param_mode="paper", optimizer="adan")
    a = gi.Fit([target], [p0], **kw)
    a.step(4)
    path = tmp_path / "codec.pt"
    torch.save(a.state_dict(), path)
    a.step(3)
    b = gi.Fit([target], [p0], **kw)
    b.load_state_dict(torch.load(path))
    b.step(3)
    torch.cuda.synchronize()
    for k in ("params", "adam_m", "adam_v", "adan_n", "adan_gprev", "codec_gb", "codebooks", "ema_count",
              "ema_total"):
        assert torch.equal(getattr(a, k), getattr(b, k)), k
    plain = gi.Fit([target], [p0], tile=T, lr=(1e-3, 1e-3, 1e-3), param_mode="paper", optimizer="adan")
    with pytest.raises(ValueError):
        plain.load_state_dict(torch.load(path))
    for f in (a, b, plain):
        f.close()
