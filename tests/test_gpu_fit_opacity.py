"""GPU fits of Table 3's ablation forms against the oracle: separate opacity
with accumulated summation ("w/o M") and sorted alpha-blending ("w/o AR").
At every step the oracle runs at the GPU's own parameters and optimiser
state. Alpha-blending decides (skip, clamp, stop) in FP32 on the GPU and in
FP64 in the oracle; pixels where the oracle finds a decision within a
relative 3e-5 of its threshold are left out of the image comparison, and
each gradient's tolerance grows by twice the magnitude of its terms on those
pixels (what a decision taken the other way can change)."""
import numpy as np
import pytest

import oracle
import synth
import tolerances

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LR = (1e-3, 1e-2, 1e-2)


@pytest.fixture(scope="module")
def gi():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_08551_gb300 as m
    m.load()
    return m


def check_grads(g_gpu, g_ref, g_abs, g_amb, t, cond_ulps):
    tolerances.check_grads(g_gpu, g_ref, g_abs, f"step {t}", cond_ulps=cond_ulps, extra=2.0 * g_amb)


def run_opacity(gi, target, p0, logit0, T, steps, mode, optimizer="adam"):
    H, W, _ = target.shape
    n = p0.shape[0]
    fit = gi.Fit([torch.from_numpy(target).cuda()], [torch.from_numpy(p0).cuda()], tile=T, lr=LR,
                 opacity=mode, opacity_logits=[torch.from_numpy(logit0.astype(np.float32)).cuda()],
                 optimizer=optimizer)
    lrv = np.tile(np.array([LR[0]] * 2 + [LR[1]] * 3 + [LR[2]] * 3 + [LR[2]]), (n, 1))
    adan = optimizer == "adan"
    for t in range(1, steps + 1):
        pg = fit.params.cpu().numpy().astype(np.float64)
        lg = fit.opacity_logit.cpu().numpy().astype(np.float64)
        views = (fit.adam_m, fit.adam_v) + ((fit.adan_n, fit.adan_gprev) if adan else ())
        state = [x.cpu().numpy().astype(np.float64) for x in views]
        ostate = [x.cpu().numpy().astype(np.float64)[:, None] for x in
                  ((fit.opacity_m, fit.opacity_v) + ((fit.opacity_n, fit.opacity_gprev) if adan else ()))]
        means, chol, color = pg[:, 0:2].astype(np.float32), pg[:, 2:5].astype(np.float32), pg[:, 5:8].astype(np.float32)
        keep = np.ones(n, bool)
        if mode == "separate":
            r = oracle.opacity_forward_backward(means, chol, color, lg.astype(np.float32), target, T)
            g, go = r["grads"], r["grads_opacity"]
            g_ref = np.concatenate([g["means"], g["chol"], go["color"], go["logit"][:, None]], axis=1)
            a = g["abs"]
            g_abs = np.concatenate([a["means"], a["chol"], go["abs_color"], go["abs_logit"][:, None]], axis=1)
            g_amb = np.zeros_like(g_abs)
            cond_ulps = tolerances.COND_ULPS
        else:
            r = oracle.blend_forward_backward(means, chol, color, lg.astype(np.float32), target, T)
            g = r["grads"]
            g_ref = np.concatenate([g["means"], g["chol"], g["color"], g["logit"][:, None]], axis=1)
            a = g["abs"]
            g_abs = np.concatenate([a[:, 0:8], g["abs_logit"][:, None]], axis=1)
            g_amb = np.concatenate([g["abs_ambiguous"][:, 0:8], g["abs_ambiguous_logit"][:, None]], axis=1)
            cond_ulps = tolerances.BLEND_COND_ULPS  # transmittances: products of up to a few hundred FP32 factors
            assert r["ambiguous"].mean() < 2e-3
            keep = ~(g_amb > 0).any(axis=1)  # Gaussians untouched by ambiguous pixels
            assert keep.sum() > 100
        fit.step(1)
        torch.cuda.synchronize()
        # forward: the image and, for alpha-blending, each pixel's walk length
        img = fit.images()[0].cpu().numpy().astype(np.float64)
        ok = np.ones((H, W), bool) if mode == "separate" else ~r["ambiguous"]
        np.testing.assert_allclose(img[ok], r["out"][ok], rtol=0,
                                   atol=5e-5 * max(1.0, np.abs(r["out"]).max()))
        if mode == "blend":
            np.testing.assert_array_equal(fit.n_last.cpu().numpy().reshape(H, W)[ok], r["n_last"][ok])
        assert fit.mse()[0] == pytest.approx(r["loss"], rel=1e-4 if mode == "blend" else 1e-5)
        g_gpu = np.concatenate([fit.grads.cpu().numpy().astype(np.float64),
                                fit.opacity_grad.cpu().numpy().astype(np.float64)[:, None]], axis=1)
        check_grads(g_gpu, g_ref, g_abs, g_amb, t, cond_ulps)
        # optimiser updates (parameters and logits) from the GPU's state
        p_all = np.concatenate([pg, lg[:, None]], axis=1)
        st = [np.concatenate([s, o], axis=1) for s, o in zip(state, ostate)]
        if adan:
            p_ref, _ = oracle.adan(p_all, g_ref, tuple(st), t, lrv)
        else:
            p_ref, _, _ = oracle.adam(p_all, g_ref, st[0], st[1], t, lrv)
        p_new = np.concatenate([fit.params.cpu().numpy(), fit.opacity_logit.cpu().numpy()[:, None]],
                               axis=1).astype(np.float64)
        close = np.abs(p_new - p_ref) <= 1e-5 * np.maximum(np.abs(p_ref), 1.0) + 1e-3 * lrv
        assert close[keep].mean() > 0.999, f"step {t}: {np.sum(~close[keep])} parameters off the oracle's update"
        bound = (4 if adan else 2) * lrv + 1e-5 * np.maximum(np.abs(p_ref), 1.0)
        assert np.all((np.abs(p_new - p_ref) <= bound)[keep])
    return fit


def case(W, H, n, seed):
    target = synth.image(W, H, seed, n_blobs=20)
    means, chol, color = synth.init_gaussians(n, W, H, seed)
    # colours of the basic form are in [0, 1]; opacities around 0.3-0.7
    color = np.clip(color * 4.0, 0.0, 1.0).astype(np.float32)
    logit = np.random.default_rng(seed).normal(0.0, 1.0, n)
    return target, np.concatenate([means, chol, color], axis=1).astype(np.float32), logit


@pytest.mark.parametrize("T", [8, 16, 32])
def test_separate_opacity_steps_track_oracle(gi, T):
    target, p0, logit = case(128, 96, 800, 51)
    run_opacity(gi, target, p0, logit, T, 5, "separate").close()


def test_blend_steps_track_oracle(gi):
    target, p0, logit = case(128, 96, 800, 52)
    run_opacity(gi, target, p0, logit, 16, 5, "blend").close()


def test_blend_adan_steps_track_oracle(gi):
    target, p0, logit = case(160, 112, 1500, 53)
    run_opacity(gi, target, p0, logit, 16, 3, "blend", optimizer="adan").close()


@pytest.mark.slow
def test_blend_full_size(gi):
    """The 768x512, 70k-Gaussian workload with alpha-blending, two steps."""
    w = synth.workload("c1_768x512_70k")
    color = np.clip(w.color * 4.0, 0.0, 1.0).astype(np.float32)
    p0 = np.concatenate([w.means, w.chol, color], axis=1).astype(np.float32)
    logit = np.random.default_rng(54).normal(0.0, 1.0, w.n)
    run_opacity(gi, w.target, p0, logit, 16, 2, "blend").close()


def test_blend_render_pass_is_the_step_forward(gi):
    """fit.render() in blend mode reproduces the training step's image for
    the same parameters (graph replay and eager launches alike)."""
    target, p0, logit = case(96, 80, 600, 55)
    fits = [gi.Fit([torch.from_numpy(target).cuda()], [torch.from_numpy(p0).cuda()], tile=16, lr=(0.0, 0.0, 0.0),
                   opacity="blend", opacity_logits=[torch.from_numpy(logit.astype(np.float32)).cuda()],
                   use_graph=ug) for ug in (True, False)]
    for f in fits:
        f.step(1)
    torch.cuda.synchronize()
    imgs = [f.images()[0].clone() for f in fits]
    for f in fits:
        f.render()
    torch.cuda.synchronize()
    assert torch.equal(imgs[0], imgs[1])
    for f, im in zip(fits, imgs):
        assert torch.equal(f.images()[0], im)
        f.close()


def test_opacity_arguments_are_validated(gi):
    target, p0, logit = case(64, 64, 100, 56)
    tg, pt = torch.from_numpy(target).cuda(), torch.from_numpy(p0).cuda()
    with pytest.raises(gi.GIError):
        gi.Fit([tg], [pt], tile=8, opacity="blend")
    with pytest.raises(gi.GIError):
        gi.Fit([tg], [pt], tile=16, opacity="separate", cov="rs")
    with pytest.raises(ValueError):
        gi.Fit([tg], [pt], tile=16, opacity="transparent")


@pytest.mark.parametrize("mode", ["separate", "blend"])
def test_batched_equals_single(gi, mode):
    """Two images of different sizes in one context take, bit for bit, the
    steps each takes alone (per-image tiles, pixels, walk lengths and
    opacity state)."""
    cases = [case(96, 64, 400, 57), case(160, 112, 900, 58)]
    lg = [torch.from_numpy(c[2].astype(np.float32)).cuda() for c in cases]
    tg = [torch.from_numpy(c[0]).cuda() for c in cases]
    pr = [torch.from_numpy(c[1]).cuda() for c in cases]
    both = gi.Fit(tg, pr, tile=16, lr=LR, opacity=mode, opacity_logits=lg, render_split=8)
    both.step(3)
    torch.cuda.synchronize()
    o = 0
    for i in range(2):
        one = gi.Fit([tg[i]], [pr[i]], tile=16, lr=LR, opacity=mode, opacity_logits=[lg[i]], render_split=8)
        one.step(3)
        torch.cuda.synchronize()
        n = pr[i].shape[0]
        assert torch.equal(both.params[o:o + n], one.params)
        assert torch.equal(both.opacity_logit[o:o + n], one.opacity_logit)
        assert torch.equal(both.images()[i], one.images()[0])
        if mode == "blend":
            H, W = tg[i].shape[0], tg[i].shape[1]
            off = 0 if i == 0 else tg[0].shape[0] * tg[0].shape[1]
            assert torch.equal(both.n_last[off:off + H * W], one.n_last)
        o += n
        one.close()
    both.close()


def test_blend_checkpoint_resume_is_bit_identical(gi, tmp_path):
    target, p0, logit = case(96, 80, 600, 59)
    tg, pt = torch.from_numpy(target).cuda(), torch.from_numpy(p0).cuda()
    lg = [torch.from_numpy(logit.astype(np.float32)).cuda()]
    a = gi.Fit([tg], [pt], tile=16, lr=LR, opacity="blend", opacity_logits=lg)
    a.step(4)
    path = tmp_path / "blend.pt"
    torch.save(a.state_dict(), path)
    a.step(3)
    b = gi.Fit([tg], [pt], tile=16, lr=LR, opacity="blend", opacity_logits=lg)
    b.load_state_dict(torch.load(path))
    b.step(3)
    torch.cuda.synchronize()
    for k in ("params", "adam_m", "adam_v", "opacity_logit", "opacity_m", "opacity_v"):
        assert torch.equal(getattr(a, k), getattr(b, k)), k
    sep = gi.Fit([tg], [pt], tile=16, lr=LR, opacity="separate", opacity_logits=lg)
    with pytest.raises(ValueError):
        sep.load_state_dict(torch.load(path))
    for f in (a, b, sep):
        f.close()
