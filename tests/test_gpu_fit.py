"""GPU fitting: Adam steps against the oracle, graph replay against eager
launches, and batched multi-image steps against one-image steps."""
import numpy as np
import pytest

import oracle
import synth
from tolerances import REL as GRAD_TOL, check_grads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LR = (1e-3, 1e-2, 1e-2)  # means, Cholesky, colour


@pytest.fixture(scope="module")
def gi():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_08551_gb300 as m
    m.load()
    return m


def pack(means, chol, color):
    return np.concatenate([means, chol, color], axis=1).astype(np.float32)


def lr_vec(n):
    return np.tile(np.array([LR[0]] * 2 + [LR[1]] * 3 + [LR[2]] * 3), (n, 1))


def oracle_grads(p, target, T, with_abs=False):
    r = oracle.forward_backward(p[:, 0:2].astype(np.float32), p[:, 2:5].astype(np.float32),
                                p[:, 5:8].astype(np.float32), target, T)
    g = np.concatenate([r["grads"]["means"], r["grads"]["chol"], r["grads"]["color"]], axis=1)
    if with_abs:
        a = r["grads"]["abs"]
        return g, r["loss"], np.concatenate([a["means"], a["chol"], a["color"]], axis=1)
    return g, r["loss"]


def test_first_step_matches_oracle(gi):
    """Step 1 from zero Adam state: the update is -lr g/(|g| + eps). The GPU
    gradient is within GRAD_TOL of the oracle's, which bounds the update
    difference element by element (a sign may flip only where |g| is below
    that tolerance)."""
    W, H, T, n = 256, 256, 16, 2000
    target = synth.image(W, H, 0, n_blobs=40)
    p0 = pack(*synth.init_gaussians(n, W, H, 0))
    fit = gi.Fit([torch.from_numpy(target).cuda()], [torch.from_numpy(p0).cuda()], tile=T, lr=LR)
    fit.step(1)
    torch.cuda.synchronize()
    g_ref, loss_ref, g_abs = oracle_grads(p0, target, T, with_abs=True)
    g_gpu = fit.grads.cpu().numpy().astype(np.float64)
    tol_g = check_grads(g_gpu, g_ref, g_abs, "step 1")
    assert fit.mse()[0] == pytest.approx(loss_ref, rel=1e-5)
    p1_ref, _, _ = oracle.adam(p0.astype(np.float64), g_ref, 0.0, 0.0, 1, lr_vec(n))
    p1 = fit.params.cpu().numpy().astype(np.float64)
    lr = lr_vec(n)
    eps = oracle.ADAM_EPS
    a = np.abs(g_ref)
    safe = a > tol_g
    bound = np.where(safe, lr * eps * tol_g / np.maximum(a - tol_g + eps, 1e-30) ** 2, 2 * lr)
    bound = bound + 4 * np.finfo(np.float32).eps * np.maximum(np.abs(p1_ref), 1.0) + 1e-6 * lr
    assert np.all(np.abs(p1 - p1_ref) <= bound)
    assert int(fit.step_count.item()) == 1
    fit.close()


def test_five_steps_track_oracle(gi):
    """Five free-running steps: the loss trajectories agree to 1e-5 and the
    parameters stay within the sign-flip envelope of the first step."""
    W, H, T, n = 128, 96, 16, 800
    target = synth.image(W, H, 21, n_blobs=20)
    p = pack(*synth.init_gaussians(n, W, H, 21))
    fit = gi.Fit([torch.from_numpy(target).cuda()], [torch.from_numpy(p).cuda()], tile=T, lr=LR)
    pr = p.astype(np.float64)
    m = np.zeros_like(pr)
    v = np.zeros_like(pr)
    lr = lr_vec(n)
    for t in range(1, 6):
        g, L = oracle_grads(pr, target, T)
        fit.step(1)
        torch.cuda.synchronize()
        assert fit.mse()[0] == pytest.approx(L, rel=1e-5)
        pr, m, v = oracle.adam(pr, g, m, v, t, lr)
    pg = fit.params.cpu().numpy().astype(np.float64)
    close = np.abs(pg - pr) <= 1e-5 * np.maximum(np.abs(pr), 1.0)
    assert close.mean() > 0.999
    assert np.all(np.abs(pg - pr) <= 2 * 5 * lr + 1e-5 * np.maximum(np.abs(pr), 1.0))
    fit.close()


@pytest.mark.slow
def test_full_size_five_steps(gi):
    """The 768x512, 70k-Gaussian fitting workload at tile 16 (the benchmark's
    configuration), first five Adam steps. At every step the oracle is
    evaluated at the GPU's own parameters, so each step's loss and gradients
    are checked exactly (tolerance of test_gpu_parity with its conditioning
    clause), and the Adam update from the GPU's own moments is checked
    against the oracle's update inside the envelope a gradient error of that
    size allows."""
    w = synth.workload("c1_768x512_70k")
    T = 16
    p0 = pack(w.means, w.chol, w.color)
    fit = gi.Fit([torch.from_numpy(w.target).cuda()], [torch.from_numpy(p0).cuda()], tile=T, lr=LR)
    lr = lr_vec(w.n)
    for t in range(1, 6):
        pg = fit.params.cpu().numpy().astype(np.float64)
        mg = fit.adam_m.cpu().numpy().astype(np.float64)
        vg = fit.adam_v.cpu().numpy().astype(np.float64)
        g_ref, loss_ref, g_abs = oracle_grads(pg, w.target, T, with_abs=True)
        fit.step(1)
        torch.cuda.synchronize()
        assert fit.mse()[0] == pytest.approx(loss_ref, rel=1e-5)
        g_gpu = fit.grads.cpu().numpy().astype(np.float64)
        check_grads(g_gpu, g_ref, g_abs, f"step {t}")
        p_ref, _, _ = oracle.adam(pg, g_ref, mg, vg, t, lr)
        p_new = fit.params.cpu().numpy().astype(np.float64)
        close = np.abs(p_new - p_ref) <= 1e-5 * np.maximum(np.abs(p_ref), 1.0) + 1e-3 * lr
        assert close.mean() > 0.999, f"step {t}: {np.sum(~close)} parameters off the oracle's update"
        assert np.all(np.abs(p_new - p_ref) <= 2 * lr + 1e-5 * np.maximum(np.abs(p_ref), 1.0))
    assert int(fit.step_count.item()) == 5
    fit.close()


def paper_raw(means, chol, color, W, H):
    """Raw App. C.1 parameters giving these pixel-space Gaussians:
    theta = atanh(2 mu / (W, H) - 1), Cholesky diagonal without its +0.5."""
    u = np.clip(means.astype(np.float64) / [W, H] * 2 - 1, -0.999, 0.999)
    theta = np.arctanh(u)
    c = chol.astype(np.float32).copy()
    c[:, 0] -= 0.5
    c[:, 2] -= 0.5
    return theta, c, color


def run_paper_adan(gi, W, H, means, chol, color, target, T, steps, lr=1e-3, halve=0):
    """Fits with the paper's parameterisation and Adan; at every step the
    oracle runs at the GPU's own raw parameters, so each step's loss and
    gradients are checked exactly, and the Adan update from the GPU's own
    state is checked against the oracle's update."""
    theta, craw, col = paper_raw(means, chol, color, W, H)
    p0 = np.concatenate([theta, craw, col], axis=1).astype(np.float32)
    fit = gi.Fit([torch.from_numpy(target).cuda()], [torch.from_numpy(p0).cuda()], tile=T, lr=(lr, lr, lr),
                 param_mode="paper", optimizer="adan", lr_halve_every=halve)
    n = p0.shape[0]
    lrv = np.full((n, 8), lr)
    for t in range(1, steps + 1):
        pg = fit.params.cpu().numpy().astype(np.float64)
        state = tuple(x.cpu().numpy().astype(np.float64) for x in (fit.adam_m, fit.adam_v, fit.adan_n, fit.adan_gprev))
        r = oracle.paper_forward_backward(pg[:, 0:2], pg[:, 2:5].astype(np.float32), pg[:, 5:8].astype(np.float32),
                                          target, T)
        gr = r["grads_raw"]
        g_ref = np.concatenate([gr["theta"], gr["chol"], gr["color"]], axis=1)
        g_abs = np.concatenate([gr["abs_theta"], r["grads"]["abs"]["chol"], r["grads"]["abs"]["color"]], axis=1)
        fit.step(1)
        torch.cuda.synchronize()
        assert fit.mse()[0] == pytest.approx(r["loss"], rel=1e-5)
        g_gpu = fit.grads.cpu().numpy().astype(np.float64)
        check_grads(g_gpu, g_ref, g_abs, f"step {t}")
        p_ref, _ = oracle.adan(pg, g_ref, state, t, oracle.lr_at(1.0, t, halve) * lrv)
        p_new = fit.params.cpu().numpy().astype(np.float64)
        close = np.abs(p_new - p_ref) <= 1e-5 * np.maximum(np.abs(p_ref), 1.0) + 1e-3 * lr
        assert close.mean() > 0.999, f"step {t}: {np.sum(~close)} parameters off the oracle's Adan update"
        assert np.all(np.abs(p_new - p_ref) <= 4 * lr + 1e-5 * np.maximum(np.abs(p_ref), 1.0))
    return fit


@pytest.mark.parametrize("T", [8, 16, 32])
def test_paper_mode_adan_steps_track_oracle(gi, T):
    W, H, n = 128, 96, 800
    target = synth.image(W, H, 25, n_blobs=20)
    means, chol, color = synth.init_gaussians(n, W, H, 25)
    fit = run_paper_adan(gi, W, H, means, chol, color, target, T, 5, halve=3)
    assert int(fit.step_count.item()) == 5
    fit.close()


@pytest.mark.slow
def test_paper_mode_adan_full_size(gi):
    """The 768x512, 70k-Gaussian workload with the paper's parameterisation
    and optimiser, first five steps."""
    w = synth.workload("c1_768x512_70k")
    fit = run_paper_adan(gi, w.W, w.H, w.means, w.chol, w.color, w.target, 16, 5)
    fit.close()


def test_graph_replay_equals_eager(gi):
    W, H, T, n = 160, 120, 16, 1500
    target = torch.from_numpy(synth.image(W, H, 22, n_blobs=20)).cuda()
    p = torch.from_numpy(pack(*synth.init_gaussians(n, W, H, 22))).cuda()
    a = gi.Fit([target], [p], tile=T, lr=LR, use_graph=True)
    b = gi.Fit([target], [p], tile=T, lr=LR, use_graph=False)
    a.step(4)
    b.step(4)
    torch.cuda.synchronize()
    assert torch.equal(a.params, b.params)
    assert torch.equal(a.adam_v, b.adam_v)
    a.close()
    b.close()


def test_checkpoint_resume_is_bit_identical(gi, tmp_path):
    """A fit saved after 4 steps (torch.save of state_dict) and restored into
    a fresh context continues exactly like the uninterrupted fit."""
    W, H, T, n = 160, 120, 16, 1500
    target = torch.from_numpy(synth.image(W, H, 24, n_blobs=20)).cuda()
    p = torch.from_numpy(pack(*synth.init_gaussians(n, W, H, 24))).cuda()
    a = gi.Fit([target], [p], tile=T, lr=LR)
    a.step(4)
    path = tmp_path / "fit.pt"
    torch.save(a.state_dict(), path)
    a.step(3)
    b = gi.Fit([target], [p], tile=T, lr=LR)
    b.load_state_dict(torch.load(path))
    b.step(3)
    torch.cuda.synchronize()
    assert torch.equal(a.params, b.params)
    assert torch.equal(a.adam_m, b.adam_m) and torch.equal(a.adam_v, b.adam_v)
    assert int(a.step_count.item()) == int(b.step_count.item()) == 7
    assert a.mse() == b.mse()
    with pytest.raises(ValueError):
        c = gi.Fit([target], [p[:100]], tile=T, lr=LR)
        try:
            c.load_state_dict(torch.load(path))
        finally:
            c.close()
    a.close()
    b.close()


def test_fit_render_is_the_forward_only(gi):
    """gi_fit_render: the image of the current parameters (same as the
    per-stage calls with the same render split), graph replay identical to
    the eager launches, and the last step's loss left in place."""
    W, H, T, n = 160, 120, 16, 1500
    target = torch.from_numpy(synth.image(W, H, 23, n_blobs=20)).cuda()
    p = torch.from_numpy(pack(*synth.init_gaussians(n, W, H, 23))).cuda()
    a = gi.Fit([target], [p], tile=T, lr=LR, use_graph=True, render_split=8)
    b = gi.Fit([target], [p], tile=T, lr=LR, use_graph=False, render_split=8)
    a.step(3)
    b.step(3)
    torch.cuda.synchronize()
    mse = a.mse()[0]
    a.render()
    b.render()
    torch.cuda.synchronize()
    assert a.mse()[0] == mse
    assert torch.equal(a.images()[0], b.images()[0])
    q = a.params
    ref = gi.rasterize(q[:, 0:2].contiguous(), q[:, 2:5].contiguous(), q[:, 5:8].contiguous(), W, H, T)
    torch.cuda.synchronize()
    assert torch.equal(a.images()[0], ref)
    a.close()
    b.close()


@pytest.mark.parametrize("T,split", [(8, 2), (8, 4), (16, 4), (16, 8), (32, 1), (32, 2)])
def test_batched_equals_single(gi, T, split):
    """Images fitted together in one launch per stage give bit-identical
    parameters to the same images fitted alone (every tile edge and render
    split)."""
    shapes = [(96, 64, 700), (130, 77, 1100), (64, 64, 300)]
    targets, params = [], []
    for i, (W, H, n) in enumerate(shapes):
        targets.append(torch.from_numpy(synth.image(W, H, 30 + i, n_blobs=10)).cuda())
        params.append(torch.from_numpy(pack(*synth.init_gaussians(n, W, H, 30 + i))).cuda())
    batched = gi.Fit(targets, params, tile=T, lr=LR, render_split=split)
    batched.step(3)
    torch.cuda.synchronize()
    pb = batched.params.clone()
    mse_b = batched.mse()
    off = 0
    for i, (W, H, n) in enumerate(shapes):
        single = gi.Fit([targets[i]], [params[i]], tile=T, lr=LR, render_split=split)
        single.step(3)
        torch.cuda.synchronize()
        assert torch.equal(single.params, pb[off:off + n]), f"image {i}"
        assert single.mse()[0] == mse_b[i]  # per-tile loss partials summed in tile order
        single.close()
        off += n
    batched.close()


@pytest.mark.parametrize("T", [8, 16, 32])
def test_tile_queue_equals_tile_order(gi, T):
    """The render fed from the device queue of tiles ordered by descending
    list length (persistent blocks) gives the same parameters, moments,
    losses and images, bit for bit, as one block per tile in tile order, on
    an uneven batch."""
    shapes = [(200, 136, 1600), (96, 64, 700), (130, 77, 1100)]
    targets, params = [], []
    for i, (W, H, n) in enumerate(shapes):
        targets.append(torch.from_numpy(synth.image(W, H, 50 + i, n_blobs=10)).cuda())
        params.append(torch.from_numpy(pack(*synth.init_gaussians(n, W, H, 50 + i))).cuda())
    a = gi.Fit(targets, params, tile=T, lr=LR, tile_queue=False)
    b = gi.Fit(targets, params, tile=T, lr=LR, tile_queue=True)
    a.step(4)
    b.step(4)
    torch.cuda.synchronize()
    assert torch.equal(a.params, b.params) and torch.equal(a.adam_m, b.adam_m) and torch.equal(a.adam_v, b.adam_v)
    assert a.mse() == b.mse()
    a.render()
    b.render()
    torch.cuda.synchronize()
    for x, y in zip(a.images(), b.images()):
        assert torch.equal(x, y)
    assert gi.device_errors(clear=True) == 0
    a.close()
    b.close()


def test_fit_reduces_loss(gi):
    W, H, T, n = 128, 128, 16, 1500
    target = torch.from_numpy(synth.image(W, H, 23, n_blobs=20)).cuda()
    p = torch.from_numpy(pack(*synth.init_gaussians(n, W, H, 23))).cuda()
    fit = gi.Fit([target], [p], tile=T, lr=LR)
    fit.step(1)
    torch.cuda.synchronize()
    first = fit.mse()[0]
    fit.step(200)
    torch.cuda.synchronize()
    last = fit.mse()[0]
    assert last < 0.5 * first
    assert gi.device_errors(clear=True) == 0
    fit.close()


def test_autotune_picks_a_measured_configuration(gi):
    shapes = [(96, 64, 600), (64, 64, 300)]
    targets = [torch.from_numpy(synth.image(W, H, 40 + i, n_blobs=8)).cuda() for i, (W, H, _) in enumerate(shapes)]
    params = [torch.from_numpy(pack(*synth.init_gaussians(n, W, H, 40 + i))).cuda()
              for i, (W, H, n) in enumerate(shapes)]
    before = [p.clone() for p in params]
    res = gi.autotune(targets, params, steps=3, warmup=1)
    assert (res["tile"], res["render_split"]) in res["ms_per_step"]
    assert len(res["ms_per_step"]) == 6 and all(v > 0 for v in res["ms_per_step"].values())
    assert res["ms_per_step"][(res["tile"], res["render_split"])] == min(res["ms_per_step"].values())
    for p, b in zip(params, before):
        assert torch.equal(p, b)


def test_render_split_is_validated(gi):
    t = torch.from_numpy(synth.image(32, 32, 41, n_blobs=2)).cuda()
    p = torch.from_numpy(pack(*synth.init_gaussians(10, 32, 32, 41))).cuda()
    with pytest.raises(gi.GIError):
        gi.Fit([t], [p], tile=16, render_split=2)


def test_target_source_pinned_host_and_device_match_the_own_copy(gi):
    """A fit reading its target from pinned host memory (over the host link,
    inside the render) or from another device buffer takes the same steps,
    bit for bit, as one reading its own copy; graph replay and eager alike."""
    W, H, T, n = 160, 120, 16, 1500
    target = synth.image(W, H, 24, n_blobs=20)
    p = torch.from_numpy(pack(*synth.init_gaussians(n, W, H, 24))).cuda()
    tg = torch.from_numpy(target).cuda()
    host = torch.from_numpy(target.reshape(-1).copy()).pin_memory()
    dev = tg.reshape(-1).clone()
    ref = gi.Fit([tg], [p], tile=T, lr=LR)
    ref.step(4)
    for ug in (True, False):
        for src in (host, dev):
            f = gi.Fit([torch.zeros_like(tg)], [p], tile=T, lr=LR, use_graph=ug)  # own copy is all zeros
            f.set_target_source(src)
            f.step(4)
            torch.cuda.synchronize()
            assert torch.equal(f.params, ref.params)
            assert f.mse()[0] == ref.mse()[0]
            f.set_target_source(None)  # back to the (zero) own copy: a different loss
            f.step(1)
            torch.cuda.synchronize()
            assert f.mse()[0] != ref.mse()[0]
            f.close()
    with pytest.raises(ValueError):
        ref.set_target_source(torch.from_numpy(target.reshape(-1).copy()))  # pageable
    ref.close()


def test_target_source_rejects_pageable_memory_in_the_abi(gi):
    import ctypes
    from paper_2403_08551_gb300 import _lib as L
    W, H, T, n = 64, 64, 16, 100
    target = synth.image(W, H, 25, n_blobs=4)
    f = gi.Fit([torch.from_numpy(target).cuda()], [torch.from_numpy(pack(*synth.init_gaussians(n, W, H, 25))).cuda()],
               tile=T, lr=LR)
    pageable = np.ascontiguousarray(target.reshape(-1), np.float32)
    rc = L.load().gi_fit_set_target_source(f._h_fit, pageable.ctypes.data_as(ctypes.c_void_p), L.stream_handle())
    assert rc != 0
    f.step(1)  # the context still works
    torch.cuda.synchronize()
    f.close()
