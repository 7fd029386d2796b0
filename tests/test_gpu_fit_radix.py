"""Fused fit steps on the radix binning path (more than 2048 tiles per
batch: the stable onesweep LSD sort, its key emission and range scan feed
the backward's pair offsets and the optimiser) against the oracle.

At every step the oracle runs at the GPU's own parameters (teacher-forced,
image by image: the images of a batch are independent), so each step is
checked exactly (Sec. 3.4 and App. A):
  - the fit's own binning of that step, bit for bit: support rectangles and
    counts, pair offsets, sorted Gaussian ids, tile keys and ranges against
    the oracle's rect_rule and bin_tiles mapped to the batch's global tile and
    Gaussian numbering;
  - each image's loss, and every gradient within tests/tolerances.py;
  - the optimiser update from the GPU's own state against the oracle's
    update, inside the envelope a gradient error of that size allows.
"""
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


def pixel_space(p, W, H, mode):
    """Pixel-space means, Cholesky vectors and colours the formation renders
    from the fit's parameters p [n, 8] (FP64 copy of the FP32 state)."""
    color = p[:, 5:8].astype(np.float32)
    if mode == "paper":
        means, chol, _ = oracle.paper_formation(p[:, 0:2], p[:, 2:5].astype(np.float32), W, H)
    elif mode == "rs":
        means, chol = p[:, 0:2].astype(np.float32), oracle.rs_to_chol(p[:, 2:5].astype(np.float32))
    else:
        means, chol = p[:, 0:2].astype(np.float32), p[:, 2:5].astype(np.float32)
    return means, chol, color


def oracle_image_step(p, target, T, mode):
    """Loss, gradients [n, 8] and their condition magnitudes for one image."""
    H, W, _ = target.shape
    if mode == "paper":
        r = oracle.paper_forward_backward(p[:, 0:2], p[:, 2:5].astype(np.float32), p[:, 5:8].astype(np.float32),
                                          target, T)
        gr = r["grads_raw"]
        g = np.concatenate([gr["theta"], gr["chol"], gr["color"]], axis=1)
        a = np.concatenate([gr["abs_theta"], r["grads"]["abs"]["chol"], r["grads"]["abs"]["color"]], axis=1)
        return r["loss"], g, a
    if mode == "rs":
        from test_gpu_fit_rs import oracle_step
        return oracle_step(p, target, T, paper=False)
    means, chol, color = pixel_space(p, W, H, mode)
    r = oracle.forward_backward(means, chol, color, target, T)
    gg, ab = r["grads"], r["grads"]["abs"]
    g = np.concatenate([gg["means"], gg["chol"], gg["color"]], axis=1)
    a = np.concatenate([ab["means"], ab["chol"], ab["color"]], axis=1)
    return r["loss"], g, a


def expected_binning(pg, shapes, counts, T, mode):
    """The oracle's binning of the whole batch in global numbering: tiles of
    image b follow those of images < b, Gaussians likewise, and the sorted
    pairs of image b follow all pairs of images < b (tiles ascending)."""
    rects, cnts, ids, ranges, offs, keys = [], [], [], [], [], []
    g0 = t0 = k0 = 0
    for (W, H), n in zip(shapes, counts):
        p = pg[g0:g0 + n]
        rect, cnt = oracle.rect_rule(*pixel_space(p, W, H, mode), W, H, T)
        i, rg, off = oracle.bin_tiles(rect, cnt, W, H, T)
        tw, th = oracle.tiles(W, H, T)
        rects.append(rect)
        cnts.append(cnt)
        ids.append(i.astype(np.int64) + g0)
        r = rg.astype(np.int64)
        live = r[:, 1] > r[:, 0]
        r[live] += k0
        ranges.append(r)
        offs.append(off[:-1] + k0)
        keys.append(np.repeat(np.arange(tw * th, dtype=np.int64) + t0, rg[:, 1] - rg[:, 0]))
        g0 += n
        t0 += tw * th
        k0 += int(off[-1])
    offs.append(np.array([k0]))
    return dict(K=k0, rect=np.concatenate(rects), cnt=np.concatenate(cnts), ids=np.concatenate(ids),
                ranges=np.concatenate(ranges), pair_off=np.concatenate(offs), keys=np.concatenate(keys))


def check_binning(fit, exp):
    b = fit.binning()
    assert b["K"] == exp["K"]
    for name in ("rect", "cnt", "pair_off", "ranges"):
        np.testing.assert_array_equal(b[name].cpu().numpy().astype(np.int64), exp[name].astype(np.int64),
                                      err_msg=name)
    np.testing.assert_array_equal(b["ids"].cpu().numpy().astype(np.int64) & 0xffffffff, exp["ids"], err_msg="ids")
    np.testing.assert_array_equal(b["keys"].cpu().numpy().astype(np.int64) & 0xffffffff, exp["keys"], err_msg="keys")


def run_batch(gi, targets, params, T, mode="pixel", optimizer="adam", lr=LR, steps=5, halve=0):
    shapes = [(t.shape[1], t.shape[0]) for t in targets]
    counts = [p.shape[0] for p in params]
    n_tiles = sum(oracle.tiles(W, H, T)[0] * oracle.tiles(W, H, T)[1] for W, H in shapes)
    assert n_tiles > 2048, "the case must take the radix binning path"
    fit = gi.Fit([torch.from_numpy(t).cuda() for t in targets], [torch.from_numpy(p).cuda() for p in params], tile=T,
                 lr=lr, param_mode="paper" if mode == "paper" else "pixel", optimizer=optimizer,
                 cov="rs" if mode == "rs" else "cholesky", lr_halve_every=halve)
    N = sum(counts)
    lrv = np.tile(np.array([lr[0]] * 2 + [lr[1]] * 3 + [lr[2]] * 3), (N, 1))
    for t in range(1, steps + 1):
        pg = fit.params.cpu().numpy().astype(np.float64)
        views = (fit.adam_m, fit.adam_v) + ((fit.adan_n, fit.adan_gprev) if optimizer == "adan" else ())
        state = tuple(x.cpu().numpy().astype(np.float64) for x in views)
        exp = expected_binning(pg, shapes, counts, T, mode)
        losses, g_ref, g_abs = [], [], []
        g0 = 0
        for tgt, n in zip(targets, counts):
            loss, g, a = oracle_image_step(pg[g0:g0 + n], tgt, T, mode)
            losses.append(loss)
            g_ref.append(g)
            g_abs.append(a)
            g0 += n
        g_ref, g_abs = np.concatenate(g_ref), np.concatenate(g_abs)
        fit.step(1)
        torch.cuda.synchronize()
        check_binning(fit, exp)
        for i, (got, want) in enumerate(zip(fit.mse(), losses)):
            assert got == pytest.approx(want, rel=1e-5), f"step {t} image {i}"
        g_gpu = fit.grads.cpu().numpy().astype(np.float64)
        tolerances.check_grads(g_gpu, g_ref, g_abs, f"step {t}")
        lr_t = oracle.lr_at(1.0, t, halve) * lrv
        if optimizer == "adan":
            p_ref, _ = oracle.adan(pg, g_ref, state, t, lr_t)
        else:
            p_ref, _, _ = oracle.adam(pg, g_ref, state[0], state[1], t, lr_t)
        p_new = fit.params.cpu().numpy().astype(np.float64)
        close = np.abs(p_new - p_ref) <= 1e-5 * np.maximum(np.abs(p_ref), 1.0) + 1e-3 * lr_t
        assert close.mean() > 0.999, f"step {t}: {np.sum(~close)} parameters off the oracle's update"
        bound = (4 if optimizer == "adan" else 2) * lr_t
        assert np.all(np.abs(p_new - p_ref) <= bound + 1e-5 * np.maximum(np.abs(p_ref), 1.0))
    assert int(fit.step_count.item()) == steps
    assert gi.device_errors(clear=True) == 0
    return fit


def pack(means, chol, color):
    return np.concatenate([means, chol, color], axis=1).astype(np.float32)


def paper_raw(means, chol, color, W, H):
    theta = np.arctanh(np.clip(means.astype(np.float64) / [W, H] * 2 - 1, -0.999, 0.999))
    c = chol.astype(np.float32).copy()
    c[:, 0] -= 0.5
    c[:, 2] -= 0.5
    return np.concatenate([theta, c, color], axis=1).astype(np.float32)


def uneven_batch(sizes, seed, mode="pixel"):
    """Images of the uneven-batch workload's sizes with its Gaussian counts
    (max(5000, 70000 P / 786432)) and generator."""
    targets, params = [], []
    for i, (W, H) in enumerate(sizes):
        n = synth.batch_gaussian_count(W, H)
        targets.append(synth.image(W, H, seed + i, n_blobs=max(10, (W * H) // 2000)))
        if mode == "rs":
            means, rs, color = synth.init_gaussians_rs(n, W, H, seed + i)
            params.append(pack(means, rs, color))
            continue
        means, chol, color = synth.init_gaussians(n, W, H, seed + i)
        params.append(paper_raw(means, chol, color, W, H) if mode == "paper" else pack(means, chol, color))
    return targets, params


BATCH = [(1024, 768), (512, 384), (256, 256), (768, 512)]  # 3072 + 768 + 256 + 1536 tiles at T = 16


@pytest.mark.slow
def test_radix_fit_large_image(gi):
    """The skewed 2040x1356 image with 100k Gaussians at T = 16 (10,880
    tiles, three radix passes of 5 bits), Adam."""
    w = synth.workload("c2_2040x1356_100k")
    run_batch(gi, [w.target], [pack(w.means, w.chol, w.color)], 16).close()


@pytest.mark.slow
@pytest.mark.parametrize("mode,optimizer", [("pixel", "adam"), ("paper", "adan")])
def test_radix_fit_uneven_batch(gi, mode, optimizer):
    """Four images of the uneven-batch sizes, one of them 1024x768 (5632
    tiles at T = 16), in one fit: the pixel-space parameters with Adam, and
    the paper's parameterisation with Adan and learning-rate halving."""
    targets, params = uneven_batch(BATCH, 3100, mode)
    lr = LR if optimizer == "adam" else (1e-3, 1e-3, 1e-3)
    run_batch(gi, targets, params, 16, mode, optimizer, lr=lr, halve=3 if optimizer == "adan" else 0).close()


def test_radix_fit_tile8_rotation_scaling(gi):
    """A two-image batch at T = 8 (4096 tiles) in the rotation-scaling form."""
    targets, params = uneven_batch([(512, 384), (256, 256)], 3200, "rs")
    run_batch(gi, targets, params, 8, "rs").close()
