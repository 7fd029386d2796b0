"""gi_fit_count_pairs: the pair count of a fitting context's first step,
computed by the library with the context's own formation (parameterisation,
covariance form, codec quantiser), against the oracle's support rule (the
sum of the tile counts of the FP32 3-sigma rectangles, Sec. 3.2 reading)
applied to the same pixel-space Gaussians, and against the K the first
fit step actually binned."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gi():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_08551_gb300 as m
    m.load()
    return m


def paper_raw(means, chol, W, H, rs=False):
    theta = np.arctanh(np.clip(means.astype(np.float64) / [W, H] * 2 - 1, -0.999, 0.999))
    c = chol.astype(np.float32).copy()
    if rs:
        c[:, 1:3] -= 0.5
    else:
        c[:, 0] -= 0.5
        c[:, 2] -= 0.5
    return theta, c


@pytest.mark.parametrize("mode", ["pixel", "paper", "rs", "paper_rs", "codec"])
@pytest.mark.parametrize("T", [8, 16])
def test_count_pairs_matches_oracle(gi, mode, T):
    shapes = [(200, 136, 1500), (96, 64, 700)] if mode != "codec" else [(200, 136, 1500)]
    targets, params, k_ref = [], [], 0
    codec = None
    for i, (W, H, n) in enumerate(shapes):
        targets.append(torch.from_numpy(synth.image(W, H, 60 + i, n_blobs=10)).cuda())
        if mode in ("rs", "paper_rs"):
            means, cov, color = synth.init_gaussians_rs(n, W, H, 60 + i)
        else:
            means, cov, color = synth.init_gaussians(n, W, H, 60 + i)
        if mode in ("paper", "paper_rs"):
            theta, raw = paper_raw(means, cov, W, H, rs=mode == "paper_rs")
            p = np.concatenate([theta, raw, color], axis=1).astype(np.float32)
            m_px, _, _ = oracle.paper_formation(p[:, 0:2], np.zeros((n, 3), np.float32), W, H)
            if mode == "paper_rs":
                rs_eff = p[:, 2:5].astype(np.float64)
                rs_eff[:, 1:3] += 0.5
                l_px = oracle.rs_to_chol(rs_eff)
            else:
                _, l_px, _ = oracle.paper_formation(p[:, 0:2], p[:, 2:5], W, H)
        else:
            p = np.concatenate([means, cov, color], axis=1).astype(np.float32)
            m_px = p[:, 0:2]
            l_px = oracle.rs_to_chol(p[:, 2:5]) if mode == "rs" else p[:, 2:5]
        pt = torch.from_numpy(p).cuda()
        if mode == "codec":
            codec = gi.codec_init(pt, bits=6, stages=2, size=8)
            m_px = oracle.fp16_round(m_px)
            l_px, _, _ = oracle.lsq_fake_quant(l_px, codec["gamma"], codec["beta"], 6)
        params.append(pt)
        _, cnt = oracle.rect_rule(m_px, l_px, p[:, 5:8], W, H, T)
        k_ref += int(cnt.astype(np.int64).sum())
    kw = dict(param_mode="paper" if mode.startswith("paper") else "pixel",
              cov="rs" if mode.endswith("rs") else "cholesky", codec=codec)
    fit = gi.Fit(targets, params, tile=T, **kw)
    assert fit.initial_pairs == k_ref
    fit.step(1)
    torch.cuda.synchronize()
    assert int(fit.k.item()) == k_ref
    fit.close()
