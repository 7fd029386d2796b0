"""Pins against numbers the paper prints (tests/golden/paper_constants.json)."""
import json
import os

import numpy as np

import oracle
import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_parameter_counts():
    # means (2) + Cholesky vector (3) + weighted colour (3) = 8 (Eq. 7)
    m, l, c = synth.init_gaussians(10, 64, 64, 0)
    per = m.shape[1] + l.shape[1] + c.shape[1]
    assert per == GOLD["params_per_gaussian_merged"]["value"]
    assert per + 1 == GOLD["params_per_gaussian_basic"]["value"]
    assert GOLD["params_3dgs"]["value"] / per == GOLD["compression_ratio_vs_3dgs"]["value"]
    assert GOLD["table1_kodak_params_k"]["value"] * 1000 // per == GOLD["table1_kodak_gaussians"]["value"]


def test_kodak_shaped_workload():
    c = synth.CONFIGS["c1_768x512_70k"]
    assert [c["W"], c["H"]] == GOLD["kodak_shape"]["value"]
    assert c["n"] == GOLD["table1_kodak_gaussians"]["value"]


def test_order_free_sum_removes_sort():
    """Sec. 3.2: accumulated summation needs no depth order, so the render of
    a reversed Gaussian list equals the original up to rounding."""
    W, H, T = 48, 40, 8
    m, l, c = synth.init_gaussians(30, W, H, 3)
    r, n = oracle.rect_rule(m, l, c, W, H, T)
    i, g, _ = oracle.bin_tiles(r, n, W, H, T)
    a = oracle.render(m, l, c, i, g, W, H, T)
    r2, n2 = oracle.rect_rule(m[::-1], l[::-1], c[::-1], W, H, T)
    i2, g2, _ = oracle.bin_tiles(r2, n2, W, H, T)
    b = oracle.render(m[::-1], l[::-1], c[::-1], i2, g2, W, H, T)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-15)
