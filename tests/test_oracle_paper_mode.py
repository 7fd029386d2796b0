"""Pins of the oracle's paper-mode parameterisation (App. C.1) and of its
Adan step (Sec. 4.1; Xie et al. 2022), each against something other than the
oracle's own arithmetic. CPU only."""
import math

import numpy as np
import pytest

import oracle
import synth


def test_atanh_init_round_trip():
    """App. C.1 initialises positions as atanh(u * 2 - 1); with the reading
    mu = (tanh(theta) + 1) / 2 * (W, H) that is the uniform draw u scaled to
    pixels, and the Jacobian is the derivative of that map."""
    u = np.random.default_rng(1).uniform(0.02, 0.98, (500, 2))
    theta = np.arctanh(u * 2 - 1)
    chol = np.ones((500, 3), np.float32)
    means, c, dmu = oracle.paper_formation(theta, chol, 768, 512)
    np.testing.assert_allclose(means, (u * [768, 512]).astype(np.float32), rtol=2e-7, atol=1e-4)
    np.testing.assert_array_equal(c, np.array([1.5, 1.0, 1.5], np.float32)[None].repeat(500, 0))
    h = 1e-6
    fd = ((np.tanh(theta + h) + 1) - (np.tanh(theta - h) + 1)) / (2 * h) * 0.5 * np.array([768, 512])
    np.testing.assert_allclose(dmu, fd, rtol=1e-7)


def test_paper_gradients_match_finite_differences():
    """Central differences of the FP64 loss in the raw parameters (theta and
    the shifted Cholesky vector), support held fixed, against the chained
    analytic gradients."""
    W, H, T, n = 24, 20, 8, 6
    means, chol, col = synth.init_gaussians(n, W, H, 43)
    target = synth.image(W, H, 43, n_blobs=5)
    theta = np.arctanh(means.astype(np.float64) / [W, H] * 2 - 1)
    chol_raw = chol.copy()
    chol_raw[:, 0] -= 0.5
    chol_raw[:, 2] -= 0.5
    r = oracle.paper_forward_backward(theta, chol_raw, col, target, T)
    ids, ranges = r["ids"], r["ranges"]

    def loss_at(th, cr):
        m, c, _ = oracle.paper_formation(th, cr, W, H)
        out = oracle.render(m, c, col, ids, ranges, W, H, T)
        return oracle.loss(out, target)[0]

    # theta: the formation rounds mu to FP32, so the step must move mu by
    # many ulps; Richardson extrapolation of two central differences.
    g_theta = np.zeros_like(theta)
    for idx in np.ndindex(theta.shape):
        def central(h):
            tp, tm = theta.copy(), theta.copy()
            tp[idx] += h
            tm[idx] -= h
            return (loss_at(tp, chol_raw) - loss_at(tm, chol_raw)) / (2 * h)
        h = 1e-3
        g_theta[idx] = (4 * central(h / 2) - central(h)) / 3
    np.testing.assert_allclose(r["grads_raw"]["theta"], g_theta, rtol=2e-4,
                               atol=1e-4 * np.abs(g_theta).max())
    g_chol = np.zeros(chol_raw.shape)
    for idx in np.ndindex(chol_raw.shape):
        v = float(chol_raw[idx])
        h = 2.0 ** (math.floor(math.log2(abs(v))) - 8) if v != 0 else 2.0 ** -12

        def central_c(hh):
            cp, cm = chol_raw.copy(), chol_raw.copy()
            cp[idx] = np.float32(v + hh)
            cm[idx] = np.float32(v - hh)
            return (loss_at(theta, cp) - loss_at(theta, cm)) / (2 * hh)
        g_chol[idx] = (4 * central_c(h / 2) - central_c(h)) / 3
    np.testing.assert_allclose(r["grads_raw"]["chol"], g_chol, rtol=1e-5,
                               atol=1e-7 * np.abs(g_chol).max())


def _zero_state(n):
    return tuple(np.zeros(n) for _ in range(4))


def test_adan_first_step_closed_form():
    """First step: the gradient difference is 0, m^ = g, n^ = g^2, so the
    step is -lr g / (|g| + eps)."""
    g = np.random.default_rng(4).standard_normal(100)
    p0 = np.random.default_rng(5).standard_normal(100)
    p1, st = oracle.adan(p0, g, _zero_state(100), 1, 1e-3)
    np.testing.assert_allclose(p1, p0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-13, atol=1e-16)


def test_adan_constant_gradient_closed_form():
    """With a constant gradient every difference is 0: each step moves by
    -lr g / (|g| + eps), whatever the averages' decay."""
    g = np.random.default_rng(6).standard_normal(50)
    p = np.zeros(50)
    st = _zero_state(50)
    for step in range(1, 30):
        p, st = oracle.adan(p, g, st, step, 2e-3)
    np.testing.assert_allclose(p, -29 * 2e-3 * g / (np.abs(g) + 1e-8), rtol=1e-11)


def test_adan_without_difference_term_is_adam():
    """b2 = 0 removes the difference average from the step and from the
    second moment: Adan is then Adam with betas (b1, b3) (torch.optim.Adam)."""
    torch = pytest.importorskip("torch")
    gen = np.random.default_rng(7)
    p = gen.standard_normal(64)
    t = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=3e-3, betas=(0.98, 0.99), eps=1e-8)
    st = _zero_state(64)
    for step in range(1, 9):
        g = gen.standard_normal(64)
        t.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        p, st = oracle.adan(p, g, st, step, 3e-3, betas=(0.98, 0.0, 0.99))
        np.testing.assert_allclose(p, t.detach().numpy(), rtol=1e-12, atol=1e-15)


def test_adan_equal_decays_is_one_average_of_the_extrapolated_gradient():
    """With b1 = b2 = b, m + b v is the exponential average (decay b) of the
    extrapolated gradient g + b (g - g_prev), the quantity whose square n
    averages (the reformulation in the Adan paper); computed here directly
    from that definition."""
    gen = np.random.default_rng(8)
    b, b3, lr, eps = 0.9, 0.99, 1e-3, 1e-8
    p = gen.standard_normal(32)
    q = p.copy()
    st = _zero_state(32)
    u = np.zeros(32)
    nn = np.zeros(32)
    g_prev = None
    for step in range(1, 12):
        g = gen.standard_normal(32)
        p, st = oracle.adan(p, g, st, step, lr, betas=(b, b, b3), eps=eps)
        ge = g + b * (g - (g if g_prev is None else g_prev))
        u = b * u + (1 - b) * ge
        nn = b3 * nn + (1 - b3) * ge * ge
        q = q - lr * (u / (1 - b ** step)) / (np.sqrt(nn / (1 - b3 ** step)) + eps)
        g_prev = g
        np.testing.assert_allclose(p, q, rtol=1e-11, atol=1e-14)


def test_lr_halving_schedule():
    """Sec. 4.1: 1e-3, halved every 20000 steps (1-based steps)."""
    assert oracle.lr_at(1e-3, 1, 20000) == 1e-3
    assert oracle.lr_at(1e-3, 20000, 20000) == 1e-3
    assert oracle.lr_at(1e-3, 20001, 20000) == 5e-4
    assert oracle.lr_at(1e-3, 50000, 20000) == 2.5e-4
    assert oracle.lr_at(1e-3, 50000, 0) == 1e-3


# --------------------------------------------------------------------------
# Rotation-scaling factorisation (Sec. 3.1, Eq. 2-3)
# --------------------------------------------------------------------------

def test_rs_to_chol_rebuilds_sigma():
    """L L^T of the returned Cholesky vector equals (R S)(R S)^T built with
    numpy matrix products, for angles in every quadrant and both orders of
    the scales."""
    gen = np.random.default_rng(11)
    rs = np.stack([gen.uniform(-4, 4, 300), gen.uniform(0.3, 9, 300), gen.uniform(0.3, 9, 300)], axis=1)
    L = oracle.rs_to_chol(rs).astype(np.float64)
    for i in range(300):
        th, s1, s2 = rs[i]
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        A = R @ np.diag([s1, s2])
        Lm = np.array([[L[i, 0], 0.0], [L[i, 1], L[i, 2]]])
        np.testing.assert_allclose(Lm @ Lm.T, A @ A.T, rtol=2e-6, atol=2e-6 * (A @ A.T).max())
        assert L[i, 0] > 0 and L[i, 2] > 0


@pytest.mark.parametrize("shift", [0.0, 0.5])
def test_rs_gradients_match_finite_differences(shift):
    """Central differences of the FP64 loss in (theta, s1, s2), support held
    fixed, against the chained analytic gradients (shift = App. C.1's +0.5
    on the scales)."""
    W, H, T, n = 24, 20, 8, 6
    means, _, col = synth.init_gaussians(n, W, H, 47)
    gen = np.random.default_rng(47)
    rs = np.stack([gen.uniform(-1.5, 1.5, n), gen.uniform(1.0, 5.0, n), gen.uniform(1.0, 5.0, n)], axis=1)
    target = synth.image(W, H, 47, n_blobs=5)
    r = oracle.rs_forward_backward(means, rs, col, target, T, shift=shift)
    ids, ranges = r["ids"], r["ranges"]

    def loss_at(x):
        y = x.copy()
        y[:, 1:] += shift
        out = oracle.render(means, oracle.rs_to_chol(y), col, ids, ranges, W, H, T)
        return oracle.loss(out, target)[0]

    num = np.zeros_like(rs)
    for idx in np.ndindex(rs.shape):
        def central(h):
            a, b = rs.copy(), rs.copy()
            a[idx] += h
            b[idx] -= h
            return (loss_at(a) - loss_at(b)) / (2 * h)
        # the render rounds the Cholesky vector to FP32: a step of 1e-2 keeps
        # that rounding far below the signal; Richardson removes the h^2 term
        h = 1e-2
        num[idx] = (4 * central(h / 2) - central(h)) / 3
    np.testing.assert_allclose(r["grads_rs"], num, rtol=3e-4, atol=1e-4 * np.abs(num).max())


def test_rs_special_cases():
    """Closed forms of Eq. 2-3: theta = 0 gives Sigma = diag(s1^2, s2^2), so
    L = (|s1|, 0, |s2|); a round Gaussian (s1 = s2) has L = (s, 0, s) at any
    angle and dL/dtheta = 0; theta and theta + pi give the same Sigma and
    the same chained gradient."""
    gen = np.random.default_rng(12)
    s = np.stack([gen.uniform(0.3, 9, 50), gen.uniform(0.3, 9, 50)], axis=1)
    L0 = oracle.rs_to_chol(np.stack([np.zeros(50), s[:, 0], s[:, 1]], axis=1))
    np.testing.assert_array_equal(L0, np.stack([s[:, 0], np.zeros(50), s[:, 1]], axis=1).astype(np.float32))
    th = gen.uniform(-4, 4, 50)
    Lr = oracle.rs_to_chol(np.stack([th, s[:, 0], s[:, 0]], axis=1)).astype(np.float64)
    np.testing.assert_allclose(Lr[:, 0], s[:, 0], rtol=1e-7)
    np.testing.assert_allclose(Lr[:, 2], s[:, 0], rtol=1e-7)
    assert np.all(np.abs(Lr[:, 1]) <= 1e-6 * s[:, 0])
    g_sigma = gen.normal(size=(50, 3))
    g_round = oracle.rs_chain(np.stack([th, s[:, 0], s[:, 0]], axis=1), g_sigma)
    np.testing.assert_array_equal(g_round[:, 0], 0.0)
    rs = np.stack([th, s[:, 0], s[:, 1]], axis=1)
    rs_pi = rs.copy()
    rs_pi[:, 0] += np.pi
    np.testing.assert_allclose(oracle.rs_to_chol(rs_pi), oracle.rs_to_chol(rs), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(oracle.rs_chain(rs_pi, g_sigma), oracle.rs_chain(rs, g_sigma), rtol=1e-9,
                               atol=1e-9 * np.abs(oracle.rs_chain(rs, g_sigma)).max())
