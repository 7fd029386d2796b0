"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (written where used):
  support rect, counts, binning keys/ids/ranges/pair offsets: bit-exact;
  rendered pixels: |C - C_ref| <= 1e-5 * max(1, |C_ref|);
  gradients, per parameter group:
      |g - g_ref| <= 1e-4 * max(|g_ref|, 1e-3 ||g_ref||_inf)
   or |g - g_ref| <= 16 u |g|_abs   (u = 2^-24, the FP32 unit roundoff;
      |g|_abs = the oracle's sum over pixels of |per-pixel contribution|),
   the second clause being the error bound of an FP32 sum whose terms cancel;
   at most 0.1 % of the elements may rely on it;
  codec decode: bit-exact.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tolerances import PIX_TOL, REL as GRAD_TOL, check_group


@pytest.fixture(scope="module")
def gi():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_08551_gb300 as m
    m.load()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_pixels(out, ref):
    out = out.detach().cpu().numpy().astype(np.float64)
    err = np.abs(out - ref)
    tol = PIX_TOL * np.maximum(1.0, np.abs(ref))
    assert np.all(err <= tol), f"max pixel err {err.max():.3e}"
    return err.max()


def check_grads(g, ref, name, absref=None, rel=GRAD_TOL, cond_rows=None):
    """The gradient bound of tests/tolerances.py on one gradient; cond_rows:
    Gaussians ill-conditioned by construction, not counted against the
    conditioning clause's share."""
    exempt = None
    if cond_rows is not None:
        exempt = np.zeros((ref.shape[0], 1), bool)
        exempt[cond_rows] = True
    check_group(g.detach().cpu().numpy(), ref, absref, name, exempt=exempt, rel_tol=rel)


def run_gpu(gi, means, chol, color, target, T, capacity=None):
    H, W, _ = target.shape
    m, l, c = dev(means), dev(chol), dev(color)
    rec, rect, cnt = gi.project(m, l, c, W, H, T)
    bins = gi.bin_tiles(rect, cnt, rec, W, H, T, capacity=capacity)
    out, dl, loss = gi.render(bins, W, H, T, target=dev(target), want_dl=True)
    gm, gl, gc, gq = gi.render_backward(bins, rect, cnt, l, dl, W, H, T, want_conic=True)
    torch.cuda.synchronize()
    return dict(rec=rec, rect=rect, cnt=cnt, bins=bins, out=out, dl=dl, loss=loss, gm=gm, gl=gl, gc=gc, gq=gq)


CASES = [
    # (W, H, n, T, seed): several tiles and ragged edges
    (256, 256, 2000, 16, 0),   # the small parity workload (256x256, 2k, 16x16 tiles)
    (100, 70, 300, 8, 1),
    (161, 97, 500, 16, 2),
    (130, 99, 400, 32, 3),
    (64, 48, 1, 16, 4),
]


@pytest.mark.parametrize("W,H,n,T,seed", CASES)
def test_forward_backward_matches_oracle(gi, W, H, n, T, seed):
    target = synth.image(W, H, seed, n_blobs=20)
    means, chol, color = synth.init_gaussians(n, W, H, seed)
    g = run_gpu(gi, means, chol, color, target, T)
    ref = oracle.forward_backward(means, chol, color, target, T)
    # formation: support rectangles and counts bit-exact; the record's scaled
    # inverse Cholesky factor M (M^T M = log2(e)/2 Sigma^-1) to FP32 rounding
    np.testing.assert_array_equal(g["rect"].cpu().numpy(), ref["rect"])
    np.testing.assert_array_equal(g["cnt"].cpu().numpy(), ref["cnt"])
    q = oracle.conic(chol)
    rec = g["rec"].cpu().numpy().astype(np.float64)
    live = ref["cnt"] > 0
    m11, m21, m22 = rec[live, 2], rec[live, 3], rec[live, 4]
    h = 0.5 * oracle.LOG2E
    np.testing.assert_allclose(m11 * m11 + m21 * m21, q[live, 0] * h, rtol=1e-6)
    np.testing.assert_allclose(m22 * m22, q[live, 2] * h, rtol=1e-6)
    np.testing.assert_allclose(m21 * m22, q[live, 1] * h, rtol=1e-6, atol=1e-6 * np.abs(q[live, 1] * h).max())
    np.testing.assert_allclose(m11, np.sqrt(h) / chol[live, 0].astype(np.float64), rtol=1e-6)
    # binning bit-exact
    b = g["bins"]
    K = ref["ids"].shape[0]
    assert b.K == K
    np.testing.assert_array_equal(b.ids[:K].cpu().numpy().astype(np.uint32), ref["ids"])
    np.testing.assert_array_equal(b.ranges.cpu().numpy(), ref["ranges"])
    np.testing.assert_array_equal(b.pair_off.cpu().numpy(), ref["pair_off"])
    tw, th = oracle.tiles(W, H, T)
    key_ref = np.repeat(np.arange(tw * th), ref["ranges"][:, 1] - ref["ranges"][:, 0])
    np.testing.assert_array_equal(b.keys[:K].cpu().numpy(), key_ref)
    # render, loss, dL/dC
    check_pixels(g["out"], ref["out"])
    assert float(g["loss"].item()) == pytest.approx(ref["loss"], rel=1e-5)
    np.testing.assert_allclose(g["dl"].cpu().numpy(), ref["dldc"], rtol=1e-4,
                               atol=1e-4 * np.abs(ref["dldc"]).max())
    # gradients
    ab = ref["grads"]["abs"]
    check_grads(g["gm"], ref["grads"]["means"], "means", ab["means"])
    check_grads(g["gl"], ref["grads"]["chol"], "chol", ab["chol"])
    check_grads(g["gc"], ref["grads"]["color"], "color", ab["color"])
    # The conic gradient is an intermediate, not a parameter: dL/dB sums
    # e dx dy over pixels with strong cancellation in FP32; checked at 3e-4.
    check_grads(g["gq"], ref["grads"]["conic"], "conic", rel=3e-4)


BIN_CASES = [
    # (W, H, n, T, seed, scale): both binning paths on either side of the
    # 2048-tile limit of the count-matrix path, several 128-Gaussian chunks
    # with a ragged last one, and wide Gaussians whose tiles are shared by
    # every lane of a warp.
    (1024, 512, 5000, 16, 21, 1.0),    # 2048 tiles: count matrix
    (1024, 528, 5000, 16, 22, 1.0),    # 2112 tiles: radix sort
    (300, 200, 1000, 8, 23, 6.0),      # 1026 tiles, wide Gaussians: count matrix
    (1400, 700, 3000, 16, 24, 6.0),    # 3872 tiles, wide Gaussians: radix sort
    (96, 96, 129, 32, 25, 1.0),        # 9 tiles, two chunks (one Gaussian in the second)
    (8192, 8192, 3000, 8, 26, 4.0),    # 1,048,576 tiles: 20-bit keys, three radix passes
]


@pytest.mark.parametrize("W,H,n,T,seed,scale", BIN_CASES)
def test_binning_paths_match_oracle(gi, W, H, n, T, seed, scale):
    means, chol, color = synth.init_gaussians(n, W, H, seed)
    chol = (chol * np.float32(scale)).astype(np.float32)
    rect_ref, cnt_ref = oracle.rect_rule(means, chol, color, W, H, T)
    ids_ref, ranges_ref, off_ref = oracle.bin_tiles(rect_ref, cnt_ref, W, H, T)
    rec, rect, cnt = gi.project(dev(means), dev(chol), dev(color), W, H, T)
    np.testing.assert_array_equal(rect.cpu().numpy(), rect_ref)
    bins = gi.bin_tiles(rect, cnt, rec, W, H, T)
    torch.cuda.synchronize()
    K = ids_ref.shape[0]
    assert bins.K == K
    np.testing.assert_array_equal(bins.ids[:K].cpu().numpy().astype(np.uint32), ids_ref)
    np.testing.assert_array_equal(bins.ranges.cpu().numpy(), ranges_ref)
    np.testing.assert_array_equal(bins.pair_off.cpu().numpy(), off_ref)
    tw, th = oracle.tiles(W, H, T)
    np.testing.assert_array_equal(bins.keys[:K].cpu().numpy(),
                                  np.repeat(np.arange(tw * th), ranges_ref[:, 1] - ranges_ref[:, 0]))
    # rec_binned[k] is the record of ids[k]
    rb = bins.rec_binned[:K].cpu().numpy()
    np.testing.assert_array_equal(rb, rec.cpu().numpy()[ids_ref.astype(np.int64)])


@pytest.mark.parametrize("W,H,n,T,seed,scale", BIN_CASES[:2])
def test_binning_records_at_16_byte_offsets(gi, W, H, n, T, seed, scale):
    """The ABI asks 16-byte alignment of rec and rec_binned; the binning
    moves each 32-byte record in one access only when both are 32-byte
    aligned. Records and binned records 16 bytes into their buffers (count
    matrix and radix path) give the same binned records."""
    import ctypes
    from paper_2403_08551_gb300 import _lib as L
    means, chol, color = synth.init_gaussians(n, W, H, seed)
    chol = (chol * np.float32(scale)).astype(np.float32)
    ids_ref, _, _ = oracle.bin_tiles(*oracle.rect_rule(means, chol, color, W, H, T), W, H, T)
    rec, rect, cnt = gi.project(dev(means), dev(chol), dev(color), W, H, T)
    K = ids_ref.shape[0]
    cap = K + 64
    img = L.GIImage(W, H, T)
    lib = L.load()
    sz = ctypes.c_size_t(0)
    L.check(lib.gi_bin_workspace_size(n, img, cap, ctypes.byref(sz)), "gi_bin_workspace_size")
    ws = torch.empty((sz.value + 256,), dtype=torch.uint8, device="cuda")
    rec_off = torch.empty((n * 8 + 4,), dtype=torch.float32, device="cuda")
    rec_off[4:] = rec.reshape(-1)
    rb_off = torch.full((cap * 8 + 4,), float("nan"), dtype=torch.float32, device="cuda")
    keys = torch.empty((cap,), dtype=torch.int32, device="cuda")
    ids = torch.empty((cap,), dtype=torch.int32, device="cuda")
    tw, th = oracle.tiles(W, H, T)
    ranges = torch.empty((tw * th, 2), dtype=torch.int32, device="cuda")
    pair_off = torch.empty((n + 1,), dtype=torch.int64, device="cuda")
    k_dev = torch.empty((1,), dtype=torch.int64, device="cuda")
    assert (rec_off[4:].data_ptr() % 32, rb_off[4:].data_ptr() % 32) == (16, 16)
    L.check(lib.gi_bin_tiles(L.ptr(rect), L.ptr(cnt), rec_off[4:].data_ptr(), n, img, cap, L.ptr(ws), sz.value,
                             L.ptr(keys), L.ptr(ids), L.ptr(ranges), rb_off[4:].data_ptr(), L.ptr(pair_off),
                             L.ptr(k_dev), L.stream_handle()), "gi_bin_tiles")
    torch.cuda.synchronize()
    assert int(k_dev.item()) == K
    rb = rb_off[4:].reshape(cap, 8)[:K].cpu().numpy()
    np.testing.assert_array_equal(rb, rec.cpu().numpy()[ids_ref.astype(np.int64)])
    assert gi.device_errors(clear=True) == 0


@pytest.mark.parametrize("l3", [1e-2, 1e-3, 1e-4])
def test_needle_gaussians(gi, l3):
    """Needle-shaped Gaussians (l1 = l2 = 8, l3 tiny: the short axis is about
    l3 px wide, Sigma's condition number ~ (16 / l3)^2) next to ordinary ones.
    The expanded quadratic form A dx^2 + 2B dx dy + C dy^2 cancels terms of
    order 1/l3^2 there and overflowed exp in long fits; sigma = 1/2 |L^-1 d|^2
    does not. Checked: every output and gradient is finite, the render and
    the other Gaussians' gradients meet the usual tolerances, and a needle's
    own gradients meet the bound its conditioning allows in FP32: rounding
    d = p - mu (|d| <= W) moves z2 = m21 dx + m22 dy by up to
    2^-23 W (|m21| + |m22|), so sigma log2(e) = z1^2 + z2^2 moves by up to
    2 z_max of that (z_max^2 = 30: smaller weights are below 2^-30) and each
    term of a gradient sum by ln 2 times that, relative to the term."""
    W, H, T = 128, 96, 16
    target = synth.image(W, H, 31, n_blobs=10)
    means, chol, color = synth.init_gaussians(200, W, H, 31)
    chol[:20] = np.array([8.0, 8.0, l3], np.float32)
    g = run_gpu(gi, means, chol, color, target, T)
    ref = oracle.forward_backward(means, chol, color, target, T)
    for key in ("out", "gm", "gl", "gc"):
        assert torch.isfinite(g[key]).all(), key
    check_pixels(g["out"], ref["out"])
    ab = ref["grads"]["abs"]
    others = np.arange(20, 200)
    for key, name in (("gm", "means"), ("gl", "chol"), ("gc", "color")):
        gg = g[key][20:]
        check_grads(gg, ref["grads"][name][others], name, ab[name][others])
        l = chol[:20].astype(np.float64)
        k = np.sqrt(0.5 * oracle.LOG2E)
        m_sum = k * np.abs(l[:, 1]) / np.abs(l[:, 0] * l[:, 2]) + k / np.abs(l[:, 2])
        rel_w = np.log(2.0) * 2 * np.sqrt(30.0) * 2.0 ** -23 * W * m_sum
        err = np.abs(g[key][:20].detach().cpu().numpy().astype(np.float64) - ref["grads"][name][:20])
        floor = 1e-3 * np.abs(ref["grads"][name]).max()
        bound = GRAD_TOL * np.maximum(np.abs(ref["grads"][name][:20]), floor) + rel_w[:, None] * ab[name][:20]
        assert np.all(err <= bound), f"needle {name}: worst err/bound {(err / bound).max():.3f}"


def test_backward_arbitrary_upstream(gi):
    """Backward with a seeded random dL/dC (not from an L2 loss)."""
    W, H, T, n = 120, 88, 16, 700
    means, chol, color = synth.init_gaussians(n, W, H, 11)
    G = synth.upstream_grad(W, H, 11)
    rect, cnt = oracle.rect_rule(means, chol, color, W, H, T)
    ref = oracle.backward(means, chol, color, rect, cnt, W, H, T, G.astype(np.float64))
    m, l, c = dev(means), dev(chol), dev(color)
    rec, rect_g, cnt_g = gi.project(m, l, c, W, H, T)
    bins = gi.bin_tiles(rect_g, cnt_g, rec, W, H, T)
    gm, gl, gc, _ = gi.render_backward(bins, rect_g, cnt_g, l, dev(G), W, H, T)
    check_grads(gm, ref["means"], "means", ref["abs"]["means"])
    check_grads(gl, ref["chol"], "chol", ref["abs"]["chol"])
    check_grads(gc, ref["color"], "color", ref["abs"]["color"])


def test_edge_cases(gi):
    """Culled, off-screen, degenerate and image-covering Gaussians; empty tiles."""
    W, H, T = 77, 45, 16
    means = np.array([[10, 10], [np.nan, 3], [-100, 10], [38, 22], [76.9, 44.9], [0, 0], [40, 20]], np.float32)
    chol = np.array([[2, 0, 2], [2, 0, 2], [2, 0, 2], [40, 5, 30], [1, -1, 0.5], [0, 1, 1], [1e-20, 0, 1e-20]],
                    np.float32)
    color = np.full((7, 3), 0.1, np.float32)
    target = synth.image(W, H, 12, n_blobs=3)
    g = run_gpu(gi, means, chol, color, target, T)
    ref = oracle.forward_backward(means, chol, color, target, T)
    np.testing.assert_array_equal(g["rect"].cpu().numpy(), ref["rect"])
    np.testing.assert_array_equal(g["cnt"].cpu().numpy(), ref["cnt"])
    np.testing.assert_array_equal(g["bins"].ids[:g["bins"].K].cpu().numpy().astype(np.uint32), ref["ids"])
    np.testing.assert_array_equal(g["bins"].ranges.cpu().numpy(), ref["ranges"])
    check_pixels(g["out"], ref["out"])
    for name, key in (("gm", "means"), ("gl", "chol"), ("gc", "color")):
        gg = g[name].cpu().numpy()
        assert np.all(np.isfinite(gg))
        assert np.all(gg[ref["cnt"] == 0] == 0)


def test_empty_set(gi):
    W, H, T = 40, 30, 8
    z2 = torch.zeros((0, 2), device="cuda")
    z3 = torch.zeros((0, 3), device="cuda")
    rec, rect, cnt = gi.project(z2, z3, z3, W, H, T)
    bins = gi.bin_tiles(rect, cnt, rec, W, H, T)
    assert bins.K == 0
    assert int(bins.ranges.abs().sum()) == 0
    out, _, _ = gi.render(bins, W, H, T)
    assert float(out.abs().sum()) == 0.0


def test_deterministic(gi):
    W, H, T, n = 200, 150, 16, 3000
    target = synth.image(W, H, 13, n_blobs=20)
    means, chol, color = synth.init_gaussians(n, W, H, 13)
    a = run_gpu(gi, means, chol, color, target, T)
    b = run_gpu(gi, means, chol, color, target, T)
    for k in ("out", "dl", "gm", "gl", "gc"):
        assert torch.equal(a[k], b[k]), k


def test_bounded_waits_give_up_and_report(gi):
    """Failure detection without a fault: a TMA-style mbarrier wait with no
    arrival and a spin on a flag nothing sets both stop after their limit and
    report it in the self-test's own status word; the context stays usable
    (a render afterwards is correct) and the library's error word is clean."""
    import time
    assert gi.device_errors(clear=True) == 0
    t0 = time.perf_counter()
    bits = gi.selftest_bounded_waits(2_000_000)  # 2 ms each
    assert time.perf_counter() - t0 < 30
    assert bits == 3
    assert gi.device_errors() == 0
    W, H, T, n = 96, 64, 16, 300
    means, chol, color = synth.init_gaussians(n, W, H, 41)
    out = gi.rasterize(dev(means), dev(chol), dev(color), W, H, T)
    torch.cuda.synchronize()
    rect, cnt = oracle.rect_rule(means, chol, color, W, H, T)
    ids, rg, _ = oracle.bin_tiles(rect, cnt, W, H, T)
    check_pixels(out, oracle.render(means, chol, color, ids, rg, W, H, T))


def test_capacity_overflow_reported(gi):
    W, H, T, n = 128, 128, 16, 500
    means, chol, color = synth.init_gaussians(n, W, H, 14)
    m, l, c = dev(means), dev(chol), dev(color)
    rec, rect, cnt = gi.project(m, l, c, W, H, T)
    K = int(cnt.sum().item())
    gi.device_errors(clear=True)
    with pytest.raises(gi.GIError):
        gi.bin_tiles(rect, cnt, rec, W, H, T, capacity=K // 2)
    assert gi.device_errors(clear=True) & 1  # GI_DEVERR_CAPACITY
    bins = gi.bin_tiles(rect, cnt, rec, W, H, T, capacity=K)
    assert bins.K == K
    assert gi.device_errors(clear=True) == 0


def test_autograd_function(gi):
    W, H, T, n = 96, 64, 16, 400
    target = dev(synth.image(W, H, 15, n_blobs=10))
    means, chol, color = synth.init_gaussians(n, W, H, 15)
    m = dev(means).requires_grad_()
    l = dev(chol).requires_grad_()
    c = dev(color).requires_grad_()
    out = gi.rasterize(m, l, c, W, H, T)
    loss = ((out - target) ** 2).mean()
    loss.backward()
    ref = oracle.forward_backward(means, chol, color, target.cpu().numpy(), T)
    ab = ref["grads"]["abs"]
    check_grads(m.grad, ref["grads"]["means"], "means", ab["means"])
    check_grads(l.grad, ref["grads"]["chol"], "chol", ab["chol"])
    check_grads(c.grad, ref["grads"]["color"], "color", ab["color"])


@pytest.mark.parametrize("n", [50000, 49999])  # four Gaussians per thread / one per thread
def test_vq_decode_bit_exact(gi, n):
    cb = synth.codebooks(4000)
    means = synth.init_gaussians(n, 768, 512, 4000)[0]
    x = synth.init_gaussians(n, 768, 512, 4001)
    idx = np.stack([oracle.rvq_encode(x[1], cb[0]), oracle.rvq_encode(x[2], cb[1])])
    m16 = means.astype(np.float16)
    rm, rl, rc = oracle.vq_decode(m16, idx, cb)
    gm, gl, gc = gi.vq_decode(dev(m16.view(np.int16)), dev(idx), dev(cb))
    for a, r in ((gm, rm), (gl, rl), (gc, rc)):
        np.testing.assert_array_equal(a.cpu().numpy().view(np.uint32), r.view(np.uint32))
    # three stages: FP64 accumulation, rounded once
    cb3 = np.concatenate([cb, synth.codebooks(4002)[:, 1:2]], axis=1)
    idx3 = synth.vq_indices(n, 4003, stages=3)
    rm, rl, rc = oracle.vq_decode(m16, idx3, cb3)
    gm, gl, gc = gi.vq_decode(dev(m16.view(np.int16)), dev(idx3), dev(cb3))
    for a, r in ((gl, rl), (gc, rc)):
        np.testing.assert_array_equal(a.cpu().numpy().view(np.uint32), r.view(np.uint32))


@pytest.mark.slow
@pytest.mark.parametrize("name,T", [("c1_768x512_70k", 16), ("c1_768x512_70k", 8), ("c2_2040x1356_200k", 16)])
def test_full_size_parity(gi, name, T):
    """Full-size workloads in the configuration the benchmark times: binning
    bit-exact, every pixel and every gradient against the oracle."""
    w = synth.workload(name)
    g = run_gpu(gi, w.means, w.chol, w.color, w.target, T)
    ref = oracle.forward_backward(w.means, w.chol, w.color, w.target, T)
    np.testing.assert_array_equal(g["rect"].cpu().numpy(), ref["rect"])
    K = ref["ids"].shape[0]
    assert g["bins"].K == K
    np.testing.assert_array_equal(g["bins"].ids[:K].cpu().numpy().astype(np.uint32), ref["ids"])
    np.testing.assert_array_equal(g["bins"].ranges.cpu().numpy(), ref["ranges"])
    check_pixels(g["out"], ref["out"])
    ab = ref["grads"]["abs"]
    check_grads(g["gm"], ref["grads"]["means"], "means", ab["means"])
    check_grads(g["gl"], ref["grads"]["chol"], "chol", ab["chol"])
    check_grads(g["gc"], ref["grads"]["color"], "color", ab["color"])
