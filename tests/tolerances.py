"""Tolerances of the GPU-vs-oracle parity tests, stated once.

Pixels (Sec. 3.2, Eq. 7): |C - C_ref| <= PIX_TOL * max(1, |C_ref|) (the
weighted colours are unbounded, so early renders exceed 1).

Gradients (App. A), per parameter group (positions, covariance, colour and,
where present, opacity):

    |g - g_ref| <= max(REL * max(|g_ref|, FLOOR * max|g_ref|),    (relative)
                       COND_ULPS * U32 * g_abs)                   (conditioning)

g_abs is the oracle's gradient with every pixel term replaced by its
magnitude: the condition magnitude of the sum. A gradient that cancels most
of its terms cannot be computed in FP32 closer than a few units of roundoff
of those terms, whatever the order of summation, so the second bound is the
accuracy FP32 allows there. It exceeds the first only where the oracle's
condition ratio

    kappa = g_abs / max(|g_ref|, FLOOR * max|g_ref|)

is above KAPPA_MIN = REL / (COND_ULPS * U32) ~ 105, i.e. for sums that cancel
more than two decimal digits. Such elements are a small minority: at most
CLAUSE_SHARE_MAX of a group's elements may fall outside the relative bound
(one constant for every workload and mode). Every check records the share it
used next to the share of elements with kappa > KAPPA_MIN (the most it could
use); tests/conftest.py prints them at the end of the run.

The sorted alpha-blending ablation multiplies up to a few hundred FP32
factors into each transmittance, so its conditioning bound uses
BLEND_COND_ULPS instead of COND_ULPS.
"""
import numpy as np

PIX_TOL = 1e-5
REL = 1e-4
FLOOR = 1e-3
U32 = 2.0 ** -24
COND_ULPS = 16
BLEND_COND_ULPS = 512
KAPPA_MIN = REL / (COND_ULPS * U32)
CLAUSE_SHARE_MAX = 1e-2

# (test id, group, used share, ill-conditioned share, elements), appended by check_group
CLAUSE_LOG = []


def _test_id():
    import os
    return os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0].split("::", 1)[-1]


def check_pixels(out, ref, tol=PIX_TOL):
    out = np.asarray(out, np.float64)
    err = np.abs(out - ref)
    bound = tol * np.maximum(1.0, np.abs(ref))
    assert np.all(err <= bound), f"max pixel err {err.max():.3e}"
    return float(err.max())


def check_group(g, ref, absref, label, cond_ulps=COND_ULPS, extra=None, exempt=None, rel_tol=REL, group=None):
    """Asserts one gradient group against the bound above and returns the
    tolerance array. extra: an additive allowance per element (the
    alpha-blending threshold ambiguity); exempt: a boolean mask of elements
    not counted against CLAUSE_SHARE_MAX (Gaussians ill-conditioned by
    construction in a test); rel_tol: the relative bound (REL for a
    parameter gradient); group: the name the end-of-run report files the
    share under (default: the last word of label)."""
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.abs(ref).max() if ref.size else 0.0
    base = np.maximum(np.abs(ref), FLOOR * scale)
    rel = rel_tol * base
    err = np.abs(g - ref)
    if extra is not None:
        err = np.maximum(err - extra, 0.0)
    if absref is None:
        tol = rel
        cond = np.zeros(err.shape, bool)
        ill = np.zeros(err.shape, bool)
    else:
        absref = np.asarray(absref, np.float64)
        ctol = cond_ulps * U32 * absref
        tol = np.maximum(rel, ctol)
        cond = (err > rel) & (err <= ctol)
        with np.errstate(divide="ignore", invalid="ignore"):
            ill = absref > (rel_tol / (cond_ulps * U32)) * base
    counted = cond if exempt is None else cond & ~np.broadcast_to(exempt, cond.shape)
    n = max(err.size, 1)
    used, ill_share = counted.sum() / n, ill.sum() / n
    CLAUSE_LOG.append((_test_id(), group or label.split()[-1], float(used), float(ill_share), int(err.size)))
    assert used <= CLAUSE_SHARE_MAX, f"{label}: {counted.sum()} of {err.size} elements need the conditioning bound"
    bad = err > tol
    assert not bad.any(), (f"{label}: {bad.sum()} of {bad.size} outside tolerance; worst "
                           f"{(err / np.maximum(tol, 1e-300)).max():.3e} of the bound")
    return tol


GROUPS = ((slice(0, 2), "means"), (slice(2, 5), "cov"), (slice(5, 8), "color"), (slice(8, 9), "opacity"))


def check_grads(g_gpu, g_ref, g_abs, label, cond_ulps=COND_ULPS, extra=None):
    """check_group over the column groups of [N, 8] (or [N, 9] with an
    opacity column) gradient arrays; returns the tolerance array."""
    tol = np.zeros_like(np.asarray(g_ref, np.float64))
    for sl, name in GROUPS:
        if sl.start >= g_ref.shape[1]:
            break
        tol[:, sl] = check_group(g_gpu[:, sl], g_ref[:, sl], None if g_abs is None else g_abs[:, sl],
                                 f"{label} {name}", cond_ulps, None if extra is None else extra[:, sl])
    return tol
