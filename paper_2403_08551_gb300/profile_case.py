"""A few fit steps of one fitting mode on the 768x512, 70,000-Gaussian
synthetic workload, for profilers: the steps run eagerly (one launch per
kernel), after `--warmup` steps, and the mean device time per step is
printed. Run from the repository root:

    python -m paper_2403_08551_gb300.profile_case --mode blend --steps 3

Modes: merged (the paper's 8-parameter form, Adam), separate (colour and
opacity kept apart, accumulated summation), blend (sorted alpha-blending),
paper (App. C.1 parameters with Adan), rs (rotation-scaling covariance with
the paper's parameters and Adan), codec (b = 6, 2 x 8 RVQ fine-tuning),
batch (64 synthetic images of uneven sizes, 5k-70k Gaussians each, fitted in
one launch per stage at tile 16, render split 4), vq (the codec's RVQ decode
of 64 x 50,000 Gaussians, FP16 means and 2 x 256-entry codebooks, into
preallocated outputs; `--steps` calls)."""
import argparse
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.getcwd())

MODES = ("merged", "separate", "blend", "paper", "rs", "codec", "batch", "vq")


def run_vq(gi, steps: int, warmup: int) -> int:
    import synth
    w = synth.workload("c4_768x512_50k")
    nb = 64 * w.n
    cb = torch.from_numpy(synth.codebooks(4000)).cuda()
    idx = torch.from_numpy(synth.vq_indices(nb, 4001)).cuda()
    m16 = torch.from_numpy(np.tile(w.means, (64, 1)).astype(np.float16)).cuda()
    out = tuple(torch.empty((nb, k), dtype=torch.float32, device="cuda") for k in (2, 3, 3))
    for _ in range(warmup):
        gi.vq_decode(m16, idx, cb, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        gi.vq_decode(m16, idx, cb, out=out)
    e1.record()
    e1.synchronize()
    err = gi.device_errors(clear=True)
    ms = e0.elapsed_time(e1) / max(1, steps)
    print(f"vq: {ms:.4f} ms per decode of {nb} Gaussians ({nb * 40 / ms / 1e6:.0f} GB/s), device errors {err}")
    return 1 if err else 0


def make_fit(gi, mode: str):
    import synth
    if mode == "batch":
        ws = synth.batch_workload(64)
        tg = [torch.from_numpy(w.target).cuda() for w in ws]
        pr = [torch.from_numpy(np.concatenate([w.means, w.chol, w.color], axis=1).astype(np.float32)).cuda()
              for w in ws]
        return gi.Fit(tg, pr, tile=16, lr=(1e-3, 1e-2, 1e-2), render_split=4, use_graph=False)
    w = synth.workload("c1_768x512_70k")
    tgt = torch.from_numpy(w.target).cuda()
    p = np.concatenate([w.means, w.chol, w.color], axis=1).astype(np.float64)
    kw = dict(tile=16, lr=(1e-3, 1e-2, 1e-2), capacity_factor=4.0, use_graph=False)
    if mode in ("separate", "blend"):
        p[:, 5:8] *= 2.0
        kw.update(opacity=mode, opacity_logits=[torch.zeros(w.n, device="cuda")])
    elif mode in ("paper", "rs", "codec"):
        p[:, 0:2] = np.arctanh(np.clip(p[:, 0:2] / [w.W, w.H] * 2 - 1, -0.999, 0.999))
        if mode == "rs":
            p[:, 2:5] = synth.init_gaussians_rs(w.n, w.W, w.H, 0)[1]
            p[:, 3:5] -= 0.5
        else:
            p[:, 2] -= 0.5
            p[:, 4] -= 0.5
        kw.update(lr=(1e-3, 1e-3, 1e-3), param_mode="paper", optimizer="adan",
                  cov="rs" if mode == "rs" else "cholesky")
    pt = torch.from_numpy(p.astype(np.float32)).cuda()
    if mode == "codec":
        kw["codec"] = gi.codec_init(pt, param_mode="paper")
    return gi.Fit([tgt], [pt], **kw)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--mode", choices=MODES, default="merged")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    args = ap.parse_args()
    import paper_2403_08551_gb300 as gi
    if args.mode == "vq":
        return run_vq(gi, args.steps, args.warmup)
    fit = make_fit(gi, args.mode)
    fit.step(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fit.step(args.steps)
    e1.record()
    e1.synchronize()
    err = gi.device_errors(clear=True)
    print(f"{args.mode}: {e0.elapsed_time(e1) / max(1, args.steps):.4f} ms/step over {args.steps} eager steps, "
          f"mse {fit.mse()[0]:.6g}, device errors {err}")
    fit.close()
    return 1 if err else 0


if __name__ == "__main__":
    sys.exit(main())
