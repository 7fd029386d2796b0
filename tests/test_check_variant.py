"""The bounds-checking build (-DGI_CHECK_BOUNDS): it compiles and exports the
same C ABI as the release build, and on a GPU it runs a forward + backward
with no device error and bit-identical results."""
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _exports(path):
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    return sorted(set(re.findall(r" T (gi_\w+)", out)))


def test_check_build_exports_the_abi():
    from paper_2403_08551_gb300 import build
    rel = build.build()
    chk = build.build(variant="check")
    assert chk != rel and os.path.exists(chk)
    assert _exports(chk) == _exports(rel) and len(_exports(rel)) > 10


CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
import synth, paper_2403_08551_gb300 as gi
gi.load()
W, H, T, n = 161, 97, 16, 500
target = torch.from_numpy(synth.image(W, H, 2, n_blobs=20)).cuda()
m, l, c = (torch.from_numpy(a).cuda() for a in synth.init_gaussians(n, W, H, 2))
rec, rect, cnt = gi.project(m, l, c, W, H, T)
bins = gi.bin_tiles(rect, cnt, rec, W, H, T)
out, dl, loss = gi.render(bins, W, H, T, target=target, want_dl=True)
gm, gl, gc, _ = gi.render_backward(bins, rect, cnt, l, dl, W, H, T)
torch.cuda.synchronize()
assert gi.device_errors(clear=True) == 0
np.savez({out_path!r}, out=out.cpu().numpy(), gm=gm.cpu().numpy(), gl=gl.cpu().numpy(), gc=gc.cpu().numpy(),
         ids=bins.ids[:bins.K].cpu().numpy())
"""


@pytest.mark.gpu
def test_check_build_runs_clean_and_identical(tmp_path):
    from paper_2403_08551_gb300 import build
    build.build()
    build.build(variant="check")
    res = {}
    for variant in ("release", "check"):
        path = str(tmp_path / f"{variant}.npz")
        env = dict(os.environ, GI_LIB_VARIANT=variant)
        r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, out_path=path)], env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        res[variant] = np.load(path)
    for k in ("out", "gm", "gl", "gc", "ids"):
        np.testing.assert_array_equal(res["release"][k], res["check"][k])
