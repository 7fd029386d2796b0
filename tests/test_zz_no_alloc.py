"""gi_bin_tiles_noalloc: binning without any device allocation.

Callers that cannot allocate device memory themselves (code living inside
another framework's memory pool, loops that must not pay for an
allocation's synchronisation, fixed-budget deployments) use this entry
point; its scratch is a fixed array inside the library. These tests call it
through the C ABI and require exactly the outputs of gi_bin_tiles (binning is
integer work, compared bit for bit), on consecutive calls with different
inputs, and check that oversized requests are refused before any launch.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_08551_gb300 import _lib
    return _lib.load()


def _img(W, H, T):
    from paper_2403_08551_gb300 import _lib
    return _lib.GIImage(W, H, T)


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _project(lib, W, H, T, n, seed):
    means, chol, color = (torch.from_numpy(a).cuda() for a in synth.init_gaussians(n, W, H, seed))
    rec = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    rect = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    cnt = torch.empty((n,), dtype=torch.int32, device="cuda")
    assert lib.gi_project(_p(means), _p(chol), _p(color), n, _img(W, H, T), _p(rec), _p(rect), _p(cnt),
                          _stream()) == 0
    return rec, rect, cnt


def _bin(lib, rec, rect, cnt, W, H, T, cap, noalloc):
    n = cnt.shape[0]
    tw, th = (W + T - 1) // T, (H + T - 1) // T
    keys = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    ids = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    ranges = torch.full((tw * th, 2), -7, dtype=torch.int32, device="cuda")
    recb = torch.zeros((cap, 8), dtype=torch.float32, device="cuda")
    pair_off = torch.empty((n + 1,), dtype=torch.int64, device="cuda")
    k = torch.empty((1,), dtype=torch.int64, device="cuda")
    if noalloc:
        rc = lib.gi_bin_tiles_noalloc(_p(rect), _p(cnt), _p(rec), n, _img(W, H, T), cap, _p(keys), _p(ids),
                                      _p(ranges), _p(recb), _p(pair_off), _p(k), _stream())
    else:
        nb = ctypes.c_size_t(0)
        assert lib.gi_bin_workspace_size(n, _img(W, H, T), cap, ctypes.byref(nb)) == 0
        ws = torch.empty((nb.value,), dtype=torch.uint8, device="cuda")
        rc = lib.gi_bin_tiles(_p(rect), _p(cnt), _p(rec), n, _img(W, H, T), cap, _p(ws), nb.value, _p(keys),
                              _p(ids), _p(ranges), _p(recb), _p(pair_off), _p(k), _stream())
    assert rc == 0, lib.gi_last_error()
    torch.cuda.synchronize()
    bits = ctypes.c_uint32(0)
    assert lib.gi_device_errors(ctypes.byref(bits), 1, _stream()) == 0
    K = int(k.item())
    Kv = min(K, cap)
    return dict(K=K, bits=bits.value, keys=keys[:Kv].cpu().numpy(), ids=ids[:Kv].cpu().numpy(),
                ranges=ranges.cpu().numpy(), recb=recb[:Kv].cpu().numpy().view(np.uint32),
                pair_off=pair_off.cpu().numpy())


def _same(a, b):
    assert a["K"] == b["K"] and a["bits"] == b["bits"]
    for key in ("keys", "ids", "ranges", "recb", "pair_off"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)


# (W, H, T, n, seed, capacity): 256 and 273 tiles take the count-matrix
# path; 768x512 at T = 8 (6144 tiles) and 1400x700 at T = 16 (3872 tiles)
# take the radix path, which reuses the array's look-back words, digit
# histograms and tickets at other offsets than the count-matrix layout.
CM_A = (256, 256, 16, 2000, 0, 40000)
CM_B = (161, 97, 8, 700, 7, 30000)
RADIX_A = (768, 512, 8, 20000, 11, 400000)
RADIX_B = (1400, 700, 16, 6000, 12, 200000)


def test_noalloc_matches_bin_tiles_on_consecutive_calls(lib):
    # Workloads back to back, alternating the two binning paths, each case
    # twice in a row: no call may see state another left in the shared array.
    for (W, H, T, n, seed, cap) in [CM_A, RADIX_A, CM_B, RADIX_B, CM_A, RADIX_A]:
        rec, rect, cnt = _project(lib, W, H, T, n, seed)
        ref = _bin(lib, rec, rect, cnt, W, H, T, cap, noalloc=False)
        first = _bin(lib, rec, rect, cnt, W, H, T, cap, noalloc=True)
        second = _bin(lib, rec, rect, cnt, W, H, T, cap, noalloc=True)
        assert 0 < ref["K"] <= cap and ref["bits"] == 0
        _same(ref, first)
        _same(ref, second)


def test_noalloc_capacity_shortfall_matches_bin_tiles(lib):
    # A capacity below the pair count: both entry points report the true K,
    # raise the capacity bit and bin the same first pairs, on either path.
    for (W, H, T, n, seed, _) in [CM_A, RADIX_A]:
        rec, rect, cnt = _project(lib, W, H, T, n, seed)
        K = int(cnt.to(torch.int64).sum().item())
        cap = K // 2
        ref = _bin(lib, rec, rect, cnt, W, H, T, cap, noalloc=False)
        got = _bin(lib, rec, rect, cnt, W, H, T, cap, noalloc=True)
        assert ref["K"] == K and ref["bits"] & 1
        _same(ref, got)


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    from paper_2403_08551_gb300 import _lib
    dummy = torch.zeros((64,), dtype=torch.int64, device="cuda")
    p = _p(dummy)
    rc = lib.gi_bin_tiles_noalloc(p, p, p, 10, _img(64, 64, 16), 524288 + 1, p, p, p, p, p, p, _stream())
    assert rc == 1 and b"capacity" in lib.gi_last_error()
    rc = lib.gi_bin_tiles_noalloc(p, p, p, 262144 + 1, _img(64, 64, 16), 1000, p, p, p, p, p, p, _stream())
    assert rc == 1 and b"n =" in lib.gi_last_error()
    assert _lib.STATUS[rc] == "GI_ERR_INVALID_ARG"
