"""The allocation-free closest-point entry point, called through the C ABI.

It exists for callers that may not call cudaMalloc once running (a controller
querying obstacle distances at a fixed rate, a fixed memory budget, a host
without an allocator for this library): its scratch is one static 8 MiB device
array.  Its results must match hopf_union_closest (same kernels, caller-owned
workspace) on two calls in a row, and oversized requests must be refused.
This file is collected last so that, if it fails, a run stopping at the first
failure has already run every other test; it also passes on its own in a fresh
process (the first call there performs the per-device address lookup).
"""
import ctypes

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1605_01799_gb300 as pkg
    pkg.lib()
    return pkg


def _outs(torch, B, n):
    return {"dist": torch.empty(B, dtype=torch.float32, device="cuda"),
            "closest": torch.empty(B, n, dtype=torch.float32, device="cuda"),
            "argmin": torch.empty(B, dtype=torch.int32, device="cuda"),
            "newton": torch.empty(B, dtype=torch.int32, device="cuda"),
            "status": torch.empty(B, dtype=torch.uint8, device="cuda")}


def test_noalloc_matches_workspace_version_twice(hg):
    import torch
    n, K, B = 96, 8, 300
    d = wl.ellipsoid_union(n=n, K=K, batch=B, w=33)
    parts = [hg.Hopf(d["a"][k], hg.H_L2, centre=d["centres"][k], tol=1e-12, max_iter=5000,
                     precision=hg.P_FP32, stop_rule=hg.STOP_UREL) for k in range(K)]
    x = torch.tensor(d["x"], device="cuda")
    ref = hg.union_closest(parts, x, s_tol=1e-6, max_newton=60)
    arr = (ctypes.c_void_p * K)(*[p.handle.value for p in parts])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = hg.lib()
    for call in range(2):
        o = _outs(torch, B, n)
        st = L.hopf_union_closest_noalloc(arr, K, B, ctypes.c_void_p(x.data_ptr()), 1e-6, 60,
                                          ctypes.c_void_p(o["dist"].data_ptr()),
                                          ctypes.c_void_p(o["closest"].data_ptr()),
                                          ctypes.c_void_p(o["argmin"].data_ptr()),
                                          ctypes.c_void_p(o["newton"].data_ptr()),
                                          ctypes.c_void_p(o["status"].data_ptr()), stream)
        assert st == hg.HOPF_OK, L.hopf_last_error()
        torch.cuda.synchronize()
        dist, rd = o["dist"].cpu().numpy(), ref["dist"].cpu().numpy()
        # the tolerances of the closest-point parity test
        assert np.abs(dist - rd).max() <= 1e-5 * max(1, np.abs(rd).max()), call
        cl, rc = o["closest"].cpu().numpy(), ref["closest"].cpu().numpy()
        assert np.abs(cl - rc).max() <= 1e-3 * max(1, np.abs(rc).max()), call
        assert (o["argmin"].cpu().numpy() == ref["argmin"].cpu().numpy()).all(), call
        assert (o["status"].cpu().numpy() == ref["status"].cpu().numpy()).all(), call


def test_noalloc_rejects_oversized_batch(hg):
    import torch
    n, K = 8, 64
    parts = [hg.Hopf(np.ones(n), hg.H_L2, tol=1e-10, max_iter=100, precision=hg.P_FP32,
                     stop_rule=hg.STOP_UREL) for _ in range(K)]
    B = 10000  # 640,000 query-part pairs: more than the static scratch holds
    x = torch.full((B, n), 3.0, dtype=torch.float32, device="cuda")
    arr = (ctypes.c_void_p * K)(*[p.handle.value for p in parts])
    o = _outs(torch, B, n)
    st = hg.lib().hopf_union_closest_noalloc(arr, K, B, ctypes.c_void_p(x.data_ptr()), 1e-6, 20,
                                             ctypes.c_void_p(o["dist"].data_ptr()), None,
                                             ctypes.c_void_p(o["argmin"].data_ptr()), None, None,
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == hg.HOPF_EINVAL
    assert b"static scratch" in hg.lib().hopf_last_error()


def _need(K, B):
    """Scratch bytes of one call: per query-part pair an FP64 phi, an FP32 s,
    an int32 count and a status byte, plus a 4-byte slot per query; each of
    the five regions rounded up to 256 bytes."""
    r = lambda v: (v + 255) // 256 * 256
    b = B * K
    return r(8 * b) + r(4 * b) + r(4 * b) + r(b) + r(4 * B)


def test_noalloc_limit_with_one_part(hg):
    """With one part the bound is batch * 21 bytes: the largest batch that
    fits runs (and matches hopf_union_closest on sampled queries), the next
    one is refused before anything is launched."""
    import torch
    cap = 8 << 20
    B = cap // 21
    while _need(1, B + 1) <= cap:
        B += 1
    while _need(1, B) > cap:
        B -= 1
    assert 398000 < B < 400000
    n = 2
    part = hg.Hopf(np.array([1.0, 4.0]), hg.H_L2, tol=1e-12, max_iter=2000, precision=hg.P_FP32,
                   stop_rule=hg.STOP_UREL)
    arr = (ctypes.c_void_p * 1)(part.handle.value)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    xs = wl.normal(3301, (B + 1) * n, 4.0).reshape(B + 1, n).astype(np.float32)
    xs[:, 0] += np.where(xs[:, 0] >= 0, 2.0, -2.0).astype(np.float32)  # outside the ellipse |x1| <= 1
    x = torch.tensor(xs, device="cuda")
    L = hg.lib()
    for batch, want in ((B + 1, hg.HOPF_EINVAL), (B, hg.HOPF_OK)):
        o = _outs(torch, batch, n)
        st = L.hopf_union_closest_noalloc(arr, 1, batch, ctypes.c_void_p(x.data_ptr()), 1e-6, 60,
                                          ctypes.c_void_p(o["dist"].data_ptr()),
                                          ctypes.c_void_p(o["closest"].data_ptr()),
                                          ctypes.c_void_p(o["argmin"].data_ptr()), None,
                                          ctypes.c_void_p(o["status"].data_ptr()), stream)
        assert st == want, (batch, L.hopf_last_error())
    torch.cuda.synchronize()
    idx = np.array([0, 1, B // 2, B - 1])
    ref = hg.union_closest([part], x[:B][torch.tensor(idx, device="cuda")], s_tol=1e-6, max_newton=60)
    torch.cuda.synchronize()
    rd = ref["dist"].cpu().numpy()
    assert np.abs(o["dist"].cpu().numpy()[idx] - rd).max() <= 1e-5 * max(1, np.abs(rd).max())
