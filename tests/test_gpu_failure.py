"""Failure paths on the GPU, in forms that fault, trap or hang nothing.

- A bounded wait that runs out: with a wait limit of a few hundred clock
  cycles the dense solvers' ordinary waits (TMA ring, accumulator hand-offs,
  grid barriers) cannot complete in time, so every CTA records the error
  word, drains its copies and MMAs, frees its tensor memory and returns.
  Every query must report HOPF_Q_ABORTED, and the next call on the same
  handle, with the default limit, must give the usual results.
- Device allocation failure: an allocator that refuses after a few requests
  makes hopf_create return HOPF_ENOMEM, having returned every block it took.
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


@pytest.mark.parametrize("precision", ["MIXED", "SPLIT", "FP32"])
def test_wait_limit_aborts_then_recovers(hg, orc, precision):
    import torch
    n, B = 256, 600
    A, Q, s = wl.spd_matrix(15101, 15102, n)
    w = wl.uniform(15103, n, 0.5, 1.5)
    x = torch.tensor(wl.normal(15104, B * n, 2.0).reshape(B, n).astype(np.float32), device="cuda")
    t = torch.tensor(wl.uniform(15105, B, 0.1, 3.0).astype(np.float32), device="cuda")
    h = hg.Hopf(A, hg.H_WL1, w=w, tol=1e-13, max_iter=2000, precision=getattr(hg, "P_" + precision))
    ref = h.eval(x, t)
    torch.cuda.synchronize()
    ref = {k: v.clone() for k, v in ref.items()}
    assert (ref["status"].cpu().numpy() == hg.Q_OK).all()
    h.set_wait_limit(200)
    bad = h.eval(x, t)
    torch.cuda.synchronize()
    assert (bad["status"].cpu().numpy() == hg.Q_ABORTED).all()
    h.set_wait_limit(0)
    again = h.eval(x, t)
    torch.cuda.synchronize()
    for key in ("phi", "grad", "iters", "status"):
        assert torch.equal(again[key], ref[key]), key


def test_allocator_failure_is_enomem(hg):
    import torch
    taken = {}
    budget = [3]
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

    def alloc(nbytes, ctx):
        if budget[0] <= 0:
            return None
        budget[0] -= 1
        t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device="cuda")
        taken[t.data_ptr()] = t
        return t.data_ptr()

    def release(ptr, ctx):
        taken.pop(ptr, None)

    fa, ff = ALLOC(alloc), FREE(release)
    L = hg.lib()
    assert L.hopf_set_allocator(ctypes.cast(fa, ctypes.c_void_p), ctypes.cast(ff, ctypes.c_void_p), None) == 0
    try:
        A, Q, s = wl.spd_matrix(15201, 15202, 200)
        with pytest.raises(hg.HopfError) as e:
            hg.Hopf(A, hg.H_L1, tol=1e-12, max_iter=100, precision=hg.P_MIXED)
        assert e.value.status == hg.HOPF_ENOMEM
        assert not taken  # every block it took was given back
        budget[0] = 1000
        h = hg.Hopf(A, hg.H_L1, tol=1e-12, max_iter=100, precision=hg.P_MIXED)
        assert taken
        h.close()
        assert not taken
    finally:
        assert L.hopf_set_allocator(None, None, None) == 0
    torch.cuda.synchronize()
