"""Degenerate inputs at every entry point of the C ABI.

- An empty batch is a no-op that still writes the summed gradients (zero).
- A query at the centre, x = c: the Hopf objective of eq. 3.3 reduces to
  J*_0(v) + c0 + t H(v), which is >= c0 with equality only at v = 0, so
  phi = -c0 = J(c), grad phi = 0 and d phi/dt = -H(0) = 0 for every t >= 0,
  every initial data and every Hamiltonian.  Every step of split Bregman
  keeps the state at exactly zero there (shrink of 0, the prox of a norm at 0
  and the l2 shrink's guard at |z| = 0), so the bar is exact.
- Identical parts tie in the union, the maximum over Hamiltonians and the
  distance: the first index wins, with the single part's value.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N = 8
C0 = 0.75
CENTRE = np.arange(N, dtype=np.float64) / 8.0 - 0.375  # exact in FP32


@pytest.fixture(scope="module")
def hg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1605_01799_gb300 as pkg
    pkg.lib()
    return pkg


def _dense_A():
    return 2.0 * np.eye(N) + 0.1 * np.ones((N, N))


def _anorm_M():
    return 1.5 * np.eye(N) + 0.2 * np.ones((N, N))


def test_empty_batch_at_every_entry_point(hg):
    import torch
    x0 = torch.zeros(0, N, dtype=torch.float32, device="cuda")
    t0 = torch.zeros(0, dtype=torch.float32, device="cuda")
    diag = hg.Hopf(np.full(N, 2.0), hg.H_WL1, w=np.ones(N), tol=1e-12, max_iter=100, precision=hg.P_FP32)
    dense = hg.Hopf(_dense_A(), hg.H_WL1, w=np.ones(N), tol=1e-13, max_iter=100, precision=hg.P_MIXED)
    for h in (diag, dense):
        out = h.eval(x0, t0)
        assert all(v.numel() == 0 for v in out.values())
        out = h.eval_control(x0, t0)
        assert out["beta"].numel() == 0 and out["x_final"].numel() == 0
        shape = (N, N) if h is dense else (N,)
        gA = torch.full(shape, float("nan"), device="cuda")
        gc = torch.full((N,), float("nan"), device="cuda")
        gc0 = torch.full((1,), float("nan"), device="cuda")
        gw = torch.full((N,), float("nan"), device="cuda")
        L = hg.lib()
        hg._check(L.hopf_backward(h.handle, 0, None, None, None, None, hg._ptr(gA), hg._stream()))
        hg._check(L.hopf_backward_params(h.handle, 0, None, None, None, None, hg._ptr(gc), hg._ptr(gc0),
                                         hg._ptr(gw), hg._stream()))
        torch.cuda.synchronize()
        for g in (gA, gc, gc0, gw):
            assert (g == 0).all()
    parts = [hg.Hopf(np.full(N, s), hg.H_L2, centre=CENTRE * s, tol=1e-12, max_iter=100, precision=hg.P_FP32)
             for s in (1.0, 2.0)]
    assert hg.union_eval(parts, x0, t0)["phi"].numel() == 0
    assert hg.union_closest(parts, x0)["dist"].numel() == 0
    assert hg.union_closest_noalloc(parts, x0)["dist"].numel() == 0
    hparts = [hg.Hopf(np.full(N, 2.0), hk, tol=1e-12, max_iter=100, precision=hg.P_FP32)
              for hk in (hg.H_L1, hg.H_L2)]
    assert hg.maxH_eval(hparts, x0, t0)["phi"].numel() == 0
    torch.cuda.synchronize()
    for h in [diag, dense] + parts + hparts:
        h.close()


def _centre_cases(hg):
    """(label, Hopf kwargs) for each initial data and Hamiltonian."""
    w = np.linspace(0.5, 1.5, N)
    hams = [(hg.H_L1, None), (hg.H_WL1, w), (hg.H_L2, None), (hg.H_LINF, None), (hg.H_DNORM, w),
            (hg.H_ANORM, _anorm_M())]
    cases = []
    for hk, hw in hams:
        cases.append(("diag-fp32-h%d" % hk, dict(A=np.linspace(0.5, 2.0, N), h_kind=hk, w=hw,
                                                  precision=hg.P_FP32)))
        cases.append(("diag-fp64-h%d" % hk, dict(A=np.linspace(0.5, 2.0, N), h_kind=hk, w=hw,
                                                  precision=hg.P_FP64)))
        for jk in (hg.J_L1SQ, hg.J_LINFSQ):
            cases.append(("j%d-h%d" % (jk, hk), dict(A=None, j_kind=jk, n=N, h_kind=hk, w=hw,
                                                     precision=hg.P_FP32)))
    for hk, hw in hams[:3]:
        for prec in (hg.P_FP32, hg.P_MIXED):
            cases.append(("dense-p%d-h%d" % (prec, hk), dict(A=_dense_A(), h_kind=hk, w=hw, precision=prec)))
    return cases


def test_query_at_the_centre(hg):
    import torch
    t = np.array([0.0, 1.0, 5.0, 40.0])
    for label, kw in _centre_cases(hg):
        A = kw.pop("A")
        h = hg.Hopf(A, centre=CENTRE, c0=C0, tol=1e-12, max_iter=200, stop_rule=hg.STOP_UREL, **kw)
        dt = torch.float64 if kw["precision"] == hg.P_FP64 else torch.float32
        x = torch.tensor(np.tile(CENTRE, (len(t), 1)), dtype=dt, device="cuda")
        out = h.eval(x, torch.tensor(t, dtype=dt, device="cuda"))
        torch.cuda.synchronize()
        assert np.array_equal(out["phi"].cpu().numpy(), np.full(len(t), -C0)), (label, out["phi"])
        assert (out["grad"] == 0).all(), label
        assert (out["dphidt"] == 0).all(), label
        assert (out["status"] == hg.Q_OK).all(), (label, out["status"])
        h.close()


@pytest.mark.parametrize("n", [6, 40])
def test_ties_go_to_the_smallest_index(hg, n):
    """Identical parts tie everywhere: the union (Section 2.2), the maximum
    over Hamiltonians and the distance (Section 3.2) report index 0 and the
    single part's value."""
    import torch
    import workloads as wl
    B = 50
    a = wl.uniform(7701, n, 0.5, 2.0)
    c = wl.normal(7702, n, 1.0)
    x = torch.tensor(wl.normal(7703, B * n, 3.0).reshape(B, n).astype(np.float32), device="cuda")
    t = torch.tensor(wl.uniform(7704, B, 0.0, 2.0).astype(np.float32), device="cuda")
    h = hg.Hopf(a, hg.H_L2, centre=c, tol=1e-12, max_iter=3000, precision=hg.P_FP32)
    one = hg.union_eval([h], x, t)
    three = hg.union_eval([h, h, h], x, t)
    mx = hg.maxH_eval([h, h], x, t)
    d1 = hg.union_closest([h], x)
    d2 = hg.union_closest([h, h], x)
    torch.cuda.synchronize()
    assert (three["argmin"] == 0).all() and torch.equal(three["phi"], one["phi"])
    assert (mx["argmax"] == 0).all() and torch.equal(mx["phi"], one["phi"])
    assert (d2["argmin"] == 0).all() and torch.equal(d2["dist"], d1["dist"])
    h.close()
