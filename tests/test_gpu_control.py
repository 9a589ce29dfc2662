"""Optimal control, terminal point and the maximum over Hamiltonians on the
GPU against the FP64 oracle (Section 2; Section 2.2).

Tolerances.  The control beta = (u - prox(u)) / tau inherits the error of u
(about 1e-6 relative, the gradient bar's source) divided by tau = t / lambda,
so it is compared with an absolute bar of 5e-5 / min(tau, 1) after the GPU's
own beta is checked to lie in dH(grad) to rounding; the terminal point
x - t beta then carries t times that.  phi and the gradient of the maximum
over Hamiltonians keep the single-instance bars (1e-6, 2e-5)."""
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


def _cuda(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


CASES = [(37, False, "FP32", 0), (300, False, "FP32", 1), (64, False, "FP32", 2),
         (256, True, "MIXED", 1), (200, True, "MIXED", 2), (160, True, "FP32", 0)]


@pytest.mark.parametrize("n,dense,prec,h_kind", CASES)
def test_control_against_oracle(hg, orc, n, dense, prec, h_kind):
    import torch
    B = 257
    seed = 13000 + 10 * n + h_kind
    if dense:
        A, Q, s = wl.spd_matrix(seed, seed + 1, n)
        tol = 1e-13
    else:
        A = wl.uniform(seed, n, 0.5, 2.0)
        tol = 1e-12
    w = wl.uniform(seed + 2, n, 0.5, 1.5) if h_kind == 1 else None
    c = wl.normal(seed + 6, n, 0.5)
    x = wl.normal(seed + 3, B * n, 2.0).reshape(B, n).astype(np.float32)
    t = wl.uniform(seed + 4, B, 0.1, 3.0).astype(np.float32)
    t[5] = 0.0  # no control at t = 0
    h = hg.Hopf(A, h_kind, w=w, centre=c, tol=tol, max_iter=3000, precision=getattr(hg, "P_" + prec),
                stop_rule=hg.STOP_UREL)
    out = h.eval_control(_cuda(x), _cuda(t))
    torch.cuda.synchronize()
    assert (out["status"].cpu().numpy() == hg.Q_OK).all()
    g = out["grad"].cpu().numpy().astype(np.float64)
    beta = out["beta"].cpu().numpy().astype(np.float64)
    xf = out["x_final"].cpu().numpy().astype(np.float64)
    wv = np.ones(n) if w is None else w
    # the GPU's beta lies in dH of its own gradient, to the rounding of
    # (u - prox(u)) / tau: u carries ~6e-8 |u| and tau divides it
    tau = np.maximum(t.astype(np.float64), 1e-30)  # lambda = 1
    bar = 5e-5 / np.minimum(tau, 1.0)
    for q in range(B):
        if t[q] == 0:
            assert np.all(beta[q] == 0) and np.array_equal(xf[q], x[q].astype(np.float64))
            continue
        if h_kind == 2:
            if np.linalg.norm(g[q]) > 1e-6:
                assert np.abs(beta[q] - g[q] / np.linalg.norm(g[q])).max() <= bar[q]
            assert np.linalg.norm(beta[q]) <= 1 + bar[q]
        else:
            on = np.abs(g[q]) > 0
            assert np.abs(beta[q][on] - (wv * np.sign(g[q]))[on]).max(initial=0) <= bar[q]
            assert np.all(np.abs(beta[q]) <= wv + bar[q])
    # against the oracle's control at its own (tight) minimiser
    P = orc.Problem(A, h_kind, w=w, centre=c, tol=1e-28, max_iter=50000, stop_rule=orc.STOP_UREL)
    ref = P.eval(x.astype(np.float64), t.astype(np.float64))
    ctl = orc.control(P, x.astype(np.float64), t.astype(np.float64), ref["grad"])
    eb = np.abs(beta - ctl["beta"]).max(1)
    assert np.all(eb <= bar), (eb / bar).max()
    ex = np.abs(xf - ctl["x_T"]).max(1)
    assert np.all(ex <= t * bar + 1e-5 * np.abs(x).max(1)), ex.max()


def test_max_over_hamiltonians_against_oracle(hg, orc):
    """Three Hamiltonians (l1, weighted l1 with weights in [0.05, 0.3], l2) and
    one diagonal J.  l1 never lies below l2, so the maximum is taken by the
    weighted l1 or the l2 part, each on some queries."""
    import torch
    n, B = 64, 300
    a = wl.uniform(13501, n, 0.5, 2.0)
    c = wl.normal(13506, n, 0.5)
    w = wl.uniform(13502, n, 0.05, 0.3)
    x = wl.normal(13503, B * n, 2.0).reshape(B, n).astype(np.float32)
    t = wl.uniform(13504, B, 0.1, 3.0).astype(np.float32)
    kinds = [(0, None), (1, w), (2, None)]
    parts = [hg.Hopf(a, hk, w=ww, centre=c, tol=1e-12, max_iter=3000, precision=hg.P_FP32,
                     stop_rule=hg.STOP_UREL) for hk, ww in kinds]
    out = hg.maxH_eval(parts, _cuda(x), _cuda(t))
    torch.cuda.synchronize()
    oparts = [orc.Problem(a, hk, w=ww, centre=c, tol=1e-28, max_iter=50000, stop_rule=orc.STOP_UREL)
              for hk, ww in kinds]
    ref = orc.maxH_eval(oparts, x.astype(np.float64), t.astype(np.float64))
    phi = out["phi"].cpu().numpy()
    am = out["argmax"].cpu().numpy()
    g = out["grad"].cpu().numpy().astype(np.float64)
    assert (out["status"].cpu().numpy() == hg.Q_OK).all()
    ep = np.abs(phi - ref["phi"]) / np.maximum(1, np.abs(ref["phi"]))
    assert ep.max() <= 1e-6, ep.max()
    # argmax: equal wherever the two best parts are not within the phi bar
    phis = np.stack([orc.Problem(a, hk, w=ww, centre=c, tol=1e-28, max_iter=50000, stop_rule=orc.STOP_UREL)
                     .eval(x.astype(np.float64), t.astype(np.float64))["phi"] for hk, ww in kinds], 1)
    srt = np.sort(phis, 1)
    clear = (srt[:, -1] - srt[:, -2]) > 1e-5 * np.maximum(1, np.abs(srt[:, -1]))
    assert np.array_equal(am[clear], ref["argmax"][clear])
    assert set(np.unique(am[clear]).tolist()) == {1, 2}
    eg = np.linalg.norm(g[clear] - ref["grad"][clear], axis=1) / np.maximum(1, np.linalg.norm(ref["grad"][clear], axis=1))
    assert eg.max() <= 2e-5, eg.max()
