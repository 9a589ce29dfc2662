"""Union of ellipsoids (phi = min_i phi_i) and distance / closest point by
Newton on s, on the GPU against the FP64 oracle and the Section 4.3
ellipsoid projection."""
import numpy as np
import pytest

import workloads as wl
from tests import pins

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


def _setup(hg, orc, n, K, B):
    d = wl.ellipsoid_union(n=n, K=K, batch=B)
    parts = [hg.Hopf(d["a"][k], hg.H_L2, centre=d["centres"][k], tol=1e-12, max_iter=5000,
                     precision=hg.P_FP32, stop_rule=hg.STOP_UREL) for k in range(K)]
    oparts = [orc.Problem(d["a"][k], orc.H_L2, centre=d["centres"][k], tol=1e-28, max_iter=100000,
                          stop_rule=orc.STOP_UREL) for k in range(K)]
    return d, parts, oparts


@pytest.mark.parametrize("n,K,B", [(256, 16, 96), (37, 5, 33)])
def test_union_phi(hg, orc, n, K, B):
    import torch
    d, parts, oparts = _setup(hg, orc, n, K, B)
    out = hg.union_eval(parts, _cuda(d["x"]), _cuda(d["t"]))
    torch.cuda.synchronize()
    ref = orc.union_eval(oparts, d["x"].astype(np.float64), d["t"].astype(np.float64))
    phi = out["phi"].cpu().numpy()
    am = out["argmin"].cpu().numpy()
    e = np.abs(phi - ref["phi"]) / np.maximum(1, np.abs(ref["phi"]))
    assert e.max() <= 1e-6, e.max()
    # argmin may differ only where two parts tie to within the tolerance
    diff = am != ref["argmin"]
    if diff.any():
        for q in np.nonzero(diff)[0]:
            a = orc.union_eval([oparts[am[q]]], d["x"][q:q + 1].astype(np.float64), d["t"][q:q + 1].astype(np.float64))
            assert abs(a["phi"][0] - ref["phi"][q]) <= 1e-6 * max(1, abs(ref["phi"][q]))
    g = out["grad"].cpu().numpy().astype(np.float64)
    ok = ~diff
    eg = np.linalg.norm(g[ok] - ref["grad"][ok], axis=1) / np.maximum(1, np.linalg.norm(ref["grad"][ok], axis=1))
    # semi-axes in [0.2, 5] give A = diag(semi^2) a condition up to 625, and the
    # FP32 gradient moves by up to ~cond * 6e-8 relative
    assert eg.max() <= 1e-4, eg.max()
    assert (out["status"].cpu().numpy() == hg.Q_OK).all()


def test_closest_point(hg, orc):
    import torch
    n, K, B = 64, 6, 48
    d, parts, oparts = _setup(hg, orc, n, K, B)
    out = hg.union_closest(parts, _cuda(d["x"]), s_tol=1e-6, max_newton=60)
    torch.cuda.synchronize()
    dist = out["dist"].cpu().numpy()
    cl = out["closest"].cpu().numpy()
    am = out["argmin"].cpu().numpy()
    assert (out["status"].cpu().numpy() == hg.Q_OK).all()
    for q in range(B):
        best, bk, bp = np.inf, -1, None
        for k in range(K):
            p, _ = pins.ellipsoid_projection(d["x"][q].astype(np.float64) - d["centres"][k], d["semi"][k])
            dk = np.linalg.norm(d["x"][q] - d["centres"][k] - p)
            if dk < best:
                best, bk, bp = dk, k, p + d["centres"][k]
        assert abs(dist[q] - best) <= 1e-5 * max(1, best), (q, dist[q], best)
        if am[q] == bk:
            # closest = x - s grad/|grad|: the FP32 direction error (~cond * 6e-8
            # with cond <= 625, times a safety factor) is scaled by s (<= ~15)
            assert np.abs(cl[q] - bp).max() <= 1e-3 * max(1, np.abs(bp).max())
    # and the oracle's own Newton-on-s route agrees
    ref = orc.union_closest(oparts, d["x"].astype(np.float64), s_tol=1e-12, max_newton=100)
    assert np.abs(dist - ref["dist"]).max() <= 1e-5 * max(1, np.abs(ref["dist"]).max())
