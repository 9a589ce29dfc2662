"""Full-size workloads in the launch configuration the benchmark times, checked
on sampled queries the oracle computes one by one, and by properties that hold
at any size on every query."""
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


def _sample(seed, count, total):
    return np.unique((wl.uniform(seed, 4 * count) * total).astype(np.int64))[:count]


# (precision, relative stop tolerance, gradient bars max / median); the SPLIT
# bars follow from its amplified accumulation error (tests/test_gpu_dense.py).
DENSE_CASES = [("SPLIT", 1e-13, 2.5e-5, 1.2e-5), ("MIXED", 1e-13, 6e-6, 3e-6), ("FP32", 1e-13, 6e-6, 3e-6)]


@pytest.mark.parametrize("precision,tol,gmax,gmed", DENSE_CASES)
def test_dense_n1024_b65536(hg, orc, precision, tol, gmax, gmed):
    """The metric's workload: n = 1024, 65,536 queries, weighted l1, relative
    stop, exactly as bench.py runs it."""
    import torch
    n, B = 1024, 65536
    A, Q, s = wl.spd_matrix(2001, 2002, n)
    w = wl.uniform(2003, n, 0.5, 1.5)
    x, t = wl.queries_dense(n, B)
    h = hg.Hopf(A, hg.H_WL1, w=w, tol=tol, max_iter=1000, precision=getattr(hg, "P_" + precision))
    out = h.eval(_cuda(x), _cuda(t))
    torch.cuda.synchronize()
    st = out["status"].cpu().numpy()
    it = out["iters"].cpu().numpy()
    g = out["grad"].cpu().numpy()
    phi = out["phi"].cpu().numpy()
    # every query: converged, finite, and d phi/dt = -H(grad) exactly as defined
    assert (st == hg.Q_OK).all()
    assert ((it >= 2) & (it < 1000)).all()
    assert np.isfinite(phi).all() and np.isfinite(g).all()
    H = (np.abs(g.astype(np.float64)) * w).sum(1)
    assert np.allclose(out["dphidt"].cpu().numpy(), -H, rtol=1e-5, atol=1e-5)
    # sampled queries against the oracle
    idx = _sample(77001, 24, B)
    P = orc.Problem(A, orc.H_WL1, w=w, tol=1e-28, max_iter=50000, stop_rule=orc.STOP_UREL)
    ref = P.eval(x[idx].astype(np.float64), t[idx].astype(np.float64))
    ep = np.abs(phi[idx] - ref["phi"]) / np.maximum(1, np.abs(ref["phi"]))
    eg = np.linalg.norm(g[idx] - ref["grad"], axis=1) / np.maximum(1, np.linalg.norm(ref["grad"], axis=1))
    assert ep.max() <= 1e-6, ep.max()
    assert eg.max() <= gmax, eg.max()
    assert np.median(eg) <= gmed, np.median(eg)


def test_union_k16_n256_b16384(hg, orc):
    """Union of 16 ellipsoids in n = 256, 16,384 exterior queries, t ~ U[0,2]:
    phi = min_i phi_i, then distance and closest point by Newton on s."""
    import torch
    d = wl.ellipsoid_union()
    K, n, B = d["K"], d["n"], len(d["t"])
    parts = [hg.Hopf(d["a"][k], hg.H_L2, centre=d["centres"][k], tol=1e-12, max_iter=5000,
                     precision=hg.P_FP32, stop_rule=hg.STOP_UREL) for k in range(K)]
    x = _cuda(d["x"])
    u = hg.union_eval(parts, x, _cuda(d["t"]))
    c = hg.union_closest(parts, x, s_tol=1e-6, max_newton=60)
    torch.cuda.synchronize()
    assert (u["status"].cpu().numpy() == hg.Q_OK).all()
    assert (c["status"].cpu().numpy() == hg.Q_OK).all()
    dist = c["dist"].cpu().numpy()
    cl = c["closest"].cpu().numpy()
    am = c["argmin"].cpu().numpy()
    # every query: the closest point lies on the boundary of its ellipsoid,
    # at the reported distance from x
    semi, cen = d["semi"], d["centres"]
    lvl = (((cl.astype(np.float64) - cen[am]) / semi[am]) ** 2).sum(1)
    assert np.abs(lvl - 1).max() <= 1e-3
    assert np.abs(np.linalg.norm(cl - d["x"], axis=1) - dist).max() <= 1e-4 * max(1, dist.max())
    # sampled queries: phi against the oracle, distance against Section 4.3
    idx = _sample(77002, 16, B)
    oparts = [orc.Problem(d["a"][k], orc.H_L2, centre=cen[k], tol=1e-28, max_iter=100000,
                          stop_rule=orc.STOP_UREL) for k in range(K)]
    ref = orc.union_eval(oparts, d["x"][idx].astype(np.float64), d["t"][idx].astype(np.float64))
    phi = u["phi"].cpu().numpy()[idx]
    assert (np.abs(phi - ref["phi"]) / np.maximum(1, np.abs(ref["phi"]))).max() <= 1e-6
    for j, q in enumerate(idx):
        best = min(np.linalg.norm(d["x"][q] - cen[k] - pins.ellipsoid_projection(d["x"][q] - cen[k], semi[k])[0])
                   for k in range(K))
        assert abs(dist[q] - best) <= 1e-5 * max(1, best)


def test_dense_n2048_b32768_forward_backward(hg, orc):
    """Differentiation workload: n = 2048, H = l1, 32,768 queries; forward in
    the MIXED form, backward by the envelope theorem; dphi/dA checked by FP64
    central differences (h = 1e-6) of exact active-set values on the 64
    sampled queries, g_x and g_t likewise, and g_A (tensor cores) against
    -1/2 V^T diag(g) V on a sampled block and the CUDA-core kernel."""
    import torch
    d = wl.dense_l1_grad()
    A, n, B = d["A"], d["n"], len(d["t"])
    h = hg.Hopf(A, hg.H_L1, tol=1e-13, max_iter=1000, precision=hg.P_MIXED)
    out = h.eval(_cuda(d["x"]), _cuda(d["t"]))
    g = wl.normal(5008, B, 1.0).astype(np.float32)
    gx, gt, gA = h.backward(_cuda(g), out["grad"])
    torch.cuda.synchronize()
    assert (out["status"].cpu().numpy() == hg.Q_OK).all()
    V = out["grad"].cpu().numpy().astype(np.float64)
    # g_A on a sampled 64 x 64 block against the definition
    rows = _sample(77003, 64, n)
    cols = _sample(77004, 64, n)
    blk = -0.5 * (V[:, rows] * g[:, None]).T @ V[:, cols]
    gAb = gA.cpu().numpy()[np.ix_(rows, cols)]
    assert np.abs(gAb - blk).max() <= 1e-5 * np.abs(blk).max()
    # the tensor-core g_A against the FP32 CUDA-core kernel on the whole matrix
    _, _, gA32 = h.backward(_cuda(g), out["grad"], want_x=False, want_t=False, tensor_cores=False)
    torch.cuda.synchronize()
    gAf = gA.cpu().numpy()
    assert np.abs(gAf - gA32.cpu().numpy()).max() <= 1e-5 * np.abs(gAf).max()
    assert np.array_equal(gAf, gAf.T)
    assert np.allclose(gx.cpu().numpy(), g[:, None] * V, rtol=1e-6, atol=1e-6)
    assert np.allclose(gt.cpu().numpy(), -g * np.abs(V).sum(1), rtol=1e-5, atol=1e-5)
    # forward parity on the 64 sampled queries, and FP64 central differences
    # (h = 1e-6) of exact active-set values in A, x and t at each of them
    idx = d["fd_queries"]
    assert len(idx) == 64
    P = orc.Problem(A, orc.H_L1, tol=1e-28, max_iter=50000, stop_rule=orc.STOP_UREL)
    ref = P.eval(d["x"][idx].astype(np.float64), d["t"][idx].astype(np.float64))
    phi = out["phi"].cpu().numpy()[idx]
    assert (np.abs(phi - ref["phi"]) / np.maximum(1, np.abs(ref["phi"]))).max() <= 1e-6
    gxh, gth = gx.cpu().numpy(), gt.cpu().numpy()
    w1 = np.ones(n)
    rng = np.random.default_rng(9)
    for j, q in enumerate(idx):
        xq, tq = d["x"][q].astype(np.float64), float(d["t"][q])
        vq, ok = pins.kkt_active_set(A, xq, tq, w1, ref["grad"][j])
        assert ok
        S = np.nonzero(vq)[0]

        def phi_at(Am, xx, tt):
            vv, ok2 = pins.kkt_active_set(Am, xx, tt, w1, vq)
            assert ok2
            return pins.objective_neg(Am, xx, tt, w1, vv)

        # the GPU's gradient error bound (the 6e-6 relative l2 bar of the
        # dense tests) carried into each derivative
        dv = 6e-6 * max(1.0, np.linalg.norm(vq))
        # d phi / dt = -H(v*) and d phi / dx_i = v*_i (g_t, g_x with g = g_q)
        fd_t = (phi_at(A, xq, tq + 1e-6) - phi_at(A, xq, tq - 1e-6)) / 2e-6
        assert abs(fd_t + np.abs(vq).sum()) <= 1e-5 * max(1, abs(fd_t))
        assert abs(gth[q] / g[q] - fd_t) <= np.sqrt(n) * dv + 1e-5 * abs(fd_t), (q, gth[q] / g[q], fd_t)
        i0 = int(rng.choice(S)) if len(S) else 0
        e = np.zeros(n)
        e[i0] = 1e-6
        fd_x = (phi_at(A, xq + e, tq) - phi_at(A, xq - e, tq)) / 2e-6
        assert abs(fd_x - vq[i0]) <= 1e-5 * max(1, abs(fd_x))
        assert abs(gxh[q, i0] / g[q] - fd_x) <= dv + 1e-5 * abs(fd_x)
        # d phi / dA_ij (symmetric perturbation: twice -1/2 v_i v_j off the
        # diagonal), against the g_A of this query alone
        one = np.zeros(B, np.float32)
        one[q] = 1.0
        _, _, gAq = h.backward(_cuda(one), out["grad"], want_x=False, want_t=False)
        torch.cuda.synchronize()
        gAq = gAq.cpu().numpy()
        for _ in range(2):
            i1, i2 = rng.choice(S, 2) if len(S) else (0, 0)
            E = np.zeros((n, n))
            E[i1, i2] += 1e-6
            if i1 != i2:
                E[i2, i1] += 1e-6
            fd = (phi_at(A + E, xq, tq) - phi_at(A - E, xq, tq)) / 2e-6
            f = 1 if i1 == i2 else 2
            exact = -0.5 * vq[i1] * vq[i2] * f  # envelope theorem at the exact minimiser
            assert abs(fd - exact) <= 1e-5 * max(1, abs(fd)), (q, i1, i2, fd, exact)
            bound = 0.5 * f * (abs(vq[i1]) * dv + abs(vq[i2]) * dv + dv * dv)
            assert abs(gAq[i1, i2] * f - exact) <= bound + 1e-5 * abs(exact), (q, i1, i2, gAq[i1, i2] * f, exact)


def _h_of(g, h_kind, w):
    g = np.abs(g.astype(np.float64))
    if h_kind == 0:
        return g.sum(1)
    if h_kind == 1:
        return (g * w).sum(1)
    return np.sqrt((g * g).sum(1))


def test_ragged_512_instances(hg, orc):
    """Ragged batch: 512 instances, n log-uniform in [16, 4096], 64 to 8,192
    queries each; instances 0-255 diagonal (FP32), 256-511 dense (MIXED); H
    cycles l1, weighted l1, l2; one graph replay.  Every query: converged,
    finite, d phi/dt = -H(grad).  Sampled queries (first and last query of
    16 seeded instances, plus the largest dense instance) against the oracle
    with the bars of the single-instance tests."""
    import torch
    descs = wl.ragged()
    inst = wl.ragged_instances(descs)
    bd = [{"A": d["A"] if "A" in d else d["a"], "h_kind": d["h_kind"], "w": d["w"], "c0": d["c0"],
           "lam": d["lam"], "tol": 1e-13 if "A" in d else 1e-12, "max_iter": 3000,
           "precision": hg.P_MIXED if "A" in d else hg.P_FP32, "stop_rule": hg.STOP_UREL} for d in inst]
    b = hg.HopfBatch(bd)
    counts = np.array([d["x"].shape[0] for d in inst], dtype=np.int64)
    ns = np.array([d["n"] for d in inst], dtype=np.int64)
    x = torch.tensor(np.concatenate([d["x"].reshape(-1) for d in inst]), device="cuda")
    t = torch.tensor(np.concatenate([d["t"] for d in inst]), device="cuda")
    out = b.eval(counts, x, t)
    torch.cuda.synchronize()
    info = b.info()
    assert info["used_graph"] and info["nstreams"] >= 1
    phi = out["phi"].cpu().numpy()
    g = out["grad"].cpu().numpy()
    st = out["status"].cpu().numpy()
    it = out["iters"].cpu().numpy()
    dt = out["dphidt"].cpu().numpy()
    del x, out
    assert (st == hg.Q_OK).all(), np.bincount(st)
    assert (it < 3000).all() and np.isfinite(phi).all() and np.isfinite(g).all()
    qoff = np.concatenate([[0], np.cumsum(counts)])
    xoff = np.concatenate([[0], np.cumsum(counts * ns)])
    for i, d in enumerate(inst):
        gi = g[xoff[i]:xoff[i + 1]].reshape(counts[i], ns[i])
        Hi = _h_of(gi, d["h_kind"], d["w"])
        assert np.allclose(dt[qoff[i]:qoff[i + 1]], -Hi, rtol=1e-5, atol=1e-5), i
    pick = sorted(set(_sample(77005, 16, len(inst)).tolist()) |
                  {int(np.argmax(np.where([("A" in d) for d in inst], ns, 0)))})
    for i in pick:
        d = inst[i]
        A = d["A"] if "A" in d else d["a"]
        q = np.unique([0, counts[i] - 1])
        P = orc.Problem(A, d["h_kind"], w=d["w"], c0=d["c0"], lam=d["lam"], tol=1e-28, max_iter=50000,
                        stop_rule=orc.STOP_UREL)
        ref = P.eval(d["x"][q].astype(np.float64), d["t"][q].astype(np.float64))
        gi = g[xoff[i]:xoff[i + 1]].reshape(counts[i], ns[i])[q]
        ep = np.abs(phi[qoff[i] + q] - ref["phi"]) / np.maximum(1, np.abs(ref["phi"]))
        eg = np.linalg.norm(gi - ref["grad"], axis=1) / np.maximum(1, np.linalg.norm(ref["grad"], axis=1))
        assert ep.max() <= 1e-6, (i, ep.max())
        assert eg.max() <= (6e-6 if "A" in d else 2e-5), (i, eg.max())
    b.close()
