"""Envelope-theorem backward on the GPU against the oracle and FP64 finite
differences."""
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


@pytest.mark.parametrize("tensor_cores", [True, False])
@pytest.mark.parametrize("n,B", [(128, 300), (200, 77), (384, 5000)])
def test_backward_dense_matches_oracle(hg, orc, n, B, tensor_cores):
    """g_x, g_t and the dense g_A = -1/2 V^T diag(g) V against the oracle's
    FP64 sums over the same minimisers, on the tensor cores (two-term FP16
    splits, chunked promotion, FP64 sums of K ranges: n = 384 has off-diagonal
    tiles and their mirrors, 5,000 queries two K ranges and a ragged last
    k-block) and on the FP32 CUDA cores."""
    import torch
    A, Q, s = wl.spd_matrix(12001 + n, 12002, n)
    x = wl.normal(12003, B * n, 2.0).reshape(B, n).astype(np.float32)
    t = wl.uniform(12004, B, 0.1, 3.0).astype(np.float32)
    g = wl.normal(12005, B, 1.0).astype(np.float32)
    h = hg.Hopf(A, hg.H_L1, tol=1e-13, max_iter=3000, precision=hg.P_FP32)
    out = h.eval(_cuda(x), _cuda(t))
    gx, gt, gA = h.backward(_cuda(g), out["grad"], tensor_cores=tensor_cores)
    torch.cuda.synchronize()
    v = out["grad"].cpu().numpy().astype(np.float64)
    ref = orc.backward(n, orc.A_DENSE, orc.H_L1, None, g.astype(np.float64), v, t.astype(np.float64))
    assert np.allclose(gx.cpu().numpy(), ref["g_x"], rtol=1e-6, atol=1e-6)
    assert np.allclose(gt.cpu().numpy(), ref["g_t"], rtol=1e-5, atol=1e-5)
    scale = np.abs(ref["g_A"]).max()
    assert np.abs(gA.cpu().numpy() - ref["g_A"]).max() <= 1e-5 * scale


def test_backward_tc_scale_and_zero_weights(hg, orc):
    """Upstream weights of very different magnitudes (1e-6 and 1e+4 scales,
    some exact zeros): the power-of-two scaling of g keeps the FP16 operands in
    range, and g_A follows the oracle at the same bar."""
    import torch
    n, B = 256, 700
    A, Q, s = wl.spd_matrix(12301, 12302, n)
    x = wl.normal(12303, B * n, 2.0).reshape(B, n).astype(np.float32)
    t = wl.uniform(12304, B, 0.1, 3.0).astype(np.float32)
    h = hg.Hopf(A, hg.H_L1, tol=1e-13, max_iter=3000, precision=hg.P_MIXED)
    out = h.eval(_cuda(x), _cuda(t))
    v = out["grad"].cpu().numpy().astype(np.float64)
    for mag in (1e-6, 1e4):
        g = (wl.normal(12305, B, 1.0) * mag).astype(np.float32)
        g[::5] = 0.0
        _, _, gA = h.backward(_cuda(g), out["grad"], want_x=False, want_t=False)
        torch.cuda.synchronize()
        ref = orc.backward(n, orc.A_DENSE, orc.H_L1, None, g.astype(np.float64), v, t.astype(np.float64))
        scale = np.abs(ref["g_A"]).max()
        assert np.abs(gA.cpu().numpy() - ref["g_A"]).max() <= 1e-5 * scale, mag


def test_backward_diag(hg, orc):
    import torch
    n, B = 50, 123
    a = wl.uniform(12101, n, 0.5, 2.0)
    w = wl.uniform(12102, n, 0.5, 1.5)
    x = wl.normal(12103, B * n, 2.0).reshape(B, n).astype(np.float32)
    t = wl.uniform(12104, B, 0.1, 3.0).astype(np.float32)
    g = wl.normal(12105, B, 1.0).astype(np.float32)
    h = hg.Hopf(a, hg.H_WL1, w=w, tol=1e-12, max_iter=2000, precision=hg.P_FP32)
    out = h.eval(_cuda(x), _cuda(t))
    gx, gt, gA = h.backward(_cuda(g), out["grad"])
    torch.cuda.synchronize()
    v = out["grad"].cpu().numpy().astype(np.float64)
    ref = orc.backward(n, orc.A_DIAG, orc.H_WL1, w, g.astype(np.float64), v, t.astype(np.float64))
    assert np.allclose(gt.cpu().numpy(), ref["g_t"], rtol=1e-5, atol=1e-5)
    assert np.allclose(gA.cpu().numpy(), ref["g_A"], rtol=1e-5, atol=1e-5 * np.abs(ref["g_A"]).max())


def test_backward_fd_on_sampled_queries(hg, orc):
    """dphi/dA_ij by FP64 central differences (h = 1e-6) of exact active-set
    values, symmetric perturbation (factor 2 off the diagonal), against the
    GPU's -1/2 v v^T for single queries (g = 1)."""
    import torch
    n, B = 96, 8
    A, Q, s = wl.spd_matrix(12201, 12202, n)
    x = wl.normal(12203, B * n, 2.0).reshape(B, n).astype(np.float32)
    t = wl.uniform(12204, B, 0.1, 3.0).astype(np.float32)
    h = hg.Hopf(A, hg.H_L1, tol=1e-13, max_iter=3000, precision=hg.P_FP32)
    out = h.eval(_cuda(x), _cuda(t))
    v_gpu = out["grad"].cpu().numpy().astype(np.float64)
    w = np.ones(n)
    rng = np.random.default_rng(3)
    for q in range(B):
        one = np.zeros(B, np.float32)
        one[q] = 1.0
        _, _, gA = h.backward(_cuda(one), out["grad"], want_x=False, want_t=False)
        torch.cuda.synchronize()
        gA = gA.cpu().numpy()
        xq, tq = x[q].astype(np.float64), float(t[q])
        vq, ok = pins.kkt_active_set(A, xq, tq, w, v_gpu[q])
        assert ok
        for _ in range(4):
            i, j = rng.integers(0, n, 2)
            E = np.zeros((n, n))
            E[i, j] += 1e-6
            if i != j:
                E[j, i] += 1e-6

            def phi_of(Am):
                vv, ok2 = pins.kkt_active_set(Am, xq, tq, w, vq)
                assert ok2
                return pins.objective_neg(Am, xq, tq, w, vv)

            fd = (phi_of(A + E) - phi_of(A - E)) / 2e-6
            expect = gA[i, j] * (1 if i == j else 2)
            assert abs(fd - expect) <= 2e-5 * max(1, abs(fd)), (q, i, j, fd, expect)


@pytest.mark.parametrize("dense,hk", [(False, 1), (False, 4), (True, 1), (False, 2)])
def test_parameter_gradients_match_oracle(hg, orc, dense, hk):
    """dL/dc, dL/dc0 and dL/dw (weighted l1, sqrt(sum w p^2)) from the GPU's
    minimisers against the oracle's formulas at the same minimisers (FP64
    sums on both sides; the GPU's are FP32-rounded), and g_w refused for an
    unweighted Hamiltonian."""
    import torch
    n, B = (128, 200) if dense else (40, 300)
    seed = 12500 + 10 * hk + (100 if dense else 0)
    A = wl.spd_matrix(seed, seed + 1, n)[0] if dense else wl.uniform(seed, n, 0.5, 2.0)
    w = wl.uniform(seed + 2, n, 0.5, 1.5) if hk in (1, 4) else None
    c = wl.normal(seed + 3, n, 1.0)
    x = wl.normal(seed + 4, B * n, 2.0).reshape(B, n).astype(np.float32)
    t = wl.uniform(seed + 5, B, 0.1, 3.0).astype(np.float32)
    g = wl.normal(seed + 6, B, 1.0).astype(np.float32)
    h = hg.Hopf(A, hk, w=w, centre=c, tol=1e-13 if dense else 1e-12, max_iter=3000,
                precision=hg.P_MIXED if dense else hg.P_FP32)
    out = h.eval(_cuda(x), _cuda(t))
    td = _cuda(t)
    want_w = hk in (1, 4)
    gc, gc0, gw = h.backward_params(_cuda(g), out["grad"], t=td, dphidt=out["dphidt"], want_w=want_w)
    torch.cuda.synchronize()
    v = out["grad"].cpu().numpy().astype(np.float64)
    ref = orc.backward_params(n, hk, w, g.astype(np.float64), v, t.astype(np.float64))
    scale = np.abs(ref["g_c"]).max()
    assert np.abs(gc.cpu().numpy() - ref["g_c"]).max() <= 1e-5 * max(1.0, scale)
    assert abs(float(gc0.cpu()) - ref["g_c0"]) <= 1e-5 * max(1.0, abs(ref["g_c0"]))
    if want_w:
        # (the GPU's H for sqrt(sum w p^2) is the forward's dphidt, FP32)
        sw = np.abs(ref["g_w"]).max()
        assert np.abs(gw.cpu().numpy() - ref["g_w"]).max() <= 2e-5 * max(1.0, sw)
    else:
        with pytest.raises(hg.HopfError):
            h.backward_params(_cuda(g), out["grad"], t=td, want_w=True)
