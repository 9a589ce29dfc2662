"""The arithmetic model of the tensor-core forms (tests/accuracy_model.py)
against the GPU on the same eight queries of the dense headline workload
(n = 1024, weighted l1, tol 1e-13): the gradient errors the kernels reach
against the FP64 oracle sit within a factor of two of the truncating model's,
for the default two-stage MIXED solve and for SPLIT, and SPLIT's error is
several times MIXED's on the hardware as in the model."""
import numpy as np
import pytest

import workloads as wl
from tests import accuracy_model as am

pytestmark = pytest.mark.gpu

N, Q = 1024, 8


@pytest.fixture(scope="module")
def hg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1605_01799_gb300 as pkg
    pkg.lib()
    return pkg


def test_model_matches_the_gpu(hg, orc):
    import torch
    A, _, _ = wl.spd_matrix(2001, 2002, N)
    w = wl.uniform(2003, N, 0.5, 1.5)
    x = wl.normal(2004, Q * N, 2.0).reshape(Q, N).astype(np.float32)
    t = wl.uniform(2005, Q, 0.1, 3.0).astype(np.float32)
    ref = orc.Problem(A, orc.H_WL1, w=w, c0=0.5, lam=1.0, tol=1e-28, max_iter=50000,
                      stop_rule=orc.STOP_UREL).eval(x.astype(np.float64), t.astype(np.float64))["grad"]

    def err(g):
        e = np.linalg.norm(g.astype(np.float64) - ref, axis=1) / np.maximum(1, np.linalg.norm(ref, axis=1))
        return np.array([e.max(), np.median(e)])

    y = np.ascontiguousarray(x.T)
    thr = t[None, :] * w.astype(np.float32)[:, None]  # FP32 products, as the kernels form t/lambda * w
    res = {}
    for prec, form in (("MIXED", "two_stage"), ("SPLIT", "split")):
        h = hg.Hopf(A, hg.H_WL1, w=w, c0=0.5, lam=1.0, tol=1e-13, max_iter=3000,
                    precision=getattr(hg, "P_" + prec), stop_rule=hg.STOP_UREL)
        out = h.eval(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
        torch.cuda.synchronize()
        assert (out["status"].cpu().numpy() == hg.Q_OK).all(), prec
        gpu = err(out["grad"].cpu().numpy())
        p, _ = am.solve(form, A, 1.0, y, thr, 1e-13, "rz")
        model = err(p.T)
        res[prec] = gpu
        print("%s: gradient error max / median, GPU %.3g / %.3g, model %.3g / %.3g" % (prec, *gpu, *model))
        assert (gpu >= 0.5 * model).all() and (gpu <= 2.0 * model).all(), (prec, gpu, model)
    assert res["SPLIT"][1] > 2 * res["MIXED"][1], res
