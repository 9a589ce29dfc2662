"""Dense-A solvers on the GPU against the FP64 oracle (same seeded inputs).

Tolerances.  A = Q diag(s) Q^T with s in [0.1, 10] has condition 100, so an
FP32 evaluation of A p or M r (relative rounding ~6e-8 per entry) moves the
fixed point by up to ~cond * 6e-8 ~ 6e-6 relative in the gradient; measured
errors sit at 1-3e-6 (l2 cases at the top: their minimiser solves
(A + mu I) v = y).  phi is stationary in v at the minimiser, so its error is
second order and FP64 accumulation keeps it below 1e-6 relative.  Bars:
phi <= 1e-6 relative (floor 1) for every query; gradient <= 6e-6 relative
(floor 1) for every query and <= 3e-6 at the median.  tests/accuracy_model.py
models the tensor-core forms' arithmetic (FP16 / BF16 operands, FP32
accumulators) and checks these bars against the oracle on the CPU.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

PHI_TOL, GRAD_MAX, GRAD_MED = 1e-6, 6e-6, 3e-6
# The SPLIT form evaluates v = M r, whose error reaches the fixed point
# amplified by |A + lambda I| (up to 11 here) where MIXED's error in A p enters
# unamplified; the tensor cores' FP32 accumulation truncates (a bias of about
# half an ulp per K = 16 step, 64 steps at n = 1024), so SPLIT's gradient
# error sits near 1e-5 (measured 6.7e-6 at n = 384, 9.6e-6 at n = 1024).
GRAD_BARS = {"FP32": (6e-6, 3e-6), "MIXED": (6e-6, 3e-6), "SPLIT": (2.5e-5, 1.2e-5)}
# Relative stop |u^k - u^{k-1}|^2 <= TOL max(1, |u^k|^2).  FP32 storage of u
# alone rounds by ~6e-8 relative, i.e. (6e-8)^2 ~ 4e-15 squared: 1e-13 keeps
# the test a decade above that floor.
TOL = 1e-13


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


def _errors(out, ref):
    phi = out["phi"].cpu().numpy()
    g = out["grad"].cpu().numpy().astype(np.float64)
    ephi = np.abs(phi - ref["phi"]) / np.maximum(1, np.abs(ref["phi"]))
    eg = np.linalg.norm(g - ref["grad"], axis=1) / np.maximum(1, np.linalg.norm(ref["grad"], axis=1))
    return ephi, eg


_REF = {}


def _case(orc, n, B, h_kind, seed):
    key = (n, B, h_kind, seed)
    if key not in _REF:
        A, Q, s = wl.spd_matrix(seed, seed + 1, n)
        w = wl.uniform(seed + 2, n, 0.5, 1.5) if h_kind == 1 else None
        x = wl.normal(seed + 3, B * n, 2.0).reshape(B, n).astype(np.float32)
        t = wl.uniform(seed + 4, B, 0.1, 3.0).astype(np.float32)
        P = orc.Problem(A, h_kind, w=w, tol=1e-28, max_iter=50000, stop_rule=orc.STOP_UREL)
        ref = P.eval(x.astype(np.float64), t.astype(np.float64))
        _REF[key] = (A, w, x, t, ref)
    return _REF[key]


@pytest.mark.parametrize("precision", ["FP32", "SPLIT", "MIXED"])
@pytest.mark.parametrize("n,B,h_kind", [(128, 300, 1), (200, 129, 1), (384, 257, 0), (256, 64, 2), (129, 1, 1)])
def test_dense_parity(hg, orc, precision, n, B, h_kind):
    """Ragged n (not a multiple of the 128-row tile) and ragged batches (not a
    multiple of the query tile) for each Hamiltonian."""
    import torch
    A, w, x, t, ref = _case(orc, n, B, h_kind, 11000 + n + h_kind)
    prec = getattr(hg, "P_" + precision)
    try:
        h = hg.Hopf(A, h_kind, w=w, tol=TOL, max_iter=3000, precision=prec)
        out = h.eval(_cuda(x), _cuda(t))
    except hg.HopfError as e:
        if e.status == hg.HOPF_EUNSUPPORTED:
            pytest.skip(str(e))
        raise
    torch.cuda.synchronize()
    ephi, eg = _errors(out, ref)
    gmax, gmed = GRAD_BARS[precision]
    assert (out["status"].cpu().numpy() == hg.Q_OK).all()
    assert ephi.max() <= PHI_TOL, ephi.max()
    assert eg.max() <= gmax, eg.max()
    assert np.median(eg) <= gmed, np.median(eg)
    dphidt = out["dphidt"].cpu().numpy()
    H = ref["dphidt"]
    assert np.allclose(dphidt, H, rtol=1e-5, atol=1e-5)


def test_dense_iteration_counts(hg, orc):
    """Same stop rule and tolerance on both sides: the GPU's counts follow the
    oracle's (FP32 rounding can move a query across the threshold by a step)."""
    import torch
    n, B = 128, 200
    A, w, x, t, ref = _case(orc, n, B, 1, 11500)
    tol = 1e-12
    h = hg.Hopf(A, 1, w=w, tol=tol, max_iter=3000, precision=hg.P_FP32)
    out = h.eval(_cuda(x), _cuda(t))
    torch.cuda.synchronize()
    same = orc.Problem(A, 1, w=w, tol=tol, max_iter=3000, stop_rule=orc.STOP_UREL).eval(
        x.astype(np.float64), t.astype(np.float64))
    it = out["iters"].cpu().numpy()
    assert np.median(np.abs(it - same["iters"])) <= 1
    assert np.abs(it - same["iters"]).max() <= 10


@pytest.mark.parametrize("precision", ["FP32", "SPLIT", "MIXED"])
def test_dense_iterates_across_row_tiles(hg, orc, precision):
    """n = 384 (three row tiles per query): an item's product reads u^{k-1}
    over all rows while the other row tiles' epilogues write u^k, so the two
    must not share storage.  Two evaluations agree bit for bit, and the
    iteration counts follow the oracle's under the same rule."""
    import torch
    n, B = 384, 1024
    A, Q, s = wl.spd_matrix(11700, 11701, n)
    w = wl.uniform(11702, n, 0.5, 1.5)
    x = wl.normal(11703, B * n, 2.0).reshape(B, n).astype(np.float32)
    t = wl.uniform(11704, B, 0.1, 3.0).astype(np.float32)
    tol = 1e-12
    h = hg.Hopf(A, 1, w=w, tol=tol, max_iter=3000, precision=getattr(hg, "P_" + precision))
    xd, td = _cuda(x), _cuda(t)
    o1 = h.eval(xd, td)
    torch.cuda.synchronize()
    snap = {k: v.clone() for k, v in o1.items()}
    o2 = h.eval(xd, td)
    torch.cuda.synchronize()
    for k in ("phi", "grad", "iters"):
        assert torch.equal(snap[k], o2[k]), k
    if precision == "FP32":
        same = orc.Problem(A, 1, w=w, tol=tol, max_iter=3000, stop_rule=orc.STOP_UREL).eval(
            x.astype(np.float64), t.astype(np.float64))
        it = o2["iters"].cpu().numpy()
        assert np.median(np.abs(it - same["iters"])) <= 1
        assert np.abs(it - same["iters"]).max() <= 10


def test_dense_t_zero_and_not_converged(hg, orc):
    """t = 0 gives phi = J(x) (eq. 1.1b); a tiny max_iter reports
    NOT_CONVERGED with iters = max_iter."""
    import torch
    n, B = 128, 40
    A, Q, s = wl.spd_matrix(11601, 11602, n)
    x = wl.normal(11603, B * n, 2.0).reshape(B, n).astype(np.float32)
    t = np.zeros(B, np.float32)
    h = hg.Hopf(A, 0, tol=TOL, max_iter=3000, precision=hg.P_FP32)
    out = h.eval(_cuda(x), _cuda(t))
    torch.cuda.synchronize()
    Ainv = (Q / s) @ Q.T
    xd = x.astype(np.float64)
    J = 0.5 * np.einsum("bi,ij,bj->b", xd, Ainv, xd) - 0.5
    assert np.abs(out["phi"].cpu().numpy() - J).max() <= 1e-6 * max(1, np.abs(J).max())
    h2 = hg.Hopf(A, 0, tol=TOL, max_iter=3, precision=hg.P_FP32)
    out = h2.eval(_cuda(x), _cuda(np.full(B, 1.0, np.float32)))
    torch.cuda.synchronize()
    assert (out["status"].cpu().numpy() == hg.Q_NOT_CONVERGED).all()
    assert (out["iters"].cpu().numpy() == 3).all()


@pytest.mark.parametrize("n,B,h_kind", [(384, 1000, 1), (256, 700, 0)])
def test_two_stage_mixed(hg, orc, n, B, h_kind):
    """MIXED with l1 / weighted l1 runs SPLIT iterations until each query's
    squared relative change is within ten times the tolerance, then the
    defect correction from there: both stages' results sit within the MIXED
    bars of the oracle (the second stage removes the SPLIT fixed point's
    bias), and the total iteration counts follow the one-stage solve's,
    including those of the t = 0 queries (prox the identity: the iteration
    contracts at lambda / (lambda + s_min), some 120 steps here)."""
    import torch
    A, Q, s = wl.spd_matrix(11821 + n, 11822 + n, n)
    w = wl.uniform(11823, n, 0.5, 1.5) if h_kind == 1 else None
    x = wl.normal(11824, B * n, 2.0).reshape(B, n).astype(np.float32)
    t = wl.uniform(11825, B, 0.1, 3.0).astype(np.float32)
    t[::9] = 0.0
    outs = {}
    for sw in (None, 0.0):
        h = hg.Hopf(A, h_kind, w=w, tol=TOL, max_iter=3000, precision=hg.P_MIXED)
        if sw is not None:
            h.set_split_start(sw)
        outs[sw] = h.eval(_cuda(x), _cuda(t))
    torch.cuda.synchronize()
    idx = np.r_[0:40, B - 24:B]
    ref = orc.Problem(A, h_kind, w=w, tol=1e-28, max_iter=50000, stop_rule=orc.STOP_UREL).eval(
        x[idx].astype(np.float64), t[idx].astype(np.float64))
    for sw, out in outs.items():
        assert (out["status"].cpu().numpy() == hg.Q_OK).all(), sw
        ephi, eg = _errors({k: v[idx] for k, v in out.items()}, ref)
        assert ephi.max() <= PHI_TOL, (sw, ephi.max())
        assert eg.max() <= GRAD_MAX and np.median(eg) <= GRAD_MED, (sw, eg.max(), np.median(eg))
    k2 = outs[None]["iters"].cpu().numpy().astype(np.int64)
    k1 = outs[0.0]["iters"].cpu().numpy().astype(np.int64)
    assert np.median(np.abs(k2 - k1)) <= 2 and np.abs(k2 - k1).max() <= 15, (np.abs(k2 - k1).max())


def test_two_stage_mixed_max_iter(hg):
    """max_iter caps the two stages' sum: a cap below the first stage's need
    reports NOT_CONVERGED with iters = max_iter, as the one-stage solve does;
    a cap between the stages' needs lets the defect correction finish within
    it.  The switch accepts 0 and rejects a negative value or another form."""
    import torch
    n, B = 256, 300
    A, Q, s = wl.spd_matrix(11831, 11832, n)
    x = wl.normal(11834, B * n, 2.0).reshape(B, n).astype(np.float32)
    t = np.full(B, 1.0, np.float32)
    h = hg.Hopf(A, 0, tol=TOL, max_iter=5, precision=hg.P_MIXED)
    out = h.eval(_cuda(x), _cuda(t))
    torch.cuda.synchronize()
    assert (out["status"].cpu().numpy() == hg.Q_NOT_CONVERGED).all()
    assert (out["iters"].cpu().numpy() == 5).all()
    full = hg.Hopf(A, 0, tol=TOL, max_iter=3000, precision=hg.P_MIXED).eval(_cuda(x), _cuda(t))
    torch.cuda.synchronize()
    need = full["iters"].cpu().numpy()
    cap = int(need.max()) + 2
    out = hg.Hopf(A, 0, tol=TOL, max_iter=cap, precision=hg.P_MIXED).eval(_cuda(x), _cuda(t))
    torch.cuda.synchronize()
    assert (out["status"].cpu().numpy() == hg.Q_OK).all()
    assert torch.equal(out["iters"], full["iters"])
    with pytest.raises(hg.HopfError) as e:
        h.set_split_start(-1.0)
    assert e.value.status == hg.HOPF_EINVAL
    h2 = hg.Hopf(A, 2, tol=TOL, max_iter=10, precision=hg.P_MIXED)  # l2: one stage
    with pytest.raises(hg.HopfError) as e:
        h2.set_split_start(1e-10)
    assert e.value.status == hg.HOPF_EUNSUPPORTED
    h2.set_split_start(0.0)


@pytest.mark.parametrize("precision", ["FP32", "SPLIT", "MIXED", "BF16"])
def test_dense_not_spd(hg, precision):
    """A + lambda I with a negative eigenvalue is refused for every dense form:
    MIXED and BF16 sweep in FP32 and confirm a non-positive pivot in FP64,
    the others sweep in FP64.  An SPD matrix whose FP32 sweep is accurate
    enough is accepted by all (n = 200: a ragged last pivot block)."""
    A = np.eye(200)
    A[3, 3] = -5.0
    with pytest.raises(hg.HopfError) as e:
        hg.Hopf(A, 0, tol=1e-12, max_iter=10, precision=getattr(hg, "P_" + precision))
    assert e.value.status == hg.HOPF_ENOTSPD
    A[3, 3] = 0.5
    hg.Hopf(A, 0, tol=1e-12, max_iter=10, precision=getattr(hg, "P_" + precision))


@pytest.mark.parametrize("precision,h_kind", [("MIXED", 1), ("SPLIT", 1), ("SPLIT", 2)])
def test_compaction_does_not_change_results(hg, orc, precision, h_kind):
    """Packing the active queries into fewer column tiles as others converge
    moves a query's columns but not its arithmetic: with and without it the
    outputs agree bit for bit.  (2,000 queries: 16 column tiles, so several
    packings happen; the SPLIT form packs the operand pair of the iteration's
    parity, and for l2 the M y plane that replaced y.)"""
    import torch
    n, B = 256, 2000
    A, Q, s = wl.spd_matrix(11801, 11802, n)
    w = wl.uniform(11803, n, 0.5, 1.5)
    x = wl.normal(11804, B * n, 2.0).reshape(B, n).astype(np.float32)
    t = wl.uniform(11805, B, 0.1, 3.0).astype(np.float32)
    t[::7] = 0.0  # queries that converge almost at once
    outs = []
    wk = w if h_kind == 1 else None
    for on in (True, False):
        h = hg.Hopf(A, h_kind, w=wk, tol=TOL, max_iter=3000, precision=getattr(hg, "P_" + precision))
        h.set_compaction(on)
        outs.append(h.eval(_cuda(x), _cuda(t)))
    torch.cuda.synchronize()
    for key in ("phi", "grad", "iters", "status", "dphidt"):
        assert torch.equal(outs[0][key], outs[1][key]), key
    ref = orc.Problem(A, h_kind, w=wk, tol=1e-28, max_iter=50000, stop_rule=orc.STOP_UREL).eval(
        x[:64].astype(np.float64), t[:64].astype(np.float64))
    phi = outs[0]["phi"][:64].cpu().numpy()
    assert (np.abs(phi - ref["phi"]) / np.maximum(1, np.abs(ref["phi"]))).max() <= PHI_TOL


@pytest.mark.parametrize("precision,h_kind,n", [("MIXED", 1, 256), ("MIXED", 0, 512), ("SPLIT", 1, 256),
                                                ("SPLIT", 2, 512), ("BF16", 1, 256)])
def test_sm_pairs_match_single_ctas(hg, orc, precision, h_kind, n):
    """An SM pair (two CTAs, one M = 256 MMA per K step over both CTAs' A
    tiles and the two halves of the query tile) forms every product from the
    same operands in the same K order as two CTAs with one 128-row tile each:
    the outputs agree bit for bit, through compactions and the final pass.
    The row-tile count is even here (2 or 4); with an odd count (n = 384)
    the pair switch keeps single CTAs (test_sm_pairs_odd_row_tiles)."""
    import torch
    B = 2000
    A, Q, s = wl.spd_matrix(11811 + n, 11812 + n, n)
    w = wl.uniform(11813, n, 0.5, 1.5)
    x = wl.normal(11814, B * n, 2.0).reshape(B, n).astype(np.float32)
    t = wl.uniform(11815, B, 0.1, 3.0).astype(np.float32)
    t[::7] = 0.0
    wk = w if h_kind == 1 else None
    outs = []
    for pairs in (True, False):
        h = hg.Hopf(A, h_kind, w=wk, tol=TOL if precision != "BF16" else 1e-6, max_iter=3000,
                    precision=getattr(hg, "P_" + precision))
        h.set_tc_pairs(pairs)
        outs.append(h.eval(_cuda(x), _cuda(t)))
    torch.cuda.synchronize()
    for key in ("phi", "grad", "iters", "status", "dphidt"):
        assert torch.equal(outs[0][key], outs[1][key]), key
    if precision == "BF16":
        return
    ref = orc.Problem(A, h_kind, w=wk, tol=1e-28, max_iter=50000, stop_rule=orc.STOP_UREL).eval(
        x[:64].astype(np.float64), t[:64].astype(np.float64))
    ephi, eg = _errors({k: v[:64] for k, v in outs[0].items()}, ref)
    gmax, _ = GRAD_BARS[precision]
    assert ephi.max() <= PHI_TOL and eg.max() <= gmax, (ephi.max(), eg.max())


def test_sm_pairs_odd_row_tiles(hg, orc):
    """Pairs switched on for n = 384 (three 128-row tiles, which do not pair
    up) and for n = 200 with one query (two row tiles, one column tile: the
    smallest pair grid): results within the oracle bars."""
    import torch
    for n, B, h_kind in ((384, 257, 0), (200, 1, 1)):
        A, w, x, t, ref = _case(orc, n, B, h_kind, 11000 + n + h_kind)
        h = hg.Hopf(A, h_kind, w=w, tol=TOL, max_iter=3000, precision=hg.P_MIXED)
        h.set_tc_pairs(True)
        out = h.eval(_cuda(x), _cuda(t))
        torch.cuda.synchronize()
        ephi, eg = _errors(out, ref)
        assert ephi.max() <= PHI_TOL and eg.max() <= GRAD_MAX, (n, ephi.max(), eg.max())


def test_batch_beyond_the_compaction_table(hg, orc):
    """More column tiles (1,094 for 140,000 queries) than the shared-memory
    table of packing offsets holds (1,024): the solver runs without packing
    until the active tiles fit, with the same results as the oracle on
    sampled queries (first, middle, and the ragged last tile)."""
    import torch
    n, B = 128, 140000
    A, Q, s = wl.spd_matrix(11901, 11902, n)
    x = wl.normal(11904, B * n, 2.0).reshape(B, n).astype(np.float32)
    t = wl.uniform(11905, B, 0.1, 3.0).astype(np.float32)
    h = hg.Hopf(A, 0, tol=TOL, max_iter=3000, precision=hg.P_MIXED)
    out = h.eval(_cuda(x), _cuda(t))
    torch.cuda.synchronize()
    assert (out["status"].cpu().numpy() == hg.Q_OK).all()
    idx = np.array([0, 1, 70000, 70001, B - 2, B - 1])
    ref = orc.Problem(A, 0, tol=1e-28, max_iter=50000, stop_rule=orc.STOP_UREL).eval(
        x[idx].astype(np.float64), t[idx].astype(np.float64))
    phi = out["phi"].cpu().numpy()[idx]
    g = out["grad"].cpu().numpy()[idx].astype(np.float64)
    assert (np.abs(phi - ref["phi"]) / np.maximum(1, np.abs(ref["phi"]))).max() <= PHI_TOL
    eg = np.linalg.norm(g - ref["grad"], axis=1) / np.maximum(1, np.linalg.norm(ref["grad"], axis=1))
    assert eg.max() <= GRAD_MAX, eg.max()
