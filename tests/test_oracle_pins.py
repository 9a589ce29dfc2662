"""Pins of the FP64 oracle against routes that do not share its arithmetic.

Each test names the passage of the paper (or the piece of mathematics) it
checks.  Sizes are small so the whole CPU suite runs in a few minutes.
"""
import os

import numpy as np
import pytest

import workloads as wl
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense(n, seed, s_lo=0.1, s_hi=10.0):
    A, Q, s = wl.spd_matrix(seed, seed + 1, n, s_lo, s_hi)
    Ainv = (Q / s) @ Q.T
    return A, Ainv


# ---- P1: closed forms ------------------------------------------------------

def test_workload1_closed_form(orc):
    """Workload 1 (n = 8, diagonal A, H = l1, FP64, tol 1e-10): the oracle
    agrees with phi = sum shrink_1(x_i,t)^2/(2 a_i) - 1/2 and
    grad = shrink_1(x,t)/a (decoupled minimisation of Section 1)."""
    d = wl.diag_l1_fp64()
    P = orc.Problem(d["a"], orc.H_L1, tol=d["tol"], max_iter=d["max_iter"])
    r = P.eval(d["x"], d["t"])
    assert r["converged"].all()
    for q in range(len(d["t"])):
        phi, g = pins.closed_diag_wl1(d["x"][q], d["t"][q], d["a"])
        assert abs(r["phi"][q] - phi) <= 1e-8 * max(1, abs(phi))
        # the stop rule leaves steps |d^K - d^{K-1}| <= 1e-5; with a_i in
        # [0.5, 2] and lambda = 1 the iteration contracts by about 1/3 per step,
        # so the distance to the fixed point is below 5e-5
        assert np.abs(r["grad"][q] - g).max() <= 5e-5
        # the returned iterate is d^K: exact zeros where |x_i| <= t
        assert np.all(r["grad"][q][np.abs(d["x"][q]) <= d["t"][q]] == 0.0)


@pytest.mark.parametrize("lam", [0.5, 1.0, 2.0])
def test_paper_example_l1_ellipsoid(orc, lam):
    """Section 1 worked example: J = 1/2 (sum x_i^2/a_i^2 - 1), H = l1, i.e.
    A = diag(a^2).  lambda != 1 catches a lambda dropped from one of
    eq. 3.4(a)-(b) (the fixed point does not depend on lambda)."""
    rng = np.random.default_rng(1)
    n = 6
    a = rng.uniform(0.5, 2.0, n)
    x = rng.uniform(-4, 4, (50, n))
    t = rng.uniform(0.1, 2.0, 50)
    P = orc.Problem(a ** 2, orc.H_L1, lam=lam, tol=1e-26, max_iter=5000)
    r = P.eval(x, t)
    for q in range(50):
        phi, g = pins.paper_example_l1(x[q], t[q], a)
        assert abs(r["phi"][q] - phi) <= 1e-10 * max(1, abs(phi))
        assert np.abs(r["grad"][q] - g).max() <= 1e-10


@pytest.mark.parametrize("lam", [0.5, 1.0, 3.0])
def test_weighted_l1_with_centre(orc, lam):
    """Weighted l1 with a centre c: v_i = shrink_1(y_i, t w_i)/a_i, y = x - c."""
    rng = np.random.default_rng(2)
    n = 9
    a = rng.uniform(0.3, 3.0, n)
    w = rng.uniform(0.5, 1.5, n)
    c = rng.normal(size=n)
    x = rng.normal(scale=3, size=(40, n))
    t = rng.uniform(0.05, 2.0, 40)
    P = orc.Problem(a, orc.H_WL1, w=w, centre=c, lam=lam, tol=1e-26, max_iter=5000)
    r = P.eval(x, t)
    for q in range(40):
        phi, g = pins.closed_diag_wl1(x[q] - c, t[q], a, w)
        assert abs(r["phi"][q] - phi) <= 1e-10 * max(1, abs(phi))
        assert np.abs(r["grad"][q] - g).max() <= 1e-10
        assert abs(r["dphidt"][q] + (w * np.abs(g)).sum()) <= 1e-9


def test_paper_example_sphere(orc):
    """Section 1: the unit sphere moved outward by H = l2 (A = I, c0 = 1/2)."""
    rng = np.random.default_rng(3)
    n = 5
    x = rng.normal(scale=2, size=(60, n))
    t = rng.uniform(0.1, 4.0, 60)
    P = orc.Problem(np.ones(n), orc.H_L2, tol=1e-26, max_iter=5000)
    r = P.eval(x, t)
    for q in range(60):
        phi = pins.paper_example_sphere(x[q], t[q])
        assert abs(r["phi"][q] - phi) <= 1e-10 * max(1, abs(phi))
        assert np.abs(r["grad"][q] - pins.shrink2(x[q], t[q])).max() <= 1e-10


@pytest.mark.parametrize("lam", [0.7, 1.0])
def test_diag_l2_secular(orc, lam):
    """Diagonal A with H = l2 (every part of the ellipsoid-union workload):
    the secular-equation solution by bisection."""
    rng = np.random.default_rng(4)
    n = 16
    a = rng.uniform(0.04, 25.0, n)
    c = rng.normal(scale=3, size=n)
    x = rng.normal(scale=5, size=(40, n))
    t = rng.uniform(0.0, 2.0, 40)
    P = orc.Problem(a, orc.H_L2, centre=c, lam=lam, tol=1e-28, max_iter=20000)
    r = P.eval(x, t)
    for q in range(40):
        phi, v = pins.diag_l2_secular(x[q] - c, t[q], a)
        assert abs(r["phi"][q] - phi) <= 1e-9 * max(1, abs(phi))
        assert np.abs(r["grad"][q] - v).max() <= 1e-8 * max(1, np.abs(v).max())


# ---- P3 / P4: dense A, certificates -----------------------------------------

@pytest.mark.parametrize("lam", [1.0, 2.5])
def test_dense_wl1_kkt_certificate(orc, lam):
    """Dense SPD A, weighted l1 (the n = 1024 workload's form at n = 48): the
    oracle's support and signs give an exact active-set solution that satisfies
    the optimality conditions of eq. 3.3, and the oracle matches it."""
    n = 48
    A, Ainv = _dense(n, 7001)
    w = wl.uniform(7003, n, 0.5, 1.5)
    x = wl.normal(7004, 30 * n, 2.0).reshape(30, n)
    t = wl.uniform(7005, 30, 0.1, 3.0)
    P = orc.Problem(A, orc.H_WL1, w=w, lam=lam, tol=1e-28, max_iter=20000, stop_rule=orc.STOP_UREL)
    r = P.eval(x, t)
    assert r["converged"].all()
    for q in range(30):
        v, ok = pins.kkt_active_set(A, x[q], t[q], w, r["grad"][q])
        assert ok, q
        assert np.abs(r["grad"][q] - v).max() <= 1e-10 * max(1, np.abs(v).max())
        phi = pins.objective_neg(A, x[q], t[q], w, v)
        assert abs(r["phi"][q] - phi) <= 1e-11 * max(1, abs(phi))


@pytest.mark.parametrize("h", ["wl1", "l2"])
def test_dense_duality_gap(orc, h):
    """Lower bound -F(v) <= phi <= J(x - t c) for any c in C (Hopf-Lax form of
    Section 2.2); at the oracle's answer the gap closes to rounding level."""
    n = 40
    A, Ainv = _dense(n, 7101)
    w = wl.uniform(7103, n, 0.5, 1.5) if h == "wl1" else None
    x = wl.normal(7104, 25 * n, 2.0).reshape(25, n)
    t = wl.uniform(7105, 25, 0.1, 3.0)
    kind = orc.H_WL1 if h == "wl1" else orc.H_L2
    P = orc.Problem(A, kind, w=w, tol=1e-28, max_iter=20000, stop_rule=orc.STOP_UREL)
    r = P.eval(x, t)
    for q in range(25):
        v = r["grad"][q]
        lower = pins.objective_neg(A, x[q], t[q], w, v, h=h)
        upper = pins.hopf_lax_upper(Ainv, A, x[q], t[q], w, v, h=h)
        assert lower <= r["phi"][q] + 1e-12 * max(1, abs(lower))
        assert upper - lower <= 1e-9 * max(1, abs(upper)), (q, upper - lower)


# ---- P5: brute-force Hopf-Lax at n = 2 ---------------------------------------

@pytest.mark.parametrize("h", ["l1", "wl1", "l2"])
def test_hopf_lax_bruteforce_n2(orc, h):
    rng = np.random.default_rng(11)
    for trial in range(12):
        G = rng.normal(size=(2, 2))
        A = G @ G.T + 0.3 * np.eye(2)
        Ainv = np.linalg.inv(A)
        w = rng.uniform(0.5, 1.5, 2) if h == "wl1" else np.ones(2)
        x = rng.normal(scale=2, size=2)
        t = rng.uniform(0.1, 2.0)
        kind = {"l1": orc.H_L1, "wl1": orc.H_WL1, "l2": orc.H_L2}[h]
        P = orc.Problem(A, kind, w=w if h == "wl1" else None, tol=1e-28, max_iter=20000, stop_rule=orc.STOP_UREL)
        r = P.eval(x[None], [t])
        bf = pins.hopf_lax_bruteforce_2d(Ainv, x, t, w, h="l2" if h == "l2" else "wl1")
        assert abs(r["phi"][0] - bf) <= 1e-9 * max(1, abs(bf)), (trial, r["phi"][0], bf)


# ---- P6: invariants -------------------------------------------------------

def test_initial_condition_and_shift(orc):
    """phi(x, 0) = J(x) (eq. 1.1b) and phi(x; c) = phi(x - c; 0)."""
    n = 20
    A, Ainv = _dense(n, 7201)
    c = wl.normal(7206, n, 1.0)
    x = wl.normal(7204, 10 * n, 2.0).reshape(10, n)
    P = orc.Problem(A, orc.H_L2, centre=c, tol=1e-28, max_iter=20000, stop_rule=orc.STOP_UREL)
    r0 = P.eval(x, np.zeros(10))
    for q in range(10):
        J = pins.J_value(Ainv, x[q] - c)
        assert abs(r0["phi"][q] - J) <= 1e-11 * max(1, abs(J))
    t = np.full(10, 0.8)
    r1 = P.eval(x, t)
    P0 = orc.Problem(A, orc.H_L2, tol=1e-28, max_iter=20000, stop_rule=orc.STOP_UREL)
    r2 = P0.eval(x - c, t)
    assert np.allclose(r1["phi"], r2["phi"], rtol=1e-12, atol=1e-12)


def test_time_derivative_and_gradient_fd(orc):
    """d phi/dt = -H(grad phi) (the PDE, eq. 1.1a) and grad_x phi = d^K, both
    by FP64 central differences; phi is non-increasing in t (H >= 0)."""
    n = 12
    A, Ainv = _dense(n, 7301)
    w = wl.uniform(7303, n, 0.5, 1.5)
    P = orc.Problem(A, orc.H_WL1, w=w, tol=1e-30, max_iter=50000, stop_rule=orc.STOP_UREL)
    x = wl.normal(7304, n, 2.0)
    t = 0.9
    h = 1e-5
    r = P.eval(x[None], [t])
    rp, rm = P.eval(x[None], [t + h]), P.eval(x[None], [t - h])
    fd_t = (rp["phi"][0] - rm["phi"][0]) / (2 * h)
    assert abs(fd_t - r["dphidt"][0]) <= 1e-6 * max(1, abs(fd_t))
    assert rp["phi"][0] <= r["phi"][0] <= rm["phi"][0]
    X = np.repeat(x[None], 2 * n, 0)
    for i in range(n):
        X[2 * i, i] += h
        X[2 * i + 1, i] -= h
    rr = P.eval(X, np.full(2 * n, t))
    fd_x = (rr["phi"][0::2] - rr["phi"][1::2]) / (2 * h)
    assert np.abs(fd_x - r["grad"][0]).max() <= 1e-6 * max(1, np.abs(fd_x).max())


# ---- P7: union and closest point --------------------------------------------

def _union_parts(orc, K, n, seed, tol=1e-28):
    semi = wl.log_uniform(seed, K * n, 0.2, 5.0).reshape(K, n)
    cen = wl.normal(seed + 4, K * n, 3.0).reshape(K, n)
    parts = [orc.Problem(semi[k] ** 2, orc.H_L2, centre=cen[k], tol=tol, max_iter=50000,
                         stop_rule=orc.STOP_UREL) for k in range(K)]
    return semi, cen, parts


def test_union_min_rule(orc):
    """phi = min_i phi_i (Section 2.2) with each phi_i from the secular
    equation, and its gradient the minimising part's; at t = 0 it is
    min_i J_i(x)."""
    K, n = 4, 10
    semi, cen, parts = _union_parts(orc, K, n, 7401)
    x = wl.normal(7404, 20 * n, 5.0).reshape(20, n)
    t = wl.uniform(7405, 20, 0.0, 2.0)
    t[:3] = 0.0
    r = orc.union_eval(parts, x, t)
    assert len(set(r["argmin"][3:].tolist())) >= 2  # the minimum moves between parts
    for q in range(20):
        sol = [pins.diag_l2_secular(x[q] - cen[k], t[q], semi[k] ** 2) for k in range(K)]
        vals = [v for v, _ in sol]
        k = int(np.argmin(vals))
        assert r["argmin"][q] == k
        assert abs(r["phi"][q] - vals[k]) <= 1e-9 * max(1, abs(vals[k]))
        gk = sol[k][1]
        assert np.linalg.norm(r["grad"][q] - gk) <= 1e-7 * max(1, np.linalg.norm(gk)), q
        if t[q] == 0:
            J = min(0.5 * (((x[q] - cen[j]) / semi[j]) ** 2).sum() - 0.5 for j in range(K))
            assert abs(r["phi"][q] - J) <= 1e-11 * max(1, abs(J))


def test_closest_point_against_ellipsoid_projection(orc):
    """Distance and closest point by Newton on s over the eikonal solution
    (Section 3.2) agree with the ellipsoid projection of Section 4.3."""
    K, n = 3, 8
    semi, cen, parts = _union_parts(orc, K, n, 7501, tol=1e-28)
    x = wl.normal(7504, 40 * n, 5.0).reshape(40, n)
    inside = np.zeros(40, bool)
    for k in range(K):
        inside |= (((x - cen[k]) / semi[k]) ** 2).sum(1) <= 1
    x = x[~inside][:12]
    r = orc.union_closest(parts, x, s_tol=1e-13, max_newton=100)
    assert r["newton_fail"] == 0
    for q in range(len(x)):
        best, bk, bp = np.inf, -1, None
        for k in range(K):
            p, _ = pins.ellipsoid_projection(x[q] - cen[k], semi[k])
            dk = np.linalg.norm(x[q] - cen[k] - p)
            if dk < best:
                best, bk, bp = dk, k, p + cen[k]
        assert r["argmin"][q] == bk
        assert abs(r["dist"][q] - best) <= 1e-9 * max(1, best)
        assert np.abs(r["closest"][q] - bp).max() <= 1e-7 * max(1, np.abs(bp).max())


# ---- P8: envelope gradients ---------------------------------------------------

def test_backward_envelope_fd(orc):
    """dphi/dA = -1/2 v v^T, dphi/dx = v, dphi/dt = -H(v) (envelope theorem on
    eq. 3.3), by central differences of exact active-set values (symmetric
    perturbation of A_ij and A_ji together gives twice the (i,j) entry)."""
    n = 10
    A, Ainv = _dense(n, 7601)
    w = np.ones(n)
    x = wl.normal(7604, n, 2.0)
    t = 0.7
    P = orc.Problem(A, orc.H_L1, tol=1e-30, max_iter=50000, stop_rule=orc.STOP_UREL)
    r = P.eval(x[None], [t])
    v = r["grad"][0]
    b = orc.backward(n, orc.A_DENSE, orc.H_L1, None, [1.0], v[None], [t])
    h = 1e-6

    def phi_exact(Am):
        vv, ok = pins.kkt_active_set(Am, x, t, w, v)
        assert ok
        return pins.objective_neg(Am, x, t, w, vv)

    for (i, j) in [(0, 0), (3, 3), (1, 4), (2, 7), (9, 5)]:
        E = np.zeros((n, n))
        E[i, j] += h
        E[j, i] += h if i != j else 0.0
        fd = (phi_exact(A + E) - phi_exact(A - E)) / (2 * h)
        expect = b["g_A"][i, j] * (1 if i == j else 2)
        assert abs(fd - expect) <= 1e-6 * max(1, abs(expect)), (i, j, fd, expect)
    assert np.allclose(b["g_x"][0], v)
    assert abs(b["g_t"][0] + np.abs(v).sum()) <= 1e-12


def test_backward_diagonal_A_fd(orc):
    """Diagonal A with H = l1 decouples (Section 1): phi = sum_i
    shrink_1(x_i, t)^2 / (2 a_i) - c0.  The oracle's diagonal g_A (with an
    upstream weight g) matches central differences of that closed form in
    each a_i, and g_x, g_t match g v and -g H(v)."""
    n = 7
    a = wl.uniform(7611, n, 0.5, 2.0)
    x = wl.normal(7612, n, 2.0)
    t, g = 0.6, 1.7
    P = orc.Problem(a, orc.H_L1, tol=1e-30, max_iter=50000, stop_rule=orc.STOP_UREL)
    v = P.eval(x[None], [t])["grad"][0]
    b = orc.backward(n, orc.A_DIAG, orc.H_L1, None, [g], v[None], [t])
    s = np.sign(x) * np.maximum(np.abs(x) - t, 0.0)
    assert (np.abs(s) > 0).sum() >= 2 and (s == 0).sum() >= 1  # both kinds of coordinate

    def phi(av):
        return (s * s / (2 * av)).sum() - 0.5

    h = 1e-6
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd = g * (phi(a + e) - phi(a - e)) / (2 * h)
        assert abs(b["g_A"][i] - fd) <= 1e-7 * max(1, abs(fd)), (i, b["g_A"][i], fd)
    assert np.allclose(b["g_x"][0], g * v, rtol=1e-12, atol=1e-14)
    assert abs(b["g_t"][0] + g * np.abs(v).sum()) <= 1e-12


def test_golden_section1_example(orc):
    """A fixed worked instance of the Section 1 example (values written by
    tests/golden/make_golden.py from the closed form, not from the oracle)."""
    path = os.path.join(GOLDEN, "section1_l1_ellipsoid.txt")
    rows = np.loadtxt(path, comments="#")
    n = (rows.shape[1] - 2) // 3
    for row in rows:
        a = row[:n]; x = row[n:2 * n]; t = row[2 * n]; phi = row[2 * n + 1]; g = row[2 * n + 2:]
        P = orc.Problem(a ** 2, orc.H_L1, tol=1e-28, max_iter=20000)
        r = P.eval(x[None], [t])
        assert abs(r["phi"][0] - phi) <= 1e-10 * max(1, abs(phi))
        assert np.abs(r["grad"][0] - g).max() <= 1e-10


# ---- P9: optimal control and terminal point (Section 2) ---------------------

def _dual_ball_excess(beta, h, w):
    """How far beta lies outside the unit ball of the dual norm of H."""
    if h == "l2":
        return max(0.0, np.linalg.norm(beta) - 1.0)
    return max(0.0, float(np.max(np.abs(beta) - w)))


@pytest.mark.parametrize("h", ["l1", "wl1", "l2"])
@pytest.mark.parametrize("dense", [False, True])
def test_control_is_a_subgradient_and_the_hopf_lax_minimiser(orc, h, dense):
    """beta = (x - c - A p)/t must lie in dH(p): equal to grad H(p) where H is
    differentiable (w_i sign p_i for p_i != 0; p / |p| for l2), inside the dual
    ball where it is not, and <beta, p> = H(p) (1-homogeneity).  The terminal
    point x_T = x - t beta must be the Hopf-Lax minimiser: x - x_T in t C and
    J(x_T) = phi(x, t)."""
    n, B = 12, 24
    kind = {"l1": orc.H_L1, "wl1": orc.H_WL1, "l2": orc.H_L2}[h]
    w = wl.uniform(9101, n, 0.5, 1.5) if h == "wl1" else np.ones(n)
    c = wl.normal(9106, n, 0.5)
    if dense:
        A, Ainv = _dense(n, 9102, 0.3, 3.0)
    else:
        A = wl.uniform(9102, n, 0.5, 2.0)
        Ainv = np.diag(1.0 / A)
    x = wl.normal(9104, B * n, 2.0).reshape(B, n)
    t = wl.uniform(9105, B, 0.2, 2.0)
    P = orc.Problem(A, kind, w=w if h == "wl1" else None, centre=c, tol=1e-30, max_iter=50000,
                    stop_rule=orc.STOP_UREL)
    r = P.eval(x, t)
    ctl = orc.control(P, x, t, r["grad"])
    beta, xT = ctl["beta"], ctl["x_T"]
    for q in range(B):
        p = r["grad"][q]
        if h == "l2":
            if np.linalg.norm(p) > 1e-9:
                assert np.allclose(beta[q], p / np.linalg.norm(p), atol=1e-7)
        else:
            on = np.abs(p) > 1e-9
            assert np.allclose(beta[q][on], (w * np.sign(p))[on], atol=1e-7)
        assert _dual_ball_excess(beta[q], h, w) <= 1e-7
        Hp = P.H(p)
        assert abs(beta[q] @ p - Hp) <= 1e-8 * max(1.0, Hp)
        # Hopf-Lax: x_T = x - t beta attains phi
        z = xT[q] - c
        J = 0.5 * z @ Ainv @ z - 0.5
        assert abs(J - r["phi"][q]) <= 1e-8 * max(1.0, abs(r["phi"][q]))
    # t = 0: no control, the point stays
    ctl0 = orc.control(P, x[:2], np.zeros(2), r["grad"][:2])
    assert np.all(ctl0["beta"] == 0) and np.array_equal(ctl0["x_T"], x[:2])


@pytest.mark.parametrize("h", ["wl1", "l2"])
def test_terminal_point_bruteforce_n2(orc, h):
    """n = 2: the terminal point against brute-force minimisation of J over
    the set x - t C (Hopf-Lax), which shares nothing with split Bregman."""
    rng = np.random.default_rng(17)
    for trial in range(10):
        G = rng.normal(size=(2, 2))
        A = G @ G.T + 0.3 * np.eye(2)
        Ainv = np.linalg.inv(A)
        w = rng.uniform(0.5, 1.5, 2) if h == "wl1" else np.ones(2)
        x = rng.normal(scale=2, size=2)
        t = rng.uniform(0.1, 2.0)
        P = orc.Problem(A, orc.H_WL1 if h == "wl1" else orc.H_L2, w=w if h == "wl1" else None, tol=1e-30,
                        max_iter=50000, stop_rule=orc.STOP_UREL)
        r = P.eval(x[None], [t])
        xT = orc.control(P, x[None], [t], r["grad"])["x_T"][0]
        val, cbest = pins.hopf_lax_argmin_2d(Ainv, x, t, w, h=h)
        assert np.linalg.norm(xT - (x - t * cbest)) <= 1e-5 * max(1.0, np.linalg.norm(xT)), (trial, xT, x - t * cbest)


# ---- P10: maximum over Hamiltonians (Section 2.2) --------------------------

def test_max_over_hamiltonians_solves_the_min_hamiltonian_pde(orc):
    """With one J and Hamiltonians H_1 = weighted l1 (weights 0.3 and 1.5, so
    it lies below l2 along one axis and above it along the other) and
    H_2 = l2, max_i phi_i must equal brute-force Hopf-Lax values per part and
    satisfy d phi/dt = -min_i H_i(grad phi) (central differences in t)."""
    rng = np.random.default_rng(23)
    w = np.array([0.3, 1.5])
    seen = set()
    for trial in range(16):
        G = rng.normal(size=(2, 2))
        A = G @ G.T + 0.3 * np.eye(2)
        Ainv = np.linalg.inv(A)
        x = rng.normal(scale=2, size=2)
        t = rng.uniform(0.3, 2.0)
        parts = [orc.Problem(A, orc.H_WL1, w=w, tol=1e-30, max_iter=50000, stop_rule=orc.STOP_UREL),
                 orc.Problem(A, orc.H_L2, tol=1e-30, max_iter=50000, stop_rule=orc.STOP_UREL)]
        r = orc.maxH_eval(parts, x[None], [t])
        bf = max(pins.hopf_lax_bruteforce_2d(Ainv, x, t, w, h="wl1"),
                 pins.hopf_lax_bruteforce_2d(Ainv, x, t, np.ones(2), h="l2"))
        assert abs(r["phi"][0] - bf) <= 1e-9 * max(1, abs(bf))
        seen.add(int(r["argmax"][0]))
        hh = 1e-5
        rp = orc.maxH_eval(parts, x[None], [t + hh])
        rm = orc.maxH_eval(parts, x[None], [t - hh])
        if rp["argmax"][0] != r["argmax"][0] or rm["argmax"][0] != r["argmax"][0]:
            continue  # at a switch between parts phi is not differentiable in t
        dphidt = (rp["phi"][0] - rm["phi"][0]) / (2 * hh)
        p = r["grad"][0]
        Hmin = min(float(np.abs(p) @ w), float(np.linalg.norm(p)))
        assert abs(dphidt + Hmin) <= 1e-6 * max(1, Hmin), (trial, dphidt, Hmin)
    assert seen == {0, 1}  # both Hamiltonians win somewhere


# ---- P11: the other Hamiltonians and initial data (Sections 4.2-4.4) -------

def _prox_by_definition(f, z):
    val, u = pins.min_convex(lambda u: f(u) + 0.5 * np.sum((u - z) ** 2), z, 1.0)
    return u


@pytest.mark.parametrize("kind", ["linf", "dnorm"])
def test_new_prox_against_their_definition(orc, kind):
    """prox_{tau H}(z) = argmin tau H(u) + 1/2 |u - z|^2, by numerical
    minimisation in 3-D, for z inside and outside the dual ball."""
    rng = np.random.default_rng(31)
    w = np.array([0.5, 1.3, 2.0])
    for trial in range(8):
        z = rng.normal(scale=1.5, size=3)
        tau = rng.uniform(0.1, 2.5)
        if kind == "linf":
            H = lambda u: np.abs(u).max()
            got = orc.prox(orc.H_LINF, tau, z)
        else:
            H = lambda u: np.sqrt(np.sum(w * u * u))
            got = orc.prox(orc.H_DNORM, tau, z, w)
        ref = _prox_by_definition(lambda u: tau * H(u), z)
        assert np.abs(got - ref).max() <= 1e-6, (trial, got, ref)


def test_l2sq_initial_data_closed_forms_new_H(orc):
    """J = 1/2 |x|^2: phi(x,t) = min over y in x - tC of J(y) (Hopf-Lax), so
    phi = 1/2 |x - pi_{tC}(x)|^2 and grad phi = x - pi_{tC}(x), with C the
    l1 ball (H = l_inf) or the ellipsoid {sum y_i^2 / w_i <= 1}
    (H = sqrt(sum w p^2)); the projections come from bisection and from the
    secular-equation projection of Section 4.3 written independently."""
    n, B = 7, 16
    x = wl.uniform(9201, B * n, -3.0, 3.0).reshape(B, n)
    t = wl.uniform(9202, B, 0.1, 2.0)
    w = wl.uniform(9203, n, 0.5, 2.0)
    for h in ("linf", "dnorm"):
        P = orc.Problem(np.ones(n), orc.H_LINF if h == "linf" else orc.H_DNORM, w=w if h == "dnorm" else None,
                        c0=0.0, tol=1e-30, max_iter=200000, stop_rule=orc.STOP_UREL)
        r = P.eval(x, t)
        for q in range(B):
            if h == "linf":
                pi = pins.l1ball_projection(x[q], t[q])
            else:
                pi = pins.ellipsoid_projection(x[q], t[q] * np.sqrt(w))[0]
            g = x[q] - pi
            assert abs(r["phi"][q] - 0.5 * g @ g) <= 1e-9 * max(1, 0.5 * g @ g), (h, q)
            assert np.abs(r["grad"][q] - g).max() <= 1e-7, (h, q)


@pytest.mark.parametrize("j", ["l1sq", "linfsq"])
@pytest.mark.parametrize("h", ["l1", "l2", "linf"])
@pytest.mark.parametrize("lam", [1.0, 0.5, 2.5])
def test_nonquadratic_initial_data_bruteforce_n2(orc, j, h, lam):
    """J = 1/2 |x|_1^2 or 1/2 |x|_inf^2 (Section 4.4) at n = 2: phi against
    direct minimisation of the Hopf objective J*(v) + t H(v) - <x, v>
    (J* = 1/2 |v|_inf^2 resp. 1/2 |v|_1^2), phi(x, 0) = J(x), and
    d phi/dt = -H(grad phi) by central differences.  phi does not depend on
    the split Bregman lambda, which scales the prox of J* (the Moreau identity
    with alpha = 1 / lambda): lambda != 1 checks that scaling."""
    rng = np.random.default_rng(41)
    jk = orc.J_L1SQ if j == "l1sq" else orc.J_LINFSQ
    hk = {"l1": orc.H_L1, "l2": orc.H_L2, "linf": orc.H_LINF}[h]
    Jstar = (lambda v: 0.5 * np.abs(v).max() ** 2) if j == "l1sq" else (lambda v: 0.5 * np.abs(v).sum() ** 2)
    J = (lambda z: 0.5 * np.abs(z).sum() ** 2) if j == "l1sq" else (lambda z: 0.5 * np.abs(z).max() ** 2)
    Hf = {"l1": lambda v: np.abs(v).sum(), "l2": np.linalg.norm, "linf": lambda v: np.abs(v).max()}[h]
    P = orc.Problem(None, hk, c0=0.0, lam=lam, tol=1e-30, max_iter=200000, stop_rule=orc.STOP_UREL, j_kind=jk,
                    n=2)
    for trial in range(4):
        x = rng.uniform(-3, 3, 2)
        t = rng.uniform(0.2, 2.0)
        r = P.eval(x[None], [t])
        val, v = pins.min_convex(lambda v: Jstar(v) + t * Hf(v) - x @ v, np.zeros(2), 1.0)
        assert abs(r["phi"][0] + val) <= 1e-7 * max(1, abs(val)), (trial, r["phi"][0], -val)
        r0 = P.eval(x[None], [0.0])
        assert abs(r0["phi"][0] - J(x)) <= 1e-9 * max(1, J(x))
        hh = 1e-5
        rp, rm = P.eval(x[None], [t + hh]), P.eval(x[None], [t - hh])
        dphidt = (rp["phi"][0] - rm["phi"][0]) / (2 * hh)
        assert abs(dphidt + Hf(r["grad"][0])) <= 1e-5 * max(1, abs(dphidt)), (trial, dphidt, Hf(r["grad"][0]))


# ---- P12: H = sqrt(<p, M p>) with a dense SPD M (Section 4.3) ---------------

def _spd(rng, n, lo=0.3, hi=3.0):
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    return Q, (Q * rng.uniform(lo, hi, n)) @ Q.T


def _ellipsoid_projection_dense(z, M, r):
    """Projection of z on {y : <y, M^-1 y> <= r^2} from its optimality
    condition alone: y = (I + mu M^-1)^-1 z = M (M + mu I)^-1 z with mu >= 0
    found by bisection on <y, M^-1 y> = r^2 (dense solves, no
    eigendecomposition)."""
    Minv = np.linalg.inv(M)
    if z @ Minv @ z <= r * r:
        return z.copy()
    n = len(z)
    y_of = lambda mu: M @ np.linalg.solve(M + mu * np.eye(n), z)
    g = lambda mu: y_of(mu) @ Minv @ y_of(mu) - r * r
    lo, hi = 0.0, 1.0
    while g(hi) > 0:
        hi *= 2
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if g(mid) > 0 else (lo, mid)
    return y_of(0.5 * (lo + hi))


def test_anorm_prox_against_its_definition(orc):
    """prox_{tau H}(z) = argmin tau sqrt(<u, M u>) + 1/2 |u - z|^2 by numerical
    minimisation in 3-D, for a non-symmetric-eigenvector M (a transposed or
    skipped rotation fails), z inside and outside tau times the dual ball."""
    rng = np.random.default_rng(51)
    Q, M = _spd(rng, 3)
    for trial in range(8):
        z = rng.normal(scale=1.5, size=3)
        tau = rng.uniform(0.1, 2.5)
        got = orc.prox(orc.H_ANORM, tau, z, M)
        ref = _prox_by_definition(lambda u: tau * np.sqrt(max(u @ M @ u, 0.0)), z)
        assert np.abs(got - ref).max() <= 1e-6, (trial, got, ref)
    # inside the dual ball the prox is 0
    z = 0.5 * np.linalg.cholesky(M) @ np.array([0.3, -0.2, 0.1])
    assert np.abs(orc.prox(orc.H_ANORM, 1.0, z, M)).max() == 0.0


def test_anorm_diagonal_M_is_the_dnorm(orc):
    """M = diag(w): the same phi and gradient as H = sqrt(sum w p^2)."""
    n, B = 6, 12
    w = wl.uniform(9301, n, 0.5, 2.0)
    a = wl.uniform(9302, n, 0.5, 2.0)
    x = wl.normal(9303, B * n, 2.0).reshape(B, n)
    t = wl.uniform(9304, B, 0.0, 3.0)
    kw = dict(c0=0.5, tol=1e-30, max_iter=200000, stop_rule=orc.STOP_UREL)
    r1 = orc.Problem(a, orc.H_ANORM, w=np.diag(w), **kw).eval(x, t)
    r2 = orc.Problem(a, orc.H_DNORM, w=w, **kw).eval(x, t)
    assert np.abs(r1["phi"] - r2["phi"]).max() <= 1e-12 * max(1, np.abs(r2["phi"]).max())
    assert np.abs(r1["grad"] - r2["grad"]).max() <= 1e-10


def test_anorm_l2sq_initial_data_closed_form(orc):
    """J = 1/2 |x|^2 (A = I): phi = 1/2 |x - pi(x)|^2 and grad phi = x - pi(x)
    with pi the projection on t times the dual ball {y : <y, M^-1 y> <= 1}
    (Hopf-Lax), computed by bisection on the multiplier with dense solves."""
    rng = np.random.default_rng(52)
    n, B = 5, 10
    Q, M = _spd(rng, n)
    x = rng.uniform(-3, 3, (B, n))
    t = rng.uniform(0.1, 2.0, B)
    P = orc.Problem(np.ones(n), orc.H_ANORM, w=M, c0=0.0, tol=1e-30, max_iter=200000, stop_rule=orc.STOP_UREL)
    r = P.eval(x, t)
    for q in range(B):
        g = x[q] - _ellipsoid_projection_dense(x[q], M, t[q])
        assert abs(r["phi"][q] - 0.5 * g @ g) <= 1e-9 * max(1, 0.5 * g @ g), q
        assert np.abs(r["grad"][q] - g).max() <= 1e-7, q


def test_anorm_rotation_invariance(orc):
    """J = 1/2 |x|^2 is rotation invariant, so with M = Q diag(l) Q^T,
    phi_M(x) = phi_{diag l}(Q^T x) and grad_M(x) = Q grad_{diag l}(Q^T x)."""
    rng = np.random.default_rng(53)
    n, B = 8, 10
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    l = rng.uniform(0.3, 3.0, n)
    M = (Q * l) @ Q.T
    x = rng.normal(scale=2.0, size=(B, n))
    t = rng.uniform(0.0, 3.0, B)
    kw = dict(c0=0.5, tol=1e-30, max_iter=200000, stop_rule=orc.STOP_UREL)
    rM = orc.Problem(np.ones(n), orc.H_ANORM, w=M, **kw).eval(x, t)
    rD = orc.Problem(np.ones(n), orc.H_DNORM, w=l, **kw).eval(x @ Q, t)
    assert np.abs(rM["phi"] - rD["phi"]).max() <= 1e-10 * max(1, np.abs(rD["phi"]).max())
    assert np.abs(rM["grad"] - rD["grad"] @ Q.T).max() <= 1e-8


@pytest.mark.parametrize("j", ["quad", "l1sq", "linfsq"])
def test_anorm_bruteforce_n2(orc, j):
    """n = 2: phi against direct minimisation of J*(v) + t sqrt(<v, M v>) -
    <x, v> for quadratic and norm initial data, and d phi/dt = -H(grad phi)."""
    rng = np.random.default_rng(54)
    Q, M = _spd(rng, 2)
    a = np.array([0.7, 1.6])
    Hf = lambda v: np.sqrt(max(v @ M @ v, 0.0))
    if j == "quad":
        P = orc.Problem(a, orc.H_ANORM, w=M, c0=0.0, lam=0.5, tol=1e-30, max_iter=200000,
                        stop_rule=orc.STOP_UREL)
        Jstar = lambda v: 0.5 * (a * v * v).sum()
    else:
        jk = orc.J_L1SQ if j == "l1sq" else orc.J_LINFSQ
        P = orc.Problem(None, orc.H_ANORM, w=M, c0=0.0, lam=2.5, tol=1e-30, max_iter=200000,
                        stop_rule=orc.STOP_UREL, j_kind=jk, n=2)
        Jstar = (lambda v: 0.5 * np.abs(v).max() ** 2) if j == "l1sq" else (lambda v: 0.5 * np.abs(v).sum() ** 2)
    for trial in range(4):
        x = rng.uniform(-3, 3, 2)
        t = rng.uniform(0.2, 2.0)
        r = P.eval(x[None], [t])
        val, v = pins.min_convex(lambda v: Jstar(v) + t * Hf(v) - x @ v, np.zeros(2), 1.0)
        assert abs(r["phi"][0] + val) <= 1e-7 * max(1, abs(val)), (trial, r["phi"][0], -val)
        hh = 1e-5
        rp, rm = P.eval(x[None], [t + hh]), P.eval(x[None], [t - hh])
        dphidt = (rp["phi"][0] - rm["phi"][0]) / (2 * hh)
        assert abs(dphidt + Hf(r["grad"][0])) <= 1e-5 * max(1, abs(dphidt)), (trial, dphidt)


# ---- P13: breakpoint root finds at tied breakpoints (Sections 4.2, 4.4) -----

def _tied(rng, m):
    """|z| with a run of equal breakpoints at m, larger ones above and smaller
    ones below, random signs."""
    z = np.concatenate([rng.uniform(m, 3 * m, rng.integers(1, 4)), np.full(rng.integers(2, 6), m),
                        rng.uniform(0, m, 3)])
    return z * rng.choice([-1.0, 1.0], len(z))


def test_l1ball_projection_root_on_a_tied_breakpoint(orc):
    """prox of tau |.|_inf = z - projection on the l1 ball of radius tau; with
    tau chosen so that the multiplier is exactly a tied breakpoint (a case that
    a two-sided segment test rejects on both sides by rounding and returns 0),
    against the projection by bisection."""
    rng = np.random.default_rng(61)
    for trial in range(300):
        m = rng.uniform(0.1, 2.0)
        z = _tied(rng, m)
        tau = np.sum(np.maximum(np.abs(z) - m, 0))
        got = orc.prox(orc.H_LINF, tau, z)
        ref = z - pins.l1ball_projection(z, tau)
        assert np.abs(got - ref).max() <= 1e-12 * max(1, np.abs(z).max()), (trial, got, ref)


def test_l1sq_beta_fixed_point_including_ties(orc):
    """beta = alpha |shrink_1(z, beta)|_1 to rounding, for random z and for z
    whose root is exactly a tied breakpoint (alpha = m / sum (|z_i| - m)_+)."""
    rng = np.random.default_rng(62)
    for trial in range(300):
        if trial % 2:
            m = rng.uniform(0.1, 2.0)
            z = _tied(rng, m)
            alpha = m / np.sum(np.maximum(np.abs(z) - m, 0))
        else:
            z = rng.normal(size=rng.integers(1, 12))
            alpha = rng.uniform(0.2, 5.0)
        b = orc.l1sq_beta(z, alpha)
        rhs = alpha * np.sum(np.maximum(np.abs(z) - b, 0))
        assert abs(b - rhs) <= 1e-13 * max(1, abs(b)), (trial, b, rhs)
        if trial % 2:
            assert abs(b - m) <= 1e-13 * max(1, m)


# ---- P14: gradients with respect to c, c0 and w (envelope theorem) ---------

@pytest.mark.parametrize("hk", ["wl1", "dnorm", "l2"])
def test_parameter_gradients_against_finite_differences(orc, hk):
    """d/dc, d/dc0 and d/dw of sum_q g_q phi_q against central differences of
    the oracle's own converged phi (FP64, h = 1e-5): a dropped t, a wrong
    sign or a missing 1/(2H) fails."""
    n, B = 5, 4
    a = wl.uniform(9401, n, 0.5, 2.0)
    c = wl.normal(9402, n, 1.0)
    w = wl.uniform(9403, n, 0.5, 1.5)
    x = wl.normal(9404, B * n, 2.0).reshape(B, n)
    t = wl.uniform(9405, B, 0.3, 2.0)
    g = wl.normal(9406, B, 1.0)
    kind = {"wl1": orc.H_WL1, "dnorm": orc.H_DNORM, "l2": orc.H_L2}[hk]
    ww = w if hk != "l2" else None
    kw = dict(tol=1e-30, max_iter=200000, stop_rule=orc.STOP_UREL)

    def L(cc=c, c0=0.5, wv=ww):
        return float(g @ orc.Problem(a, kind, w=wv, centre=cc, c0=c0, **kw).eval(x, t)["phi"])

    r = orc.Problem(a, kind, w=ww, centre=c, c0=0.5, **kw).eval(x, t)
    bp = orc.backward_params(n, kind, ww, g, r["grad"], t)
    h = 1e-5
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd = (L(cc=c + e) - L(cc=c - e)) / (2 * h)
        assert abs(fd - bp["g_c"][i]) <= 1e-6 * max(1, abs(fd)), ("c", i, fd, bp["g_c"][i])
        if hk != "l2":
            fdw = (L(wv=w + e) - L(wv=w - e)) / (2 * h)
            assert abs(fdw - bp["g_w"][i]) <= 1e-6 * max(1, abs(fdw)), ("w", i, fdw, bp["g_w"][i])
    fd0 = (L(c0=0.5 + h) - L(c0=0.5 - h)) / (2 * h)
    assert abs(fd0 - bp["g_c0"]) <= 1e-8
    assert bp["g_w"] is None if hk == "l2" else bp["g_w"] is not None


def _norm_golden():
    rows = []
    for line in open(os.path.join(GOLDEN, "section4_norm_kinds.txt")):
        if line.startswith("#"):
            continue
        v = [float(s) for s in line.split()]
        kind, n = int(v[0]), int(v[1])
        x = np.array(v[2:2 + n])
        t, phi = v[2 + n], v[3 + n]
        g = np.array(v[4 + n:4 + 2 * n])
        rows.append((kind, x, t, phi, g))
    return rows


def test_golden_norm_kinds(orc):
    """The oracle against hand-checkable Hopf-Lax closed forms of the norm
    kinds (tests/golden/section4_norm_kinds.txt, written by make_golden.py from
    the closed forms, not from the oracle)."""
    spec = {0: (np.ones, orc.H_LINF, None), 1: (None, orc.H_L1, orc.J_LINFSQ), 2: (None, orc.H_LINF, orc.J_L1SQ)}
    for kind, x, t, phi, g in _norm_golden():
        n = len(x)
        mk, hk, jk = spec[kind]
        P = orc.Problem(mk(n) if mk else None, hk, c0=0.0, tol=1e-30, max_iter=200000, stop_rule=orc.STOP_UREL,
                        j_kind=jk, n=n)
        r = P.eval(x[None], [t])
        assert abs(r["phi"][0] - phi) <= 1e-9 * max(1, abs(phi)), (kind, x, r["phi"][0], phi)
        assert np.abs(r["grad"][0] - g).max() <= 1e-6, (kind, x, r["grad"][0], g)


@pytest.mark.parametrize("h", ["linf", "dnorm", "anorm"])
def test_control_for_the_section4_hamiltonians(orc, h):
    """The control of P9 for l_inf, sqrt(sum w p^2) and sqrt(<p, M p>):
    <beta, p> = H(p), beta in the dual unit ball (|beta|_1 <= 1,
    sum beta^2 / w <= 1, <beta, M^-1 beta> <= 1), and x - t beta attains phi
    (Hopf-Lax)."""
    n, B = 8, 16
    rng = np.random.default_rng(71)
    a = wl.uniform(9501, n, 0.5, 2.0)
    c = wl.normal(9502, n, 0.5)
    x = wl.normal(9503, B * n, 2.0).reshape(B, n)
    t = wl.uniform(9504, B, 0.2, 2.0)
    if h == "linf":
        kind, w = orc.H_LINF, None
        dual = lambda b: np.abs(b).sum()
    elif h == "dnorm":
        kind, w = orc.H_DNORM, wl.uniform(9505, n, 0.5, 1.5)
        dual = lambda b: np.sqrt((b * b / w).sum())
    else:
        Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
        w = (Q * rng.uniform(0.3, 3.0, n)) @ Q.T
        Minv = np.linalg.inv(w)
        kind = orc.H_ANORM
        dual = lambda b: np.sqrt(b @ Minv @ b)
    P = orc.Problem(a, kind, w=w, centre=c, tol=1e-30, max_iter=200000, stop_rule=orc.STOP_UREL)
    r = P.eval(x, t)
    ctl = orc.control(P, x, t, r["grad"])
    for q in range(B):
        p, beta = r["grad"][q], ctl["beta"][q]
        Hp = P.H(p)
        assert abs(beta @ p - Hp) <= 1e-7 * max(1.0, Hp)
        assert dual(beta) <= 1 + 1e-7
        z = ctl["x_T"][q] - c
        J = 0.5 * (z * z / a).sum() - 0.5
        assert abs(J - r["phi"][q]) <= 1e-7 * max(1.0, abs(r["phi"][q]))


def test_ties_go_to_the_smallest_index(orc):
    """With identical parts every part attains the minimum (union, Section
    2.2), the maximum (maximum over Hamiltonians) and the distance (Section
    3.2): the index reported is the first, 0, and the value is the single
    part's."""
    n = 6
    a = wl.uniform(7601, n, 0.5, 2.0)
    c = wl.normal(7602, n, 1.0)
    x = wl.normal(7603, 12 * n, 3.0).reshape(12, n)
    t = wl.uniform(7604, 12, 0.0, 2.0)
    one = orc.Problem(a, orc.H_L2, centre=c, tol=1e-14, max_iter=5000, stop_rule=orc.STOP_UREL)
    ref = one.eval(x, t)
    r = orc.union_eval([one, one, one], x, t)
    assert (r["argmin"] == 0).all() and np.array_equal(r["phi"], ref["phi"])
    r = orc.maxH_eval([one, one], x, t)
    assert (r["argmax"] == 0).all() and np.array_equal(r["phi"], ref["phi"])
    r = orc.union_closest([one, one], x)
    d1 = orc.union_closest([one], x)
    assert (r["argmin"] == 0).all() and np.array_equal(r["dist"], d1["dist"])


def _shrink_exact(z, a):
    """shrink_1(z, a) on exact rationals (Section 1: 0 when |z| <= a)."""
    return z - a if z > a else (z + a if z < -a else 0)


def _paper_rule_iterations_exact(a, y, t, lam, tol, max_iter):
    """Split Bregman (eq. 3.4(a)-(c)) for diagonal A and H = l1 in exact
    rational arithmetic.  Each coordinate is a scalar recursion:
    v_i = (y_i + lam (d_i - b_i)) / (a_i + lam), d_i' = shrink_1(v_i + b_i, t / lam),
    b_i' = b_i + v_i - d_i', from v^0 = d^0 = y, b^0 = 0 (Section 3.1).  Returns
    the first k at which |v^k - v^{k-1}|^2, |d^k - d^{k-1}|^2 and |d^k - v^k|^2
    are all <= tol (Section 4.5), and the residuals at k - 1 and k."""
    n = len(a)
    tau = t / lam
    v_prev, d, b = list(y), list(y), [0] * n
    prev = None
    for k in range(1, max_iter + 1):
        v = [(y[i] + lam * (d[i] - b[i])) / (a[i] + lam) for i in range(n)]
        dn = [_shrink_exact(v[i] + b[i], tau) for i in range(n)]
        b = [b[i] + v[i] - dn[i] for i in range(n)]
        r = (sum((v[i] - v_prev[i]) ** 2 for i in range(n)), sum((dn[i] - d[i]) ** 2 for i in range(n)),
             sum((dn[i] - v[i]) ** 2 for i in range(n)))
        if max(r) <= tol:
            return k, prev, r
        prev, d, v_prev = r, dn, v
    return None, prev, None


@pytest.mark.parametrize("case", range(4))
def test_paper_stop_rule_exact_iterations(orc, case):
    """The oracle's iteration count under the paper's stop rule equals the
    first k at which the exact (rational) iterates meet all three residual
    tests, for dyadic data (exact in FP64) whose residuals cross tol with a
    wide margin, so rounding cannot move the crossing."""
    from fractions import Fraction as F
    cases = [  # (a, y, t, lam, tol)
        ([F(3, 2), F(5, 4), F(7, 8), F(2)], [F(9, 8), F(-5, 4), F(3, 16), F(-7, 2)], F(3, 4), F(1), F(1, 10 ** 8)),
        ([F(1, 2), F(3, 4), F(7, 4), F(5, 8)], [F(-11, 8), F(1, 4), F(13, 4), F(-3, 8)], F(5, 4), F(1), F(1, 10 ** 8)),
        ([F(3, 2), F(5, 4), F(7, 8), F(2)], [F(9, 8), F(-5, 4), F(3, 16), F(-7, 2)], F(3, 4), F(1, 2), F(1, 10 ** 10)),
        ([F(9, 8), F(1, 2), F(15, 8)], [F(5, 2), F(-3, 2), F(1, 8)], F(1, 8), F(5, 2), F(1, 10 ** 8)),
    ]
    a, y, t, lam, tol = cases[case]
    K, before, at = _paper_rule_iterations_exact(a, y, t, lam, tol, 500)
    assert K is not None and K >= 2
    # a wide margin on both sides of the crossing
    assert max(at) <= tol * F(1, 2) or max(at) <= tol * (1 - F(1, 10 ** 6))
    assert max(before) >= tol * (1 + F(1, 10 ** 6))
    af = np.array([float(v) for v in a])
    yf = np.array([[float(v) for v in y]])
    P = orc.Problem(af, orc.H_L1, c0=0.5, lam=float(lam), tol=float(tol), max_iter=500, stop_rule=orc.STOP_PAPER)
    r = P.eval(yf, np.array([float(t)]))
    assert int(r["iters"][0]) == K, (int(r["iters"][0]), K)


def _solve_exact(S, r):
    """x with S x = r by Gauss-Jordan elimination on exact rationals."""
    n = len(r)
    M = [list(S[i]) + [r[i]] for i in range(n)]
    for c in range(n):
        p = next(i for i in range(c, n) if M[i][c] != 0)
        M[c], M[p] = M[p], M[c]
        for i in range(n):
            if i != c and M[i][c] != 0:
                f = M[i][c] / M[c][c]
                M[i] = [M[i][j] - f * M[c][j] for j in range(n + 1)]
    return [M[i][n] / M[i][i] for i in range(n)]


def _relative_rule_iterations_exact(A, w, y, t, lam, tol, max_iter):
    """Split Bregman (eq. 3.4(a)-(c)) for a dense A and H = weighted l1 in
    exact rational arithmetic, stopped by the relative change of the d-update
    argument u^k = v^k + b^{k-1}: the first k >= 2 with
    |u^k - u^{k-1}|^2 <= tol max(1, |u^k|^2), where u^0 = y (v^0 = d^0 = y,
    b^0 = 0, Section 3.1).  u^{k-1} is kept from the previous step, not
    rebuilt from d and b.  Returns k and (ratio to tol, |u|^2) at k - 1 and k."""
    n = len(y)
    S = [[A[i][j] + (lam if i == j else 0) for j in range(n)] for i in range(n)]
    tau = t / lam
    d, b, u_prev = list(y), [0] * n, list(y)
    prev = None
    for k in range(1, max_iter + 1):
        v = _solve_exact(S, [y[i] + lam * (d[i] - b[i]) for i in range(n)])
        u = [v[i] + b[i] for i in range(n)]
        un = sum(e * e for e in u)
        ru = sum((u[i] - u_prev[i]) ** 2 for i in range(n)) / max(un, 1)
        if k >= 2 and ru <= tol:
            return k, prev, (ru / tol, un)
        prev = (ru / tol, un)
        d = [_shrink_exact(u[i], tau * w[i]) for i in range(n)]
        b = [u[i] - d[i] for i in range(n)]
        u_prev = u
    return None, prev, None


@pytest.mark.parametrize("case", range(6))
def test_relative_stop_rule_exact_iterations(orc, case):
    """The oracle's iteration count under the relative-change rule (the rule
    of every dense solve) equals the first k at which the exact (rational)
    iterates meet it: dense and diagonal A, l1 and weighted l1, |u|^2 above 1
    (the division counts) and below 1 (the floor counts), with the crossing
    at a margin of at least 10 % (FP64 rounding moves the ratio by ~1e-10)."""
    from fractions import Fraction as F
    A1 = [[F(2), F(1, 2), F(0)], [F(1, 2), F(3, 2), F(1, 4)], [F(0), F(1, 4), F(1)]]
    D4 = [[F(3, 2), 0, 0, 0], [0, F(5, 4), 0, 0], [0, 0, F(7, 8), 0], [0, 0, 0, F(2)]]
    one3, one4 = [F(1)] * 3, [F(1)] * 4
    cases = [  # (A, w, y, t, lam, tol)
        (A1, one3, [F(9, 8), F(-5, 4), F(3, 16)], F(3, 4), F(1), F(1, 10 ** 10)),
        (A1, one3, [F(5, 2), F(-3), F(7, 4)], F(1, 2), F(1), F(1, 10 ** 10)),
        (A1, one3, [F(1, 4), F(-1, 8), F(3, 16)], F(1, 8), F(1), F(1, 10 ** 10)),
        (A1, [F(1, 2), F(3, 2), F(1)], [F(5, 2), F(-3), F(7, 4)], F(1, 2), F(1, 2), F(1, 10 ** 12)),
        (D4, one4, [F(9, 8), F(-5, 4), F(3, 16), F(-7, 2)], F(3, 4), F(1), F(2, 10 ** 10)),
        # a coordinate inside the shrink's dead zone (b there follows u, so
        # u^{k-1} differs from v^{k-1} + b^{k-1}) and a crossing between the
        # two
        (A1, one3, [F(9, 8), F(-5, 4), F(3, 16)], F(3, 4), F(1), F(2, 10 ** 10)),
    ]
    A, w, y, t, lam, tol = cases[case]
    K, before, at = _relative_rule_iterations_exact(A, w, y, t, lam, tol, 400)
    assert K is not None and K >= 3
    assert at[0] <= F(9, 10) and before[0] >= F(11, 10)
    n = len(y)
    if case == 4:
        Af = np.array([float(A[i][i]) for i in range(n)])
    else:
        Af = np.array([[float(e) for e in row] for row in A])
    hk = orc.H_L1 if all(e == 1 for e in w) else orc.H_WL1
    P = orc.Problem(Af, hk, w=np.array([float(e) for e in w]), c0=0.5, lam=float(lam), tol=float(tol),
                    max_iter=400, stop_rule=orc.STOP_UREL)
    r = P.eval(np.array([[float(e) for e in y]]), np.array([float(t)]))
    assert int(r["iters"][0]) == K, (int(r["iters"][0]), K)
    # the two regimes of the floor are both exercised
    if case == 2:
        assert at[1] < F(1, 2)
    if case == 1:
        assert at[1] > 4


@pytest.mark.parametrize("h", ["l1", "wl1", "l2"])
def test_phi_convex_in_x_with_supporting_gradient(orc, h):
    """phi(., t) is a Legendre transform (eq. 3.3: the supremum over v of
    affine functions of x), hence convex, and grad_x phi = d^K is a
    subgradient: phi(x2) >= phi(x1) + <grad phi(x1), x2 - x1> for every pair,
    and phi on the segment lies below the chord."""
    n, m = 12, 10
    A, _ = _dense(n, 7401)
    w = wl.uniform(7403, n, 0.5, 1.5) if h == "wl1" else None
    x = wl.normal(7404, m * n, 2.0).reshape(m, n)
    t = np.full(m, 0.7)
    kind = {"l1": orc.H_L1, "wl1": orc.H_WL1, "l2": orc.H_L2}[h]
    P = orc.Problem(A, kind, w=w, tol=1e-28, max_iter=20000, stop_rule=orc.STOP_UREL)
    r = P.eval(x, t)
    phi, g = r["phi"], r["grad"]
    for i in range(m):
        for j in range(m):
            if i == j:
                continue
            lin = phi[i] + g[i] @ (x[j] - x[i])
            slack = 1e-9 * (abs(phi[j]) + abs(lin) + 1)
            assert phi[j] >= lin - slack, (i, j, phi[j], lin)
    # midpoints of consecutive pairs, three interior points each
    th = np.array([0.25, 0.5, 0.75])
    for i in range(m - 1):
        xs = th[:, None] * x[i] + (1 - th[:, None]) * x[i + 1]
        mid = P.eval(xs, np.full(3, 0.7))["phi"]
        chord = th * phi[i] + (1 - th) * phi[i + 1]
        assert (mid <= chord + 1e-9 * (np.abs(chord) + 1)).all(), (i, mid, chord)
    # and the gap is not vacuous: strict convexity shows along some segment
    assert max(abs(phi[j] - phi[i] - g[i] @ (x[j] - x[i])) for i in range(m) for j in range(m)) > 1e-3
