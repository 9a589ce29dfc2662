"""Independent routes to the Hopf solution, used to pin the oracle.

Nothing here calls the oracle's iteration: each function follows a different
passage of the paper or a different algorithm, so that an error in the oracle
(a dropped term, a sign, a wrong iterate) disagrees with at least one of them.
"""
import numpy as np


def shrink1(z, a):
    """Soft threshold (Section 1, definition of shrink_1): 0 when |z| <= a."""
    return np.sign(z) * np.maximum(np.abs(z) - a, 0.0)


def shrink2(z, a):
    """Block soft threshold (Section 1, definition of shrink_2)."""
    nz = np.linalg.norm(z)
    return np.zeros_like(z) if nz == 0 else z / nz * max(nz - a, 0.0)


def closed_diag_wl1(y, t, a, w=None):
    """Diagonal A = diag(a), c0 = 1/2, H = sum w_i |p_i|: the minimisation in
    eq. 3.3 decouples per coordinate (the worked example of Section 1, there
    with a_i^2 in place of a_i and w = 1), giving v_i = shrink_1(y_i, t w_i)/a_i
    and phi = sum shrink_1(y_i, t w_i)^2 / (2 a_i) - 1/2."""
    w = np.ones_like(a) if w is None else w
    s = shrink1(y, t * w)
    return (s * s / (2 * a)).sum() - 0.5, s / a


def paper_example_l1(x, t, a):
    """Section 1 worked example verbatim: J = 1/2 (sum x_i^2/a_i^2 - 1),
    H = l1: phi = -1/2 + sum_{|x_i| > t} 1/2 ((|x_i| - t)/a_i)^2 and
    d phi / d x_i = shrink_1(x, t)_i / a_i^2."""
    m = np.abs(x) > t
    phi = -0.5 + 0.5 * (((np.abs(x[m]) - t) / a[m]) ** 2).sum()
    return phi, shrink1(x, t) / a ** 2


def paper_example_sphere(x, t):
    """Section 1: unit sphere moved outward with H = l2:
    phi = 1/2 (|x| - t)^2 - 1/2 if |x| > t, else -1/2."""
    r = np.linalg.norm(x)
    return (0.5 * (r - t) ** 2 - 0.5) if r > t else -0.5


def diag_l2_secular(y, t, a, c0=0.5):
    """Diagonal A, H = l2.  If |y| <= t the minimiser is 0 and phi = -c0;
    otherwise v_j = y_j/(a_j + mu) with mu > 0 solving
    sum_j (mu y_j/(a_j + mu))^2 = t^2 (KKT of eq. 3.3: A v - y + t v/|v| = 0
    with mu = t/|v|).  The left side increases in mu; bisection to the last bit."""
    if np.linalg.norm(y) <= t:
        v = np.zeros_like(y)
        return -c0, v
    f = lambda mu: np.sum((mu * y / (a + mu)) ** 2) - t * t
    lo, hi = 0.0, 1.0
    while f(hi) < 0:
        hi *= 2
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) < 0:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-17 * hi:
            break
    mu = 0.5 * (lo + hi)
    v = y / (a + mu)
    phi = y @ v - 0.5 * (a * v * v).sum() - c0 - t * np.linalg.norm(v)
    return phi, v


def kkt_active_set(A, y, t, w, v_guess, zero_tol=0.0):
    """Exact minimiser of 1/2 v^T A v - <y,v> + t sum w_i |v_i| from a guessed
    support S and signs sigma (those of v_guess): solve
    A_SS v_S = y_S - t (w sigma)_S, v = 0 off S, then accept only if the signs
    agree and |(y - A v)_i| <= t w_i off S (optimality conditions of eq. 3.3).
    Returns (v, ok)."""
    S = np.abs(v_guess) > zero_tol
    sig = np.sign(v_guess[S])
    v = np.zeros_like(y)
    if S.any():
        L = np.linalg.cholesky(A[np.ix_(S, S)])
        rhs = y[S] - t * (w[S] * sig)
        v[S] = np.linalg.solve(L.T, np.linalg.solve(L, rhs))
    r = y - A @ v
    ok = np.all(np.sign(v[S]) == sig) and np.all(np.abs(r[~S]) <= t * w[~S] * (1 + 1e-12) + 1e-13)
    return v, ok


def objective_neg(A, y, t, w, v, c0=0.5, h="wl1"):
    """-(J*(v) + t H(v) - <x,v>) with J*(v) = 1/2 v^T A v + <c,v> + c0."""
    Av = A @ v if A.ndim == 2 else A * v
    H = np.linalg.norm(v) if h == "l2" else (w * np.abs(v)).sum()
    return y @ v - 0.5 * v @ Av - c0 - t * H


def J_value(Ainv, z, c0=0.5):
    return 0.5 * z @ (Ainv @ z) - c0


def hopf_lax_upper(Ainv, A, y, t, w, v, c0=0.5, h="wl1"):
    """Hopf-Lax (Section 2.2): phi = min_{c in C} J(x - t c) where C is the
    unit ball of H's dual norm (box [-w_i, w_i] for weighted l1, the Euclidean
    unit ball for l2).  Any feasible c gives an upper bound; c = P_C((y-Av)/t)
    is the one suggested by the optimality conditions."""
    g = (y - A @ v) / t
    if h == "l2":
        ng = np.linalg.norm(g)
        c = g if ng <= 1 else g / ng
    else:
        c = np.clip(g, -w, w)
    return J_value(Ainv, y - t * c, c0)


def hopf_lax_bruteforce_2d(Ainv, y, t, w, c0=0.5, h="wl1"):
    """n = 2 brute force of min_{c in C} J(y - t c) (the value)."""
    return hopf_lax_argmin_2d(Ainv, y, t, w, c0, h)[0]


def hopf_lax_argmin_2d(Ainv, y, t, w, c0=0.5, h="wl1"):
    """n = 2 brute force of min_{c in C} J(y - t c): returns (value, c at the
    minimum).  For the box the convex quadratic's minimum is enumerated over
    the interior, the four edges (clamped 1-D minimum) and the four corners;
    for the disk, over the interior minimum and a 200,001-point sweep of the
    circle refined by golden section."""
    q = lambda c: J_value(Ainv, y - t * c, c0)
    P = t * t * Ainv
    cands = []
    c_int = np.linalg.solve(P, t * (Ainv @ y))  # unconstrained minimiser: gradient zero
    if h == "l2":
        if np.linalg.norm(c_int) <= 1:
            cands.append(c_int)
        th = np.linspace(0, 2 * np.pi, 200001)
        C = np.stack([np.cos(th), np.sin(th)], 1)
        Z = y[None, :] - t * C
        vals = 0.5 * np.einsum("ij,jk,ik->i", Z, Ainv, Z) - c0
        k = int(np.argmin(vals))
        a, b = th[max(k - 1, 0)], th[min(k + 1, len(th) - 1)]
        gr = (np.sqrt(5) - 1) / 2
        f = lambda a_: q(np.array([np.cos(a_), np.sin(a_)]))
        for _ in range(200):
            c1, c2 = b - gr * (b - a), a + gr * (b - a)
            if f(c1) < f(c2):
                b = c2
            else:
                a = c1
        m = 0.5 * (a + b)
        cands.append(np.array([np.cos(m), np.sin(m)]))
    else:
        if np.all(np.abs(c_int) <= w):
            cands.append(c_int)
        for i in range(2):
            j = 1 - i
            for s in (-1, 1):
                c = np.zeros(2)
                c[i] = s * w[i]
                # minimise over c[j] with c[i] fixed: P_jj c_j + P_ji c_i = t (Ainv y)_j
                cj = (t * (Ainv @ y)[j] - P[j, i] * c[i]) / P[j, j]
                c[j] = np.clip(cj, -w[j], w[j])
                cands.append(c.copy())
        for s0 in (-1, 1):
            for s1 in (-1, 1):
                cands.append(np.array([s0 * w[0], s1 * w[1]]))
    vals = [q(c) for c in cands]
    k = int(np.argmin(vals))
    return vals[k], cands[k]


def ellipsoid_projection(yv, semi, tol=1e-15, max_iter=200):
    """Section 4.3: projection of w onto {sum (x_i/d_i)^2 <= 1}: x_i =
    d_i^2 w_i/(d_i^2 + mu) with mu the root of sum d_i^2 w_i^2/(d_i^2 + mu)^2
    = 1, found by Newton's method on the minimisation of
    mu -> sum d_i^2 w_i^2/(d_i^2 + mu) + mu from mu_0 = 0."""
    d2 = semi ** 2
    if np.sum((yv / semi) ** 2) <= 1:
        return yv.copy(), 0.0
    mu = 0.0
    for _ in range(max_iter):
        den = d2 + mu
        f1 = 1.0 - np.sum(d2 * yv * yv / den ** 2)
        f2 = 2.0 * np.sum(d2 * yv * yv / den ** 3)
        step = f1 / f2
        mu -= step
        if abs(step) <= tol * max(1.0, mu):
            break
    return d2 * yv / (d2 + mu), mu


def l1ball_projection(z, r, iters=200):
    """Projection on {y : |y|_1 <= r} by bisection on the threshold mu of
    shrink_1(z, mu) (no sorting): |shrink_1(z, mu)|_1 decreases in mu."""
    z = np.asarray(z, dtype=np.float64)
    if np.abs(z).sum() <= r:
        return z.copy()
    lo, hi = 0.0, np.abs(z).max()
    for _ in range(iters):
        mu = 0.5 * (lo + hi)
        if np.maximum(np.abs(z) - mu, 0).sum() > r:
            lo = mu
        else:
            hi = mu
    mu = 0.5 * (lo + hi)
    return np.sign(z) * np.maximum(np.abs(z) - mu, 0)


def min_convex(f, x0, scale):
    """Minimum of a convex function of a few variables: Nelder-Mead from
    several starts, refined."""
    from scipy.optimize import minimize
    best = None
    rng = np.random.default_rng(5)
    starts = [np.asarray(x0, dtype=np.float64)] + [np.asarray(x0) + scale * rng.normal(size=len(x0)) for _ in range(2)]
    for s in starts:
        r = minimize(f, s, method="Nelder-Mead", options={"xatol": 1e-12, "fatol": 1e-15, "maxiter": 40000,
                                                           "maxfev": 80000})
        r = minimize(f, r.x, method="Nelder-Mead", options={"xatol": 1e-13, "fatol": 1e-16, "maxiter": 40000,
                                                             "maxfev": 80000})
        if best is None or r.fun < best.fun:
            best = r
    return best.fun, best.x
