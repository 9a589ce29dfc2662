"""FP64 CPU oracle for the Hopf-formula evaluation (test infrastructure only).

This package wraps ``hopf_oracle.c``: a plain, unblocked FP64 implementation of
the split Bregman evaluation of the Hopf formula (Section 3.1, eqs. 3.3 and
3.4(a)-(c)), the min-over-initial-data rule for unions (Section 2.2), the
level-set distance / closest point by Newton on s (Section 3.2) and the
envelope-theorem gradients.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it;
the CUDA library shares no code with it.

Pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_pins.py``:
closed forms of Section 1 (l1 with a diagonal ellipsoid, l2 with a sphere),
their weighted / diagonal generalisations, phi(x,0) = J(x), an exact
active-set (KKT) solve, duality-gap bounds, brute-force Hopf-Lax minimisation
at n = 2, finite differences in x and t, the ellipsoid projection of
Section 4.3, the control's membership in dH and the Hopf-Lax value
J(x_T) = phi, and brute-force minimisation at n = 2 of the Hopf formula with
the Hamiltonian min_i H_i, the new proxes against numerical minimisation of
their definitions, closed forms through Hopf-Lax projections for J = 1/2|x|^2
with H = l_inf and sqrt(sum w p^2), and brute-force Hopf objectives at n = 2
for the non-quadratic initial data (with lambda != 1), and the iteration
counts of both stop rules against exact rational iterates (l1 and weighted
l1, diagonal and dense A).  Parity unpinned: iteration counts with the
Hamiltonians whose proxes take square roots or roots of piecewise functions
(l2, l_inf, the D- and A-norms), which no exact rational run reproduces; the
paper prints no counts.
``tests/test_oracle_mutants.py`` plants plausible mistakes one at a time in a
scratch copy of the C source and checks that the pins named for each fail.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "hopf_oracle.c")

A_DIAG, A_DENSE = 0, 1
J_L1SQ, J_LINFSQ = 2, 3   # J = 1/2 |x - c|_1^2 - c0, 1/2 |x - c|_inf^2 - c0 (Section 4.4)
H_L1, H_WL1, H_L2 = 0, 1, 2
H_LINF, H_DNORM = 3, 4    # |p|_inf (Section 4.2), sqrt(sum w_i p_i^2) (Section 4.3)
H_ANORM = 5               # sqrt(<p, M p>), M symmetric positive definite (Section 4.3)


def anorm_weights(M):
    """The weight block of H = sqrt(<p, M p>): M, then its eigenvectors and
    eigenvalues (M = P diag(l) P^T, numpy's symmetric eigensolver as the
    library step), the layout the C oracle reads."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    l, P = np.linalg.eigh(0.5 * (M + M.T))
    if not (l > 0).all():
        raise ValueError("oracle: M is not positive definite")
    return np.concatenate([M.ravel(), np.ascontiguousarray(P).ravel(), l])
STOP_PAPER, STOP_UREL = 0, 1


def build(force=False):
    """Compile the oracle with gcc (plain C, -O2, OpenMP over queries)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _SO, _SRC, "-lm"])
    return _SO


class _Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("a_kind", ctypes.c_int32),
                ("A", ctypes.c_void_p), ("c", ctypes.c_void_p), ("c0", ctypes.c_double),
                ("h_kind", ctypes.c_int32), ("w", ctypes.c_void_p),
                ("lam", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("stop_rule", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("phi", ctypes.c_double), ("phi_v", ctypes.c_double), ("dphidt", ctypes.c_double),
                ("iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("res_paper", ctypes.c_double), ("res_u", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.orc_eval_batch.restype = ctypes.c_int
        _lib.orc_union_eval.restype = ctypes.c_int
        _lib.orc_union_closest.restype = ctypes.c_int
        _lib.orc_maxH_eval.restype = ctypes.c_int
        _lib.orc_control.restype = None
        _lib.orc_backward_params.restype = None
        _lib.orc_prox.restype = None
        _lib.orc_factor.restype = ctypes.c_int
        _lib.orc_num_threads.restype = ctypes.c_int
        _lib.orc_H.restype = ctypes.c_double
        _lib.orc_l1sq_beta.restype = ctypes.c_double
        _lib.orc_neg_objective.restype = ctypes.c_double
    return _lib


def num_threads():
    return lib().orc_num_threads()


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Problem:
    """One instance: J(x) = 1/2 (x-c)^T A^{-1} (x-c) - c0 with A diagonal
    (vector ``a``) or dense (matrix ``A``), or a norm J (``j_kind``); H one of
    l1, weighted l1, l2, l_inf, sqrt(sum w p^2) and sqrt(<p, M p>) (``w`` = M,
    n x n)."""

    def __init__(self, A, h_kind, w=None, centre=None, c0=0.5, lam=1.0, tol=1e-10,
                 max_iter=500, stop_rule=STOP_PAPER, j_kind=None, n=None):
        """A: the diagonal (1-D) or dense (2-D) matrix of a quadratic J, or None
        with j_kind = J_L1SQ / J_LINFSQ and the dimension n."""
        if A is None:
            assert j_kind in (J_L1SQ, J_LINFSQ) and n is not None
            self.a_kind, self.n = j_kind, int(n)
        else:
            A = np.ascontiguousarray(A, dtype=np.float64)
            self.a_kind = A_DIAG if A.ndim == 1 else A_DENSE
            self.n = A.shape[0]
        self.A = A
        self.w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        if self.w is not None and int(h_kind) == H_ANORM:
            self.w = anorm_weights(self.w.reshape(self.n, self.n))
        self.c = None if centre is None else np.ascontiguousarray(centre, dtype=np.float64)
        self.c0, self.h_kind, self.lam, self.tol = float(c0), int(h_kind), float(lam), float(tol)
        self.max_iter, self.stop_rule = int(max_iter), int(stop_rule)

    def _struct(self):
        return _Problem(self.n, self.a_kind, _p(self.A), _p(self.c), self.c0, self.h_kind, _p(self.w),
                        self.lam, self.tol, self.max_iter, self.stop_rule)

    def eval(self, x, t):
        """Returns dict with phi, phi_v, grad, dphidt, iters, converged, res_paper, res_u."""
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, self.n)
        t = np.ascontiguousarray(t, dtype=np.float64).reshape(-1)
        B = x.shape[0]
        grad = np.empty_like(x)
        res = (_Result * max(B, 1))()
        st = self._struct()
        rc = lib().orc_eval_batch(ctypes.byref(st), ctypes.c_int64(B), _p(x), _p(t), _p(grad), res)
        if rc != 0:
            raise ValueError("oracle: A + lambda I is not symmetric positive definite" if rc == -1 else "oracle failure")
        out = {k: np.array([getattr(res[i], k) for i in range(B)]) for k in
               ("phi", "phi_v", "dphidt", "iters", "converged", "res_paper", "res_u")}
        out["grad"] = grad
        return out

    def H(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        return lib().orc_H(self.h_kind, self.n, _p(self.w), _p(q))


def union_eval(parts, x, t):
    """phi = min_i phi_i over parts (Section 2.2), argmin (ties -> smallest),
    gradient of the minimising part, and the summed iteration count."""
    n = parts[0].n
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, n)
    t = np.ascontiguousarray(t, dtype=np.float64).reshape(-1)
    B = x.shape[0]
    arr = (_Problem * len(parts))(*[p._struct() for p in parts])
    phi = np.empty(B); grad = np.empty_like(x)
    am = np.empty(B, np.int32); it = np.empty(B, np.int32)
    rc = lib().orc_union_eval(arr, len(parts), ctypes.c_int64(B), _p(x), _p(t), _p(phi), _p(grad), _p(am), _p(it))
    if rc != 0:
        raise ValueError("oracle: a part is not SPD")
    return {"phi": phi, "grad": grad, "argmin": am, "iters": it}


def union_closest(parts, x, s_tol=1e-12, max_newton=50):
    """Distance to the union of {J_i <= 0} and the closest point, by Newton on
    s over the eikonal solution (Section 3.2), min over parts (Section 2.2)."""
    n = parts[0].n
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, n)
    B = x.shape[0]
    arr = (_Problem * len(parts))(*[p._struct() for p in parts])
    dist = np.empty(B); closest = np.empty_like(x); am = np.empty(B, np.int32)
    fails = ctypes.c_int32(0)
    rc = lib().orc_union_closest(arr, len(parts), ctypes.c_int64(B), _p(x), ctypes.c_double(s_tol),
                                 ctypes.c_int32(max_newton), _p(dist), _p(closest), _p(am), ctypes.byref(fails))
    if rc != 0:
        raise ValueError("oracle: a part is not SPD")
    return {"dist": dist, "closest": closest, "argmin": am, "newton_fail": fails.value}


def backward(n, a_kind, h_kind, w, g_phi, vstar, t, want_A=True):
    """Envelope-theorem gradients: g_x = g v*, g_t = -g H(v*),
    g_A = -1/2 sum_q g_q v*_q v*_q^T (or its diagonal)."""
    vstar = np.ascontiguousarray(vstar, dtype=np.float64).reshape(-1, n)
    B = vstar.shape[0]
    g_phi = np.ascontiguousarray(g_phi, dtype=np.float64).reshape(-1)
    t = np.ascontiguousarray(t, dtype=np.float64).reshape(-1)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    g_x = np.empty_like(vstar); g_t = np.empty(B)
    g_A = None
    if want_A:
        g_A = np.empty((n, n) if a_kind == A_DENSE else (n,))
    lib().orc_backward(n, a_kind, h_kind, _p(w), ctypes.c_int64(B), _p(g_phi), _p(vstar), _p(t),
                       _p(g_x), _p(g_t), _p(g_A))
    return {"g_x": g_x, "g_t": g_t, "g_A": g_A}


def backward_params(n, h_kind, w, g_phi, vstar, t):
    """Gradients of sum_q g_q phi_q with respect to the centre c, the constant
    c0 and the weights w (weighted l1, sqrt(sum w p^2)), by the envelope
    theorem at the minimisers vstar."""
    vstar = np.ascontiguousarray(vstar, dtype=np.float64).reshape(-1, n)
    B = vstar.shape[0]
    g_phi = np.ascontiguousarray(g_phi, dtype=np.float64).reshape(-1)
    t = np.ascontiguousarray(t, dtype=np.float64).reshape(-1)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    g_c = np.empty(n)
    g_c0 = ctypes.c_double(0.0)
    g_w = np.empty(n) if int(h_kind) in (H_WL1, H_DNORM) else None
    lib().orc_backward_params(n, int(h_kind), _p(w), ctypes.c_int64(B), _p(g_phi), _p(vstar), _p(t), _p(g_c),
                              ctypes.byref(g_c0), _p(g_w))
    return {"g_c": g_c, "g_c0": g_c0.value, "g_w": g_w}


def control(problem, x, t, grad):
    """Optimal control beta = (x - c - A p) / t in dH(p) for the minimiser p
    (= grad phi), and the terminal point x_T = x - t beta (Section 2: the
    control beta = grad H(grad phi); the Hopf-Lax minimiser).  beta = 0 and
    x_T = x at t = 0."""
    n = problem.n
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, n)
    t = np.ascontiguousarray(t, dtype=np.float64).reshape(-1)
    grad = np.ascontiguousarray(grad, dtype=np.float64).reshape(-1, n)
    B = x.shape[0]
    beta = np.empty_like(x)
    x_T = np.empty_like(x)
    st = problem._struct()
    lib().orc_control(ctypes.byref(st), ctypes.c_int64(B), _p(x), _p(t), _p(grad), _p(beta), _p(x_T))
    return {"beta": beta, "x_T": x_T}


def maxH_eval(parts, x, t):
    """phi = max_i phi_i over parts that share J and differ in H (Section 2.2:
    the solution for the Hamiltonian min_i H_i), argmax (ties -> smallest),
    gradient of the maximising part, and the summed iteration count."""
    n = parts[0].n
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, n)
    t = np.ascontiguousarray(t, dtype=np.float64).reshape(-1)
    B = x.shape[0]
    arr = (_Problem * len(parts))(*[p._struct() for p in parts])
    phi = np.empty(B); grad = np.empty_like(x)
    am = np.empty(B, np.int32); it = np.empty(B, np.int32)
    rc = lib().orc_maxH_eval(arr, len(parts), ctypes.c_int64(B), _p(x), _p(t), _p(phi), _p(grad), _p(am), _p(it))
    if rc != 0:
        raise ValueError("oracle: A + lambda I is not SPD")
    return {"phi": phi, "grad": grad, "argmax": am, "iters": it}


def l1sq_beta(z, alpha):
    """beta = alpha |shrink_1(z, beta)|_1 (Section 4.4) as the oracle finds it."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    return lib().orc_l1sq_beta(len(z), _p(z), ctypes.c_double(alpha))


def prox(h_kind, tau, z, w=None):
    """prox of tau H at z (the d-update, eq. 3.4(b)) as the oracle computes it
    (w: the weights, or M for H_ANORM)."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    if w is not None and int(h_kind) == H_ANORM:
        w = anorm_weights(w.reshape(len(z), len(z)))
    out = np.empty_like(z)
    lib().orc_prox(int(h_kind), len(z), _p(w), ctypes.c_double(tau), _p(z), _p(out))
    return out
