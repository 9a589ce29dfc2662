"""The dense forms' gradient bars, derived from a model of their arithmetic.

``accuracy_model`` runs the SPLIT and MIXED iterations with FP16 / BF16
operands, exact 16-term MMA products and FP32 accumulators that round to
nearest or truncate, on queries of the dense headline workload (n = 1024,
weighted l1, tol 1e-13), and compares d^K with the FP64 oracle.  What it
shows, and what the GPU tests' bars rest on:

- MIXED meets its bars (6e-6 max, 3e-6 median) but not 1e-6: at tol 1e-13
  the remaining step of the stop rule, not the accumulation, sets its error
  (rounding to nearest gives the same error);
- SPLIT's error in v = M r reaches the fixed point through A + lam I, and a
  truncating accumulator makes it several times larger than rounding to
  nearest would: the measured SPLIT error (1.1e-5) is the truncating
  model's, within SPLIT's bars (2.5e-5 max, 1.2e-5 median);
- with a tighter stop (1e-15) the truncating MIXED model keeps a floor near
  2e-6 over the 64 K steps of n = 1024.

No GPU is involved."""
import numpy as np
import pytest

import workloads as wl
from tests import accuracy_model as am

N, Q = 1024, 8


@pytest.fixture(scope="module")
def problem(orc):
    A, _, _ = wl.spd_matrix(2001, 2002, N)
    w = wl.uniform(2003, N, 0.5, 1.5)
    x = wl.normal(2004, Q * N, 2.0).reshape(Q, N)
    t = wl.uniform(2005, Q, 0.1, 3.0)
    ref = orc.Problem(A, orc.H_WL1, w=w, c0=0.5, lam=1.0, tol=1e-28, max_iter=50000,
                      stop_rule=orc.STOP_UREL).eval(x, t)
    y = np.ascontiguousarray(x.T, dtype=np.float32)
    thr = (t[None, :] * w[:, None]).astype(np.float32)
    return A, y, thr, ref["grad"]


_RUNS = {}


def _solve(problem, form, tol, mode):
    """am.solve on the module's queries, each (form, tol, mode) run once."""
    key = (form, tol, mode)
    if key not in _RUNS:
        A, y, thr, _ = problem
        _RUNS[key] = am.solve(form, A, 1.0, y, thr, tol, mode)
    return _RUNS[key]


def _err(problem, form, tol, mode):
    ref = problem[3]
    p, iters = _solve(problem, form, tol, mode)
    assert (iters < 3000).all()
    e = np.linalg.norm(p.T - ref, axis=1) / np.maximum(1, np.linalg.norm(ref, axis=1))
    return e.max(), np.median(e)


def test_mixed_bar(problem):
    rz, rn = _err(problem, "mixed", 1e-13, "rz"), _err(problem, "mixed", 1e-13, "rn")
    assert rz[0] <= 6e-6 and rz[1] <= 3e-6, rz
    assert rz[0] > 1e-6, rz
    assert 0.67 < rz[0] / rn[0] < 1.5, (rz, rn)


def test_split_bar_and_truncation(problem):
    rz, rn = _err(problem, "split", 1e-13, "rz"), _err(problem, "split", 1e-13, "rn")
    assert rz[0] <= 2.5e-5 and rz[1] <= 1.2e-5, rz
    assert rz[0] > 3 * rn[0], (rz, rn)


def test_mixed_truncation_floor(problem):
    rz = _err(problem, "mixed", 1e-15, "rz")
    assert rz[1] > 1e-6, rz


def test_two_stage_keeps_mixed_accuracy(problem):
    """SPLIT down to 10 tol, then MIXED from each query's last u: the defect
    correction's fixed point does not depend on its start, so the two stages
    keep MIXED's bars, at about the same total number of iterations."""
    A, y, thr, ref = problem
    p2, it2 = am.solve("two_stage", A, 1.0, y, thr, 1e-13, "rz")
    _, it1 = _solve(problem, "mixed", 1e-13, "rz")
    e = np.linalg.norm(p2.T - ref, axis=1) / np.maximum(1, np.linalg.norm(ref, axis=1))
    assert e.max() <= 6e-6 and np.median(e) <= 3e-6, e
    assert abs(it2.mean() - it1.mean()) <= 5 and np.abs(it2 - it1).max() <= 15, (it1, it2)


def test_split_stage_precision_schedule(problem):
    """A next-step design, checked in the model before any kernel: on a tile
    of the 8 queries, a one-term SPLIT product (M_hi r_hi) while the tile's
    largest squared relative change exceeds 1e-5 takes over a quarter of the
    tile's SPLIT iterations at under one extra iteration per query and keeps
    the two-stage solve's gradient bars."""
    A, y, thr, ref = problem
    p, it, tile_iters, cheap = am.two_stage_scheduled(A, 1.0, y, thr, 1e-13, "rz", 1e-5)
    _, it0, _, cheap0 = am.two_stage_scheduled(A, 1.0, y, thr, 1e-13, "rz", np.inf)
    assert cheap0 <= 2 and cheap >= 0.25 * tile_iters, (cheap0, cheap, tile_iters)
    assert it.mean() - it0.mean() <= 1.0, (it.mean(), it0.mean())
    e = np.linalg.norm(p.T - ref, axis=1) / np.maximum(1, np.linalg.norm(ref, axis=1))
    assert e.max() <= 6e-6 and np.median(e) <= 3e-6, e


def test_fp32_form_at_the_same_accuracy(problem):
    """The CUDA-core FP32 form (v = M r, FMA chains rounded to nearest) meets
    the same bars, and MIXED's gradient error is within a factor 1.5 of it:
    the metric compares the two forms at one tolerance."""
    fp32 = _err(problem, "fp32", 1e-13, "rn")
    mixed = _err(problem, "mixed", 1e-13, "rz")
    assert fp32[0] <= 6e-6 and fp32[1] <= 3e-6, fp32
    assert 1 / 1.5 <= mixed[0] / fp32[0] <= 1.5, (mixed, fp32)


def test_bf16_form_is_a_comparison_row(problem):
    """The paper's v-update in BF16 alone (one MMA per K step) stops at its
    own fixed point, ~1e-2 from the FP64 one (BF16's 2^-9 relative rounding
    of M and r, amplified through A + lam I): the form is kept for
    comparison, not for the metric's accuracy."""
    e = _err(problem, "bf16", 1e-6, "rz")
    assert 1e-3 <= e[1] and e[0] <= 5e-2, e


def test_unbuilt_tf32_and_bf16x3_forms(problem):
    """Why the TF32 and BF16 hi/lo forms are not built: in the model TF32
    (10-bit operands) stalls near a squared relative change of 1e-8 with
    ~1e-3 in the gradient, and the BF16 hi/lo split (~2^-16) cannot reach
    tol 1e-13 and at 1e-11 carries several times the error of the FP16 split
    (SPLIT) at 1e-13, which costs the same three MMAs per K step."""
    tf32 = _err(problem, "tf32", 1e-8, "rz")
    assert tf32[1] >= 3e-4, tf32
    bf3 = _err(problem, "bf16x3", 1e-11, "rz")
    split = _err(problem, "split", 1e-13, "rz")
    assert bf3[0] >= 1.5 * split[0] and bf3[0] > 2.5e-5, (bf3, split)


def test_backward_syrk_promotion():
    """The tensor-core g_A (n = 2048, 32,768 queries) in the model, on one
    off-diagonal 128 x 128 tile with shrink-sparse minimisers: promoting the
    main product every 512 queries and summing 4,096-query ranges in FP64
    keeps the error an order of magnitude inside the test bar (1e-5 of
    max |g_A|); one truncating accumulator over all the queries would not."""
    B, n = 32768, 256
    z = wl.normal(7001, B * n, 2.0).reshape(B, n)
    thr = wl.uniform(7002, B, 0.1, 3.0)[:, None]
    V = (np.sign(z) * np.maximum(np.abs(z) - thr, 0)).astype(np.float32)
    g = wl.normal(7003, B, 1.0) * 1e-3
    gs = (g * 2.0 ** np.floor(np.log2(1000.0 / np.abs(g).max()))).astype(np.float32)  # exact power-of-two scale
    X, Y = (gs[:, None] * V[:, :128]).astype(np.float32), V[:, 128:]
    exact = X.astype(np.float64).T @ Y.astype(np.float64)
    m = np.abs(exact).max()
    promoted = np.abs(am.syrk_tile(X, Y, 512, 4096) - exact).max() / m
    single = np.abs(am.syrk_tile(X, Y, B, B) - exact).max() / m
    assert promoted <= 2e-6, promoted
    assert single >= 2e-5, single


def test_mixed_l2_bar(orc):
    """H = l2 converges more slowly (about 115 iterations on these queries
    against 79 for weighted l1), so the stop rule's remaining step leaves
    more: the model's l2 gradient error sits near the median bar (3e-6) and
    within both bars, as the GPU tests find for their l2 cases."""
    A, _, _ = wl.spd_matrix(2001, 2002, N)
    x = wl.normal(2004, Q * N, 2.0).reshape(Q, N)
    t = wl.uniform(2005, Q, 0.1, 3.0)
    ref = orc.Problem(A, orc.H_L2, c0=0.5, lam=1.0, tol=1e-28, max_iter=50000,
                      stop_rule=orc.STOP_UREL).eval(x, t)["grad"]
    y = np.ascontiguousarray(x.T, dtype=np.float32)
    p, iters = am.mixed_l2(A, 1.0, y, t.astype(np.float32)[None, :], 1e-13, "rz")
    assert (iters < 3000).all() and iters.mean() > 100
    e = np.linalg.norm(p.T - ref, axis=1) / np.maximum(1, np.linalg.norm(ref, axis=1))
    assert e.max() <= 6e-6 and np.median(e) <= 3e-6, e
    assert np.median(e) >= 1.5e-6, e
