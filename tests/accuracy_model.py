"""A numpy model of the dense tensor-core forms' arithmetic (test support).

It derives the gradient tolerances of the dense parity tests from the
arithmetic: it runs the split Bregman iteration (eq. 3.4(a)-(c), in the
u-form u^k = v^k + b^{k-1}) with the number formats and the accumulation
order that the tensor-core kernels use, and compares the returned gradient
d^K with the FP64 oracle's.

- Operands: FP16 (RN) with the two-term split x ~ hi + 2^-11 lo',
  lo' = fp16((x - hi) 2^11); BF16 (RN) for the defect-correction step.
- Products: one MMA multiplies K = 16 pairs; the 16 products and their sum
  are taken exactly (FP16 x FP16 products are exact in FP32), then added to
  an FP32 accumulator, either rounded to nearest ("rn") or truncated toward
  zero ("rz").  Accumulators sum the n / 16 K steps in order; the correction
  terms of a split product share one accumulator, interleaved per K step,
  and the BF16 product alternates K steps between two accumulators.
- Elementwise work (prox, b, g, the state) in FP32.
- BF16 ("bf16"): v = bf16(M) bf16(r), the paper's form in one MMA per K
  step (alternating accumulators).
- Forms not built, for comparison: TF32 ("tf32": v = tf32(M) tf32(r), K = 8
  per MMA) and the BF16 hi/lo split ("bf16x3": x = bf16(x) + bf16(x - hi),
  three MMAs per K step, ~2^-16).
- The CUDA-core form ("fp32"): v = M r with FP32 M and r, one fused
  multiply-add per term in order, rounded to nearest.

SPLIT:  v^{k+1} = M r^k with both M and r^k = y + lam (2 p^k - u^k) split;
        u^{k+1} = v^{k+1} + u^k - p^k.
MIXED:  g^k = y - A p^k - lam (u^k - p^k) with A p^k split (g stored in
        BF16), u^{k+1} = u^k + bf16(M) g^k; the fixed point g = 0 does not
        depend on the rounding of M.
Both stop at the first k >= 2 with |u^k - u^{k-1}|^2 <= tol max(1, |u^k|^2).
Two stages: SPLIT down to a looser tolerance, then MIXED from each query's
last u (a stop allowed from its first step), as the library's default MIXED
solve for l1 and weighted l1 does.

The backward contraction g_A = -1/2 V^T diag(g) V (syrk_tile): the same
splits, the main product promoted to FP32 registers every chunk of queries,
the ranges of queries summed in FP64.

This is a model of the hardware's arithmetic, not of the kernels' code:
the parity tests on the GPU measure the kernels themselves.  Only ``tests/``
uses it.
"""
import numpy as np

K_STEP = 16
LO_SCALE = np.float32(2048.0)


def round_f32(s, mode):
    """FP64 values to FP32, rounded to nearest ("rn") or toward zero ("rz")."""
    f = s.astype(np.float32)
    if mode == "rz":
        over = np.abs(f.astype(np.float64)) > np.abs(s)
        f[over] = np.nextafter(f[over], np.float32(0))
    return f


def to_bf16(x):
    """FP32 to BF16 (round to nearest, ties to even), returned as FP32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + (((b >> 16) & 1) + 0x7FFF)) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32)


def split_fp16(x):
    """Two-term FP16 split (hi, lo') of an FP32 array, returned as FP32."""
    hi = x.astype(np.float16).astype(np.float32)
    lo = ((x - hi) * LO_SCALE).astype(np.float16).astype(np.float32)
    return hi, lo


def to_tf32(x):
    """FP32 to TF32 (10 explicit mantissa bits, round to nearest even), as FP32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + (((b >> 13) & 1) + 0xFFF)) & 0xFFFFE000).astype(np.uint32)
    return b.view(np.float32)


def k_step_products(A, B, ks=K_STEP):
    """P[k] = A[:, ks k:ks (k+1)] @ B[ks k:ks (k+1), :], exact in FP64
    (ks = 16 for FP16 / BF16 MMAs, 8 for TF32)."""
    nk = A.shape[1] // ks
    Ar = A.astype(np.float64).reshape(A.shape[0], nk, ks).transpose(1, 0, 2)
    return np.matmul(Ar, B.astype(np.float64).reshape(nk, ks, B.shape[1]))


def accumulate(products, mode):
    """One FP32 accumulator over the K steps of each product array in
    ``products`` (issued in turn within each K step)."""
    acc = None
    for k in range(products[0].shape[0]):
        for P in products:
            acc = round_f32(P[k] if acc is None else acc.astype(np.float64) + P[k], mode)
    return acc


def split_product(Xh, Xl, Yh, Yl, mode):
    """X Y ~ D1 + 2^-11 D2, D1 = Xh Yh, D2 = Xh Yl' + Xl' Yh."""
    d1 = accumulate([k_step_products(Xh, Yh)], mode)
    d2 = accumulate([k_step_products(Xh, Yl), k_step_products(Xl, Yh)], mode)
    return d1 + d2 / LO_SCALE


def _prox(u, thr):
    return (np.sign(u) * np.maximum(np.abs(u) - thr, 0)).astype(np.float32)


def _iterate(step, y, thr, tol, max_iter, u0=None, k_min=2):
    """Run ``step(u, p) -> u_next`` per query until the relative rule stops
    it (from k >= k_min).  The start is u = p = y (v^0 = d^0 = y, b^0 = 0),
    or u = u0 with p = prox(u0) for a warm start.  Returns (p, iters, u)."""
    q = y.shape[1]
    if u0 is None:
        u, p = y.copy(), y.copy()
    else:
        u, p = u0.copy(), _prox(u0, thr)
    iters, done = np.zeros(q, np.int64), np.zeros(q, bool)
    for k in range(1, max_iter + 1):
        un = step(u, p)
        du = (un - u).astype(np.float64)
        ru = (du * du).sum(0) / np.maximum(1.0, (un.astype(np.float64) ** 2).sum(0))
        act = ~done
        pn = _prox(un, thr)
        u[:, act], p[:, act] = un[:, act], pn[:, act]
        iters[act] = k
        if k >= k_min:
            done |= ru <= tol
        if done.all():
            break
    return p, iters, u


def solve(form, A, lam, y, thr, tol, mode, max_iter=3000, split_start=None):
    """Gradients d^K (n x q, FP32) and iteration counts of the weighted-l1
    problem with J*(v) = 1/2 v^T A v and thresholds thr = (t / lam) w
    (n x q), for y = x - c given as n x q columns.  form "two_stage": SPLIT
    iterations down to split_start (default 10 tol), then MIXED ones from
    each query's last u, stopping from their first step on; the counts add."""
    if form == "two_stage":
        s = 10 * tol if split_start is None else split_start
        _, it1, u1 = _iterate(_step("split", A, lam, y, mode), y, thr, s, max_iter)
        p, it2, _ = _iterate(_step("mixed", A, lam, y, mode), y, thr, tol, max_iter, u0=u1, k_min=1)
        return p, it1 + it2
    p, iters, _ = _iterate(_step(form, A, lam, y, mode), y, thr, tol, max_iter)
    return p, iters


def two_stage_scheduled(A, lam, y, thr, tol, mode, theta, max_iter=3000):
    """The two-stage solve with a precision schedule in its SPLIT stage, for
    one column tile (all columns of y): the tile takes v = M_hi r_hi (one
    MMA per K step) until the largest squared relative change among its
    active queries is within theta, the three-term product after; queries
    stop (at 10 tol) only once the tile is precise.  Returns (p, total
    iterations per query, the tile's SPLIT iterations, how many of them
    were one-term)."""
    n, q = y.shape
    M = np.linalg.inv(A + lam * np.eye(n)).astype(np.float32)
    Mh, Ml = split_fp16(M)
    lam32 = np.float32(lam)
    u, p = y.copy(), y.copy()
    it1, done = np.zeros(q, np.int64), np.zeros(q, bool)
    precise, cheap = False, 0
    for k in range(1, max_iter + 1):
        r = (y + lam32 * (np.float32(2) * p - u)).astype(np.float32)
        rh, rl = split_fp16(r)
        if precise:
            v = split_product(Mh, Ml, rh, rl, mode)
        else:
            v = accumulate([k_step_products(Mh, rh)], mode)
            cheap += 1
        un = (v + (u - p)).astype(np.float32)
        du = (un - u).astype(np.float64)
        ru = (du * du).sum(0) / np.maximum(1.0, (un.astype(np.float64) ** 2).sum(0))
        act = ~done
        u[:, act], p[:, act] = un[:, act], _prox(un, thr)[:, act]
        it1[act] = k
        if k >= 2:
            if precise:
                done |= ru <= 10 * tol
            else:
                precise = ru[act].max() <= theta
        if done.all():
            break
    p, it2, _ = _iterate(_step("mixed", A, lam, y, mode), y, thr, tol, max_iter, u0=u, k_min=1)
    return p, it1 + it2, int(it1.max()), cheap


def _step(form, A, lam, y, mode):
    n = A.shape[0]
    M = np.linalg.inv(A + lam * np.eye(n)).astype(np.float32)
    lam32 = np.float32(lam)
    if form == "split":
        Mh, Ml = split_fp16(M)

        def step(u, p):
            r = (y + lam32 * (np.float32(2) * p - u)).astype(np.float32)
            v = split_product(Mh, Ml, *split_fp16(r), mode)
            return (v + (u - p)).astype(np.float32)
    elif form == "mixed":
        Ah, Al = split_fp16(A.astype(np.float32))
        Mb = to_bf16(M)

        def step(u, p):
            ap = split_product(Ah, Al, *split_fp16(p), mode)
            g = to_bf16(y - ap - lam32 * (u - p))
            P = k_step_products(Mb, g)
            du = accumulate([P[0::2]], mode) + accumulate([P[1::2]], mode)
            return (u + du).astype(np.float32)
    elif form == "bf16":
        Mb = to_bf16(M)

        def step(u, p):
            r = to_bf16(y + lam32 * (np.float32(2) * p - u))
            P = k_step_products(Mb, r)
            v = accumulate([P[0::2]], mode) + accumulate([P[1::2]], mode)
            return (v + (u - p)).astype(np.float32)
    elif form == "tf32":
        Mt = to_tf32(M)

        def step(u, p):
            r = to_tf32(y + lam32 * (np.float32(2) * p - u))
            P = k_step_products(Mt, r, 8)
            v = accumulate([P[0::2]], mode) + accumulate([P[1::2]], mode)
            return (v + (u - p)).astype(np.float32)
    elif form == "bf16x3":
        Mh = to_bf16(M)
        Ml = to_bf16(M - Mh)

        def step(u, p):
            r = (y + lam32 * (np.float32(2) * p - u)).astype(np.float32)
            rh = to_bf16(r)
            rl = to_bf16(r - rh)
            d1 = accumulate([k_step_products(Mh, rh)], mode)
            d2 = accumulate([k_step_products(Mh, rl), k_step_products(Ml, rh)], mode)
            return (d1 + d2 + (u - p)).astype(np.float32)
    elif form == "fp32":
        def step(u, p):
            r = (y + lam32 * (np.float32(2) * p - u)).astype(np.float32)
            return (fma_chain(M, r) + (u - p)).astype(np.float32)
    else:
        raise ValueError(form)
    return step


def fma_chain(X, Y):
    """X Y as one FP32 fused multiply-add per term, in order over K (the
    CUDA-core form's accumulation): each step rounds acc + x y once."""
    Xd, Yd = X.astype(np.float64), Y.astype(np.float64)
    acc = np.zeros((X.shape[0], Y.shape[1]), np.float32)
    for k in range(X.shape[1]):
        acc = round_f32(acc.astype(np.float64) + Xd[:, k:k + 1] * Yd[k:k + 1, :], "rn")
    return acc


def syrk_tile(X, Y, chunk_q, range_q, mode="rz"):
    """One tile of the backward contraction X^T Y over the queries (X, Y:
    [B][128] FP32, query-major), as the tensor-core SYRK forms it: two-term
    FP16 splits, X_hi Y_hi accumulated chunk_q queries at a time and promoted
    into FP32 registers, X_hi Y_lo' + X_lo' Y_hi in a correction accumulator
    over each range of range_q queries, the ranges summed in FP64."""
    B = X.shape[0]
    Xh, Xl = split_fp16(X)
    Yh, Yl = split_fp16(Y)
    total = np.zeros((X.shape[1], Y.shape[1]))
    for r0 in range(0, B, range_q):
        r1 = min(B, r0 + range_q)
        acc = np.zeros((X.shape[1], Y.shape[1]), np.float32)
        for c0 in range(r0, r1, chunk_q):
            c1 = min(r1, c0 + chunk_q)
            acc = (acc + accumulate([k_step_products(Xh[c0:c1].T, Yh[c0:c1])], mode)).astype(np.float32)
        corr = accumulate([k_step_products(Xh[r0:r1].T, Yl[r0:r1]), k_step_products(Xl[r0:r1].T, Yh[r0:r1])],
                          mode)
        total += (acc + corr / LO_SCALE).astype(np.float32).astype(np.float64)
    return total


def mixed_l2(A, lam, y, tau, tol, mode, max_iter=3000):
    """The MIXED form with H = l2 (one stage): p = s u with
    s = max(0, 1 - tau / |u|) (shrink_2), the operand planes hold u and
    A p = s (A u); the first product takes p = y.  tau: (1, q) FP32."""
    n, q = y.shape
    M = np.linalg.inv(A + lam * np.eye(n)).astype(np.float32)
    Ah, Al = split_fp16(A.astype(np.float32))
    Mb = to_bf16(M)
    lam32 = np.float32(lam)

    def prox(u):
        nrm = np.sqrt((u.astype(np.float64) ** 2).sum(0)).astype(np.float32)
        s = np.where(nrm > tau[0], 1 - tau[0] / np.maximum(nrm, np.float32(1e-30)), 0).astype(np.float32)
        return (u * s[None, :]).astype(np.float32), s

    u, p, s = y.copy(), y.copy(), np.ones(q, np.float32)
    iters, done = np.zeros(q, np.int64), np.zeros(q, bool)
    for k in range(1, max_iter + 1):
        au = split_product(Ah, Al, *split_fp16(u if k > 1 else y), mode)
        ap = au * s[None, :] if k > 1 else au
        g = to_bf16(y - ap - lam32 * (u - p))
        P = k_step_products(Mb, g)
        du = accumulate([P[0::2]], mode) + accumulate([P[1::2]], mode)
        un = (u + du).astype(np.float32)
        ru = (du.astype(np.float64) ** 2).sum(0) / np.maximum(1.0, (un.astype(np.float64) ** 2).sum(0))
        act = ~done
        pn, sn = prox(un)
        u[:, act], p[:, act], s[act] = un[:, act], pn[:, act], sn[act]
        iters[act] = k
        if k >= 2:
            done |= ru <= tol
        if done.all():
            break
    return p, iters
