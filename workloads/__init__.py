"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module only draws numbers: it holds none of the Hopf method's arithmetic.
Every array comes from SplitMix64 (Steele, Lea & Flood 2014, the constants of
its published definition) used in counter form: the i-th draw of stream
``seed`` is mix(seed + (i+1) * 0x9E3779B97F4A7C15).  Uniforms take the top 53
bits; normals come from Box-Muller pairs; a Haar-distributed orthogonal Q is
the QR factor of a Gaussian matrix with the signs of diag(R) folded in
(Mezzadri 2007).  Seeds are ``1000 * workload + role`` with roles
1 = A / Q, 2 = spectrum or semi-axes, 3 = weights, 4 = x, 5 = t, 6 = centres,
7 = sampled query indices.

The workloads follow the shapes of the paper's experiments (ellipsoidal
initial sets, l1 / l2 Hamiltonians, Section 4.5: uniform draws of (x, t))
scaled up to the dimensions and batch sizes of the GPU workloads.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, count, offset=0):
    """Counter-based SplitMix64: ``count`` 64-bit outputs of stream ``seed``."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed, count, lo=0.0, hi=1.0, offset=0):
    u = (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def log_uniform(seed, count, lo, hi, offset=0):
    return np.exp(uniform(seed, count, np.log(lo), np.log(hi), offset))


def normal(seed, count, std=1.0, offset=0):
    """Box-Muller: pairs (u1, u2) -> sqrt(-2 ln(1-u1)) (cos, sin)(2 pi u2).
    Normal i of the stream is the cos (i even) or sin (i odd) of pair i // 2,
    whose uniforms are numbers 2 (i // 2) and 2 (i // 2) + 1 of the uniform
    stream, so a call with an offset returns a slice of the same stream."""
    if count <= 0:
        return np.zeros(0)
    p0, p1 = offset // 2, (offset + count - 1) // 2
    u = uniform(seed, 2 * (p1 - p0 + 1), offset=2 * p0)
    r = np.sqrt(-2.0 * np.log1p(-u[0::2]))
    th = 2.0 * np.pi * u[1::2]
    z = np.empty(2 * (p1 - p0 + 1))
    z[0::2] = r * np.cos(th)
    z[1::2] = r * np.sin(th)
    s = offset - 2 * p0
    return std * z[s:s + count]


def haar_orthogonal(seed, n):
    G = normal(seed, n * n).reshape(n, n)
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))


def spd_matrix(seed_q, seed_s, n, s_lo=0.1, s_hi=10.0):
    """A = Q diag(s) Q^T with Q Haar and s log-uniform in [s_lo, s_hi].
    Returns (A, Q, s) so that tests can use the known eigen-decomposition."""
    Q = haar_orthogonal(seed_q, n)
    s = log_uniform(seed_s, n, s_lo, s_hi)
    A = (Q * s) @ Q.T
    A = 0.5 * (A + A.T)
    return A, Q, s


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# --- workload 1: plain method, FP64, n = 8, diagonal A, H = l1 -------------
def diag_l1_fp64(n=8, batch=1000, w=1):
    a = uniform(1000 * w + 2, n, 0.5, 2.0)
    x = uniform(1000 * w + 4, batch * n, -3.0, 3.0).reshape(batch, n)
    t = uniform(1000 * w + 5, batch, 0.1, 2.0)
    return {"n": n, "a": a, "x": x, "t": t, "h_kind": 0, "c0": 0.5, "lam": 1.0, "tol": 1e-10, "max_iter": 500}


# --- workload 2: dense A, n = 1024, weighted l1, 65,536 queries --------------
def dense_wl1(n=1024, batch=65536, w=2, x_std=2.0, t_lo=0.1, t_hi=3.0):
    A, Q, s = spd_matrix(1000 * w + 1, 1000 * w + 2, n)
    wts = uniform(1000 * w + 3, n, 0.5, 1.5)
    x = _f32(normal(1000 * w + 4, batch * n, x_std).reshape(batch, n))
    t = _f32(uniform(1000 * w + 5, batch, t_lo, t_hi))
    return {"n": n, "A": A, "Q": Q, "s": s, "w": wts, "x": x, "t": t, "h_kind": 1, "c0": 0.5, "lam": 1.0}


def queries_dense(n, batch, w=2, x_std=2.0, t_lo=0.1, t_hi=3.0, offset=0):
    """Only the (x, t) draws of a dense workload (lets a caller regenerate a
    slice of the query stream without rebuilding A)."""
    x = _f32(normal(1000 * w + 4, batch * n, x_std, offset=offset * n).reshape(batch, n))
    t = _f32(uniform(1000 * w + 5, batch, t_lo, t_hi, offset=offset))
    return x, t


# --- workload 3: union of K ellipsoids, n = 256, H = l2 -----------------------
def ellipsoid_union(n=256, K=16, batch=16384, w=3, x_std=5.0, c_std=3.0, t_lo=0.0, t_hi=2.0):
    semi = log_uniform(1000 * w + 2, K * n, 0.2, 5.0).reshape(K, n)
    centres = normal(1000 * w + 6, K * n, c_std).reshape(K, n)
    xs, ts = [], []
    drawn = 0
    chunk = max(1024, batch)
    while sum(len(v) for v in xs) < batch:
        x = normal(1000 * w + 4, chunk * n, x_std, offset=drawn * n).reshape(chunk, n).astype(np.float32)
        drawn += chunk
        # reject points inside any ellipsoid: sum(((x - c)/semi)^2) <= 1
        inside = np.zeros(chunk, bool)
        xd = x.astype(np.float64)
        for k in range(K):
            inside |= (((xd - centres[k]) / semi[k]) ** 2).sum(1) <= 1.0
        xs.append(x[~inside])
    x = np.concatenate(xs)[:batch]
    t = _f32(uniform(1000 * w + 5, batch, t_lo, t_hi))
    return {"n": n, "K": K, "semi": semi, "a": semi ** 2, "centres": centres, "x": _f32(x), "t": t,
            "h_kind": 2, "c0": 0.5, "lam": 1.0}


# --- workload 4: ragged batch of instances ----------------------------------
def ragged(count=512, n_lo=16, n_hi=4096, q_lo=64, q_hi=8192, w=4, dense_from=None):
    """Instance descriptions only (A and queries are drawn per instance by
    ``ragged_instance`` so that a caller can build a subset)."""
    ns = np.rint(log_uniform(1000 * w + 2, count, n_lo, n_hi)).astype(int)
    qs = np.rint(log_uniform(1000 * w + 7, count, q_lo, q_hi)).astype(int)
    dense_from = count // 2 if dense_from is None else dense_from
    return [{"index": i, "n": int(ns[i]), "queries": int(qs[i]), "dense": i >= dense_from, "h_kind": i % 3}
            for i in range(count)]


def ragged_instance(desc, w=4):
    i, n, B = desc["index"], desc["n"], desc["queries"]
    base = 1000 * w + 10 * (i + 1) * 1000
    out = {"n": n, "h_kind": desc["h_kind"], "c0": 0.5, "lam": 1.0}
    if desc["dense"]:
        A, Q, s = spd_matrix(base + 1, base + 2, n)
        out.update(A=A, Q=Q, s=s)
    else:
        out["a"] = uniform(base + 2, n, 0.5, 2.0)
    out["w"] = uniform(base + 3, n, 0.5, 1.5) if desc["h_kind"] == 1 else None
    out["x"] = _f32(normal(base + 4, B * n, 2.0).reshape(B, n))
    out["t"] = _f32(uniform(base + 5, B, 0.1, 3.0))
    return out


def ragged_instances(descs, w=4, workers=None):
    """``ragged_instance`` for every description, drawn in a pool of
    ``spawn``-started processes (safe after CUDA is initialised).  x, t, the
    diagonals and weights equal those of the serial loop bit for bit; a dense
    A agrees to rounding (the QR factorisation behind the Haar Q runs with
    one BLAS thread per worker, which may round differently)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    workers = workers or min(16, os.cpu_count() or 1)
    if workers <= 1 or len(descs) < 2:
        return [ragged_instance(d, w) for d in descs]
    # largest first so that the pool stays busy to the end
    order = sorted(range(len(descs)), key=lambda i: -descs[i]["n"] * (descs[i]["n"] if descs[i]["dense"] else 1))
    out = [None] * len(descs)
    # one BLAS thread per worker: the pool is the parallelism
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            futs = {ex.submit(ragged_instance, descs[i], w): i for i in order}
            for f in cf.as_completed(futs):
                out[futs[f]] = f.result()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return out


# --- workload 5: differentiation, n = 2048, H = l1 ---------------------------
def dense_l1_grad(n=2048, batch=32768, w=5):
    A, Q, s = spd_matrix(1000 * w + 1, 1000 * w + 2, n)
    x = _f32(normal(1000 * w + 4, batch * n, 2.0).reshape(batch, n))
    t = _f32(uniform(1000 * w + 5, batch, 0.1, 3.0))
    idx = np.sort(np.unique((uniform(1000 * w + 7, 256) * batch).astype(int)))[:64]
    return {"n": n, "A": A, "Q": Q, "s": s, "w": None, "x": x, "t": t, "h_kind": 0, "c0": 0.5, "lam": 1.0,
            "fd_queries": idx}
