"""Ragged batches: many instances with their own A, H, n and query count in
one graph replay, checked per instance against the FP64 oracle and bit for
bit against single-instance evaluation (the batch runs the same kernels on
the same data; only their placement on streams and SMs changes).

Bars per instance kind are those of the single-instance tests: diagonal FP32
phi <= 1e-6 and gradient <= 2e-5 relative (floor 1); dense MIXED phi <= 1e-6
and gradient <= 6e-6 relative (floor 1)."""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

# (n, queries, dense, H): diagonal and dense instances, ragged n and query
# counts (one empty instance, several below one 128-query tile, several
# spanning tiles with a ragged tail), H cycling over l1, weighted l1, l2.
SHAPES = [(16, 5, False, 0), (37, 0, False, 1), (300, 33, False, 2), (1100, 130, False, 0),
          (20, 7, True, 1), (100, 64, True, 2), (300, 129, True, 0), (700, 3, True, 1),
          (129, 260, True, 2), (4096, 17, False, 1)]


@pytest.fixture(scope="module")
def hg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1605_01799_gb300 as pkg
    pkg.lib()
    return pkg


def _instances():
    out = []
    for i, (n, B, dense, hk) in enumerate(SHAPES):
        d = wl.ragged_instance({"index": 100 + i, "n": n, "queries": B, "dense": dense, "h_kind": hk})
        d["A"] = d["A"] if dense else d["a"]
        out.append(d)
    return out


def _descs(inst, hg):
    return [{"A": d["A"], "h_kind": d["h_kind"], "w": d["w"], "c0": d["c0"], "lam": d["lam"],
             "tol": 1e-13 if d["A"].ndim == 2 else 1e-12, "max_iter": 3000,
             "precision": hg.P_MIXED if d["A"].ndim == 2 else hg.P_FP32, "stop_rule": hg.STOP_UREL}
            for d in inst]


def _flat(inst):
    import torch
    x = np.concatenate([d["x"].reshape(-1) for d in inst]).astype(np.float32)
    t = np.concatenate([d["t"] for d in inst]).astype(np.float32)
    return torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")


def _split(out, inst):
    """Per-instance views of the batch outputs (numpy)."""
    phi = out["phi"].cpu().numpy()
    g = out["grad"].cpu().numpy()
    it = out["iters"].cpu().numpy()
    st = out["status"].cpu().numpy()
    res, q, e = [], 0, 0
    for d in inst:
        B, n = d["x"].shape
        res.append({"phi": phi[q:q + B], "grad": g[e:e + B * n].reshape(B, n), "iters": it[q:q + B],
                    "status": st[q:q + B]})
        q += B
        e += B * n
    return res


def _alloc(inst):
    import torch
    Q = sum(d["x"].shape[0] for d in inst)
    X = sum(d["x"].size for d in inst)
    return {"phi": torch.full((Q,), np.nan, dtype=torch.float64, device="cuda"),
            "grad": torch.full((X,), np.nan, dtype=torch.float32, device="cuda"),
            "dphidt": torch.empty(Q, dtype=torch.float32, device="cuda"),
            "iters": torch.empty(Q, dtype=torch.int32, device="cuda"),
            "status": torch.empty(Q, dtype=torch.uint8, device="cuda")}


@pytest.mark.parametrize("mode", [1, 2, 0])
def test_ragged_batch_against_oracle_and_single(hg, orc, mode):
    """Each schedule (1: the persistent launch, 2: per-instance launches on
    streams, 0: the tuner's pick)."""
    import torch
    inst = _instances()
    descs = _descs(inst, hg)
    b = hg.HopfBatch(descs)
    b.set_mode(mode)
    counts = [d["x"].shape[0] for d in inst]
    x, t = _flat(inst)
    out = b.eval(counts, x, t, out=_alloc(inst))
    torch.cuda.synchronize()
    info = b.info()
    assert info["nstreams"] in (1, 2, 4, 8, 16, 32) and info["used_graph"]
    assert all(ms > 0 for ms in info["tuned_ms"][:5])
    if mode:
        assert info["schedule"] == {1: "persistent", 2: "streams"}[mode]
    per = _split(out, inst)
    for i, (d, desc, r) in enumerate(zip(inst, descs, per)):
        B = d["x"].shape[0]
        if B == 0:
            continue
        assert (r["status"] == hg.Q_OK).all(), i
        # bit-identical to the same instance evaluated alone (MIXED with l1 and
        # weighted l1 in two stages on both sides)
        h = hg.Hopf(desc["A"], desc["h_kind"], w=desc["w"], c0=desc["c0"], lam=desc["lam"], tol=desc["tol"],
                    max_iter=desc["max_iter"], precision=desc["precision"], stop_rule=desc["stop_rule"])
        one = h.eval(torch.tensor(d["x"], device="cuda"), torch.tensor(d["t"], device="cuda"))
        torch.cuda.synchronize()
        assert np.array_equal(one["phi"].cpu().numpy(), r["phi"]), i
        assert np.array_equal(one["grad"].cpu().numpy(), r["grad"]), i
        assert np.array_equal(one["iters"].cpu().numpy(), r["iters"]), i
        # against the oracle
        P = orc.Problem(d["A"], d["h_kind"], w=d["w"], c0=d["c0"], lam=d["lam"], tol=1e-28, max_iter=50000,
                        stop_rule=orc.STOP_UREL)
        ref = P.eval(d["x"].astype(np.float64), d["t"].astype(np.float64))
        ep = np.abs(r["phi"] - ref["phi"]) / np.maximum(1, np.abs(ref["phi"]))
        eg = np.linalg.norm(r["grad"] - ref["grad"], axis=1) / np.maximum(1, np.linalg.norm(ref["grad"], axis=1))
        assert ep.max() <= 1e-6, (i, ep.max())
        assert eg.max() <= (6e-6 if d["A"].ndim == 2 else 2e-5), (i, eg.max())
    b.close()


def test_ragged_batch_replay_and_recapture(hg):
    """A second call with the same buffers replays the graph and reproduces
    every output bit for bit; new counts (here: every instance cut to its
    first half, one instance emptied) are captured afresh and agree with the
    first call on the rows they share, since queries are independent."""
    import torch
    inst = _instances()
    b = hg.HopfBatch(_descs(inst, hg))
    counts = [d["x"].shape[0] for d in inst]
    x, t = _flat(inst)
    out1 = b.eval(counts, x, t, out=_alloc(inst))
    torch.cuda.synchronize()
    snap = {k: v.clone() for k, v in out1.items()}
    for k in ("phi", "grad"):
        out1[k].fill_(np.nan)
    b.eval(counts, x, t, out=out1)
    torch.cuda.synchronize()
    for k in snap:
        assert torch.equal(snap[k], out1[k]), k
    # halve every instance's queries
    half = [c // 2 for c in counts]
    half[6] = 0
    sub = []
    for d, c in zip(inst, half):
        e = dict(d)
        e["x"], e["t"] = d["x"][:c], d["t"][:c]
        sub.append(e)
    xs, ts = _flat(sub)
    out2 = b.eval(half, xs, ts, out=_alloc(sub))
    torch.cuda.synchronize()
    full, part = _split(snap, inst), _split(out2, sub)
    for i, (f, p) in enumerate(zip(full, part)):
        c = half[i]
        assert np.array_equal(f["phi"][:c], p["phi"]), i
        assert np.array_equal(f["grad"][:c], p["grad"]), i
    b.close()


def test_persistent_schedule_every_branch(hg, orc):
    """The persistent launch with every kind of instance it meets: a wide
    dense instance (152 tiles: the whole grid), dense MIXED and SPLIT
    instances on lanes, a dense FP32 one and a diagonal l_inf one on their
    own launches beside it, and diagonal instances of every work-list shape
    (thread per query for n <= 4, 8, 16; warp per query for n <= 64, 256, 512;
    256 threads per query for n <= 4096).  Every output bit-identical to the
    instance evaluated alone; sampled queries against the oracle."""
    import torch
    P = hg
    spec = [  # (n, queries, dense, h_kind, precision)
        (512, 4864, True, 1, P.P_MIXED), (200, 300, True, 0, P.P_SPLIT), (150, 100, True, 2, P.P_FP32),
        (260, 700, True, 2, P.P_MIXED), (3, 1000, False, 0, P.P_FP32), (6, 500, False, 1, P.P_FP32),
        (12, 300, False, 2, P.P_FP32), (40, 257, False, 0, P.P_FP32), (200, 90, False, 1, P.P_FP32),
        (400, 33, False, 2, P.P_FP32), (3000, 40, False, 0, P.P_FP32), (20, 100, False, P.H_LINF, P.P_FP32)]
    inst, descs = [], []
    for i, (n, B, dense, hk, prec) in enumerate(spec):
        d = wl.ragged_instance({"index": 300 + i, "n": n, "queries": B, "dense": dense, "h_kind": hk % 3})
        d["A"] = d["A"] if dense else d["a"]
        d["h_kind"] = hk
        inst.append(d)
        descs.append({"A": d["A"], "h_kind": hk, "w": d["w"], "c0": d["c0"], "lam": d["lam"],
                      "tol": 1e-13 if dense else 1e-12, "max_iter": 3000, "precision": prec,
                      "stop_rule": P.STOP_UREL})
    b = hg.HopfBatch(descs)
    b.set_mode(1)
    counts = [d["x"].shape[0] for d in inst]
    x, t = _flat(inst)
    out = b.eval(counts, x, t, out=_alloc(inst))
    torch.cuda.synchronize()
    assert b.info()["schedule"] == "persistent"
    per = _split(out, inst)
    for i, (d, desc, r) in enumerate(zip(inst, descs, per)):
        assert (r["status"] == P.Q_OK).all(), i
        h = hg.Hopf(desc["A"], desc["h_kind"], w=desc["w"], c0=desc["c0"], lam=desc["lam"], tol=desc["tol"],
                    max_iter=desc["max_iter"], precision=desc["precision"], stop_rule=desc["stop_rule"])
        one = h.eval(torch.tensor(d["x"], device="cuda"), torch.tensor(d["t"], device="cuda"))
        torch.cuda.synchronize()
        for key in ("phi", "grad", "iters", "status"):
            assert np.array_equal(one[key].cpu().numpy().reshape(r[key].shape), r[key]), (i, key)
        q = np.unique([0, len(r["phi"]) // 2, len(r["phi"]) - 1])
        ref = orc.Problem(d["A"], desc["h_kind"], w=d["w"], c0=d["c0"], lam=d["lam"], tol=1e-28, max_iter=100000,
                          stop_rule=orc.STOP_UREL).eval(d["x"][q].astype(np.float64), d["t"][q].astype(np.float64))
        ep = np.abs(r["phi"][q] - ref["phi"]) / np.maximum(1, np.abs(ref["phi"]))
        assert ep.max() <= 1e-6, (i, ep.max())
    b.close()
