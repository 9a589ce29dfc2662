"""The multi-rank path of bench.py on the host: two gloo ranks on 127.0.0.1.

With N GPUs the benchmark runs one process per GPU; each rank evaluates its
own shard of the query stream (weak scaling, no collective on the data
path), the job's time is the slowest rank's, and the throughput counts the
queries of all ranks.  No GPU is involved here: the ranks exchange their
times over gloo, and the shards are checked against a single-process draw
of the same stream."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    A, w, x, t = bench.workload(16, 8, rank)
    # a rank's own "time": the slowest rank's must come back on every rank
    mx = bench.max_over_ranks([10.0 + 3.0 * rank, 5.0 - rank], ws)
    rate = bench.whole_job_rate(8, ws, mx[0])
    np.savez(os.path.join(out_dir, "rank%d.npz" % rank), x=x, t=t, mx=np.array(mx), rate=rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce(tmp_path):
    import torch.multiprocessing as mp
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, str(tmp_path))) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    import bench
    _, _, x_all, t_all = bench.workload(16, 16, 0)  # one process drawing both shards
    for r in range(ws):
        d = np.load(tmp_path / ("rank%d.npz" % r))
        # the shards partition one query stream, in rank order
        assert np.array_equal(d["x"], x_all[8 * r:8 * (r + 1)])
        assert np.array_equal(d["t"], t_all[8 * r:8 * (r + 1)])
        # element-wise maximum over the ranks, the same on every rank
        assert list(d["mx"]) == [13.0, 5.0]
        assert float(d["rate"]) == pytest.approx(2 * 8 / 13.0e-3)


def test_reference_arm_prints_on_rank_zero_only():
    """bench.py --impl reference under two ranks: rank 0 times the oracle and
    prints one JSON line; rank 1 exits 0 without work."""
    outs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1")
        p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                            "--steps", "1", "--warmup", "1", "--n", "64", "--cpu-sample", "16"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
        assert p.returncode == 0, p.stderr[-2000:]
        outs.append([l for l in p.stdout.splitlines() if l.startswith("{")])
    assert len(outs[0]) == 1 and outs[1] == []
    import json
    line = json.loads(outs[0][0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    # the same workload name as the GPU arm's line at these sizes
    assert line["config"]["workload"] == "dense_wl1_n64_b65536"
    # the line's contract: the GPU arm's keys, a cpu_baseline describing this
    # run and an e2e of the line's own value with no device copies
    for key in ("metric", "unit", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "dtype",
                "data", "vs_baseline"):
        assert key in line, key
    assert line["higher_is_better"] is True and line["unit"] == "evals/s"
    cb = line["cpu_baseline"]
    assert cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_generator_offsets_slice_one_stream():
    """The seeded generators return slices of one stream for any offset, odd
    ones included (normals come in Box-Muller pairs)."""
    sys.path.insert(0, ROOT)
    import workloads as wl
    full_n, full_u = wl.normal(7, 1001), wl.uniform(7, 1001)
    for off, cnt in [(0, 10), (1, 7), (2, 9), (13, 100), (500, 499), (1000, 1)]:
        assert np.array_equal(wl.normal(7, cnt, offset=off), full_n[off:off + cnt])
        assert np.array_equal(wl.uniform(7, cnt, offset=off), full_u[off:off + cnt])


def test_dense_work_counts():
    """The roofline's algorithmic work is the method's one n x n product per
    iteration plus the set-up and final products, 2 n^2 (K + 2) per query,
    for every form; the executed work is the form's own product count."""
    sys.path.insert(0, ROOT)
    import bench
    n, K = 1024, np.array([44, 75, 120])
    alg, exe = bench.dense_work(n, K, "mixed")
    assert alg == 2.0 * n * n * (K + 2).sum()
    assert exe == 2.0 * n * n * (4 * K + 3).sum()
    assert bench.dense_work(n, K, "bf16") == (alg, 2.0 * n * n * (K + 3).sum())
    assert bench.dense_work(n, K, "fp32") == (alg, 2.0 * n * n * (K + 1).sum())


def test_clock_record_parsing(tmp_path):
    """The clocks record of a timed region (nvidia-smi CSV, no units): the
    median SM clock and the max clock of the benchmarked GPU only, every
    throttle reason seen active at least once, lines from other GPUs and
    malformed lines ignored, and "unsampled" when nothing was read."""
    sys.path.insert(0, ROOT)
    import bench
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join([
        "0, 2070, 2070, 910.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1, 1200, 2070, 300.0, 0x0000000000000020, Not Active, Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
        "0, 2040, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    ]) + "\n")
    r = bench.read_clocks(str(p), 0)
    assert r == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    r1 = bench.read_clocks(str(p), 1)
    assert r1["sm_mhz"] == 1200.0 and r1["reasons"] == ["hw_thermal_slowdown"]
    assert bench.read_clocks(str(tmp_path / "missing.csv"), 0)["reasons"] == ["unsampled"]


def test_splitmix64_matches_its_definition():
    """The input generator is SplitMix64 (Steele, Lea & Flood 2014): the
    counter form used here equals the sequential definition (state advanced
    by the golden-ratio increment modulo 2^64, then the two xor-shift-multiply
    rounds) written out with Python integers, at any offset; seed 1234567
    gives the widely published first outputs; uniforms are the top 53 bits."""
    sys.path.insert(0, ROOT)
    import workloads as wl
    mask = (1 << 64) - 1

    def sequential(seed, count):
        s, out = seed & mask, []
        for _ in range(count):
            s = (s + 0x9E3779B97F4A7C15) & mask
            z = s
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
            out.append(z ^ (z >> 31))
        return out

    for seed in (0, 1, 1234567, 2004, (1 << 64) - 1):
        ref = sequential(seed, 300)
        assert [int(v) for v in wl.splitmix64(seed, 300)] == ref
        assert [int(v) for v in wl.splitmix64(seed, 50, offset=123)] == ref[123:173]
        u = wl.uniform(seed, 300)
        assert np.array_equal(u, np.array([(v >> 11) / 2.0 ** 53 for v in ref]))
        assert (u >= 0).all() and (u < 1).all()
    assert [int(v) for v in wl.splitmix64(1234567, 5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431, 16408922859458223821]


def test_matrix_and_normal_generators():
    """The workloads' dense A = Q diag(s) Q^T: symmetric, Q orthogonal, the
    spectrum exactly the drawn s (within FP64 rounding), so cond(A) is
    bounded by s_hi / s_lo; Haar Q: E[Q_ij^2] = 1/n over many draws.  The
    Box-Muller normals have mean 0 and variance std^2 (5-sigma bounds)."""
    sys.path.insert(0, ROOT)
    import workloads as wl
    n = 64
    A, Q, s = wl.spd_matrix(9101, 9102, n)
    assert np.array_equal(A, A.T)
    assert np.abs(Q.T @ Q - np.eye(n)).max() < 1e-13
    ev = np.linalg.eigvalsh(A)
    assert np.allclose(ev, np.sort(s), rtol=1e-12, atol=1e-13)
    assert s.min() >= 0.1 and s.max() <= 10.0
    # a Haar row is uniform on the sphere: E[x_j^2] = 1/m, Var = (2m - 2) / (m^2 (m + 2))
    m, draws = 8, 400
    sq = np.mean([wl.haar_orthogonal(9200 + k, m)[0] ** 2 for k in range(draws)], axis=0)
    sd = np.sqrt((2 * m - 2) / (m * m * (m + 2)) / draws)
    assert np.abs(sq - 1 / m).max() < 5 * sd
    z = wl.normal(9301, 200000, std=2.0)
    assert abs(z.mean()) < 5 * 2.0 / np.sqrt(z.size)
    assert abs(z.var() / 4.0 - 1) < 5 * np.sqrt(2.0 / z.size)
