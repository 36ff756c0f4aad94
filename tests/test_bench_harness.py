"""bench.py host logic without a GPU: the reference (oracle) arm's JSON
line, the rank-0-only rule, and the cross-rank aggregation used for N > 1
replicas, run as world_size-2 gloo process groups on the CPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "rmat16", "--steps", "2", "--warmup", "3",
                          "--ref-moves", "1"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "dtype", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_warmup_below_three_rejected():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--warmup", "1"], capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert out.returncode != 0


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist = bench.init_dist(world, "gloo")
    bench.barrier(dist)
    mx = bench.max_over_ranks(dist, float(rank + 1))
    sm = bench.sum_over_ranks(dist, 10.0 * (rank + 1))
    q.put((rank, mx, sm))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    # value = units of all ranks / the slowest rank's time
    assert res == [(0, 2.0, 30.0), (1, 2.0, 30.0)]


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "rmat16", "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, timeout=120, cwd=ROOT, env=env)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_source_hash_ignores_comments_only():
    """The committed DRAM traffic is keyed by a hash of the kernel code: a
    comment change keeps it, a code change drops it."""
    sys.path.insert(0, ROOT)
    import bench
    a = "int f(int x) { // add one\n  return x + 1; /* done */ }\n"
    b = "// header\nint f(int x) {\n  return x + 1; }\n\n"
    c = "int f(int x) { return x + 2; }\n"
    norm = lambda t: "".join(bench.code_only(t).split())
    assert norm(a) == norm(b)
    assert norm(a) != norm(c)
    assert len(bench.source_hash()) == 16


def test_sweep_bytes_skip_the_statistics_pass_of_stale_moves():
    """Algorithmic bytes of the sweep's moves: a move whose log entry has no
    statistics time (the stale threshold) carries no statistics bytes."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from paper_2008_02710_gb300 import synth
    g = bench.GpuBench.__new__(bench.GpuBench)
    g.csr = synth.CSR(4, np.array([0, 1, 2, 3, 4], np.int64), np.array([1, 2, 3, 0], np.int32), None)
    g.wl = {"precision": "mixed"}
    rec = lambda st: {"edges_pushed": 2, "green": 2, "mode": 1, "phase_us": [st, st, 1.0, 1.0, 1.0, 1.0]}
    fresh = g.alg_bytes("link_threshold", [rec(1.0), rec(1.0)], sweep=True)
    stale = g.alg_bytes("link_threshold", [rec(1.0), rec(0.0)], sweep=True)
    assert fresh["stats"] == 2 * 4 * 4 and stale["stats"] == 4 * 4
    assert fresh["select"] == stale["select"] and fresh["push"] == stale["push"]
    # per move: a 4-byte scan of every node, 48 B per green node (44 in the
    # select, the frontier read back by the push), 8 B per edge pushed
    assert fresh["select"] == 2 * (4 * 4 + 2 * 44) and fresh["push"] == 2 * (2 * 8 + 2 * 4)
    phase = g.alg_bytes("link_threshold", [rec(0.0), rec(0.0)], sweep=False)
    assert phase["stats"] == fresh["stats"]
    # all-green pulls every in-link: 8 B per link and 36 B per node with the
    # statistics pass (MIXED)
    pull = {"edges_pushed": 4, "green": 4, "mode": 2, "phase_us": [1.0] * 6}
    ag = g.alg_bytes("all_green", [pull], sweep=True)
    assert sum(ag.values()) == 4 * 8 + 4 * 36
