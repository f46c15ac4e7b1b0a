"""CPU: the replica plumbing of bench.py with world size 2 on gloo (barrier,
max over ranks, whole-job throughput), and the reference arm (the oracle on
host cores) printing its one line on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import bench
    d = bench.Dist(device=torch.device("cpu"))
    try:
        d.barrier()
        # rank r "took" 10 + 5 r ms for its images and "saw" clock 1400 + r MHz
        ms, mhz = d.max(10.0 + 5.0 * rank, 1400.0 + rank)
        value = bench.replica_value(2.0e6, ms, d.world)
        d.barrier()
        q.put((rank, ms, mhz, value))
    finally:
        d.close()


def test_two_replicas_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms, mhz, value in out:
        assert ms == 15.0 and mhz == 1401.0              # max over both ranks on every rank
        assert value == pytest.approx(2 * 2.0e6 / 15e-3 / 1e9)   # both ranks' units / slowest time


def test_replica_value_single():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_value(16777216, 0.1, 1) == pytest.approx(167.77216)


def _run_reference(rank, workload="config1"):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                           workload, "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env,
                          stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, timeout=600)


def test_reference_arm_other_ranks_exit_quietly():
    r = _run_reference(1)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line_on_rank0():
    r = _run_reference(0)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    for key in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
                "cpu_baseline", "e2e"):
        assert key in line
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_kernel_hash_ignores_comments(tmp_path, monkeypatch):
    # the recorded DRAM traffic stays valid across comment edits of the kernel
    import importlib
    import sys
    sys.path.insert(0, ROOT)
    bench = importlib.import_module("bench")
    src = open(os.path.join(ROOT, bench.KERNEL_SOURCES[1][0])).read()
    (tmp_path / "a.cuh").write_text(src)
    (tmp_path / "b.cuh").write_text("// a new comment\n" + src.replace("namespace gb {", "namespace gb {  /* x */", 1))
    (tmp_path / "c.cuh").write_text(src.replace("kBand = 8", "kBand = 16", 1))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    hashes = []
    for name in ("a.cuh", "b.cuh", "c.cuh"):
        monkeypatch.setattr(bench, "KERNEL_SOURCES", {1: [name]})
        hashes.append(bench.kernel_hash(1))
    assert hashes[0] == hashes[1] and hashes[0] != hashes[2]
