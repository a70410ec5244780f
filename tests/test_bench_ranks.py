"""Host logic of bench.py for N > 1 ranks, on the CPU (gloo, world size 2).

The path does not shard (every rank compresses its own field), so the only
multi-rank logic is the timing: whole-job throughput is every rank's bytes
over the slowest rank's time, and the reference arm runs on rank 0 alone.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, vals, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        q.put((rank, bench.max_over_ranks(vals[rank], "cpu")))
    finally:
        torch.distributed.destroy_process_group()


def test_max_over_ranks_gloo():
    ws, vals = 2, [3.25, 7.5]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, vals, q)) for r in range(ws)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 7.5, 1: 7.5}


def test_max_over_ranks_single_process():
    assert bench.max_over_ranks(2.5, "cpu") == 2.5


def test_whole_job_throughput():
    # two ranks of 1 GB each, the slower one taking 10 ms: 200 GB/s
    assert bench.whole_job_gbs(2, 1e9, 10.0) == pytest.approx(200.0)
    assert bench.whole_job_gbs(1, 2.16e9, 5.4) == pytest.approx(400.0)


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-edge", "16"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_profiled_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    """The DRAM traffic recorded under profiles/ is reported only while the
    block-kernel sources still hash to the digest recorded with it."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    digest = bench.kernel_source_digest()
    (prof / "block_fwd_grf513.md").write_text(
        "- traffic_bytes_per_launch: 123456\n- kernel_source_sha256: `%s`\n" % digest)
    src = tmp_path / "paper_2609_00205_gb300" / "csrc"
    src.mkdir(parents=True)
    for rel in bench.BLOCK_KERNEL_SOURCES:
        (tmp_path / rel).write_bytes(open(os.path.join(ROOT, rel), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._profiled_traffic() == 123456.0
    (tmp_path / bench.BLOCK_KERNEL_SOURCES[0]).write_text("// changed\n")
    assert bench._profiled_traffic() is None
