"""The N > 1 benchmark path (replicas, max over ranks) on CPU with gloo, world size 2."""
import json
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2602_09020_gb300 import replicas
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = 0.5 + rank  # rank 1 is the slowest
    tmax = replicas.max_over_ranks(t, dist)
    rate = replicas.whole_job_rate(1000.0, tmax, world)
    out.put((rank, tmax, rate))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, rate in res:
        assert tmax == 1.5
        assert abs(rate - 2 * 1000.0 / 1.5) < 1e-9


def test_single_process_identity():
    sys.path.insert(0, ROOT)
    from paper_2602_09020_gb300 import replicas
    assert replicas.max_over_ranks(3.25) == 3.25
    assert replicas.whole_job_rate(10, 2.0, 1) == 5.0
    with pytest.raises(ValueError):
        replicas.whole_job_rate(10, 0.0, 1)


def test_reference_arm_prints_one_json_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "10", "--terms", "60",
           "--trotter-steps", "1", "--steps", "1", "--warmup", "1"]
    res = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr
    lines = [l for l in res.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "rotations/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
