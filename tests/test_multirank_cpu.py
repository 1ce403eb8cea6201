"""The N > 1 benchmark path on CPU ranks (gloo, world size 2).

The filter shards as independent replicas (no data-path collective): the
only cross-rank step is the whole-job aggregation of bench.py (work summed
over ranks, the slowest rank's time), checked here on two gloo ranks; and
the reference arm run under torchrun prints exactly one line, from rank 0.
"""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.job_totals(100.0 * (rank + 1), 2.0 + 3.0 * rank, world, "cpu")))
    finally:
        dist.destroy_process_group()


def test_job_totals_on_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # units summed over the ranks, the slowest rank's time, the same on both
    assert out[0] == out[1] == (300.0, 5.0)
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(7.0, 1.5, 1) == (7.0, 1.5)


def test_reference_arm_under_torchrun_prints_one_line():
    env = dict(os.environ, PHD_REF_BUDGET_S="20")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
