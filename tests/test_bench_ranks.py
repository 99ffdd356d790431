"""The multi-rank (N > 1) figures of bench.py on two gloo ranks on the CPU: every rank fits its own
replica, the job time is the slowest rank's, the iterations are summed over the ranks, and the
reference arm prints from rank 0 only."""
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, it = bench.job_totals(dist, 1.0 + rank, 100 * (rank + 1), torch.device("cpu"))
    out.put((rank, t, it))
    dist.destroy_process_group()


def test_job_totals_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, it in res:
        assert t == 2.0 and it == 300.0


def test_single_process_totals():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(None, 1.5, 7, None) == (1.5, 7.0)


def test_reference_arm_prints_from_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, env=env,
                       timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
