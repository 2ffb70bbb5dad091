"""The N > 1 host logic of bench.py on CPU: gloo ranks (world size 2) agree on the max-over-ranks
step time and the whole-job throughput; the reference arm's other ranks exit without work."""
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


def _rank(rank, world, port, ms, n_dof, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        q.put((rank, bench.rank_aggregate(ms[rank], n_dof, world, device="cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_rank_aggregate_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ms, n_dof, port = [3.0, 5.0], 1000, _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, ms, n_dof, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = dict(q.get(timeout=10) for _ in range(2))
    for r in range(2):
        ms_max, value = got[r]
        assert ms_max == 5.0
        assert value == pytest.approx(2 * n_dof / 5e-3, rel=1e-15)


def test_rank_aggregate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    ms_max, value = bench.rank_aggregate(2.5, 400, 1, device="cpu")
    assert ms_max == 2.5 and value == pytest.approx(400 / 2.5e-3)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    assert res.stdout.strip() == ""
