"""Host logic of the multi-GPU bench path (independent replicas, one series
per rank) on CPU with two gloo ranks: each rank draws its own series, the
step time is the maximum over ranks, and the whole-job rate counts every
rank's units over that time.  Also: a non-zero rank of the reference leg
exits without work."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    import synth
    wl = synth.workload("tiny")
    x = synth.make_series(wl.n, wl.injections, bench.rank_seed(wl.seed, rank))
    t_ms = 100.0 + 25.0 * rank          # rank 1 is the slower one
    tmax = bench.max_over_ranks(t_ms, ws, "cpu")
    rate = bench.aggregate_rate(ws, wl.K * 2 * wl.nb, 10, tmax)
    q.put((rank, tmax, rate, x[:64].copy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_replica_bookkeeping():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        rank, tmax, rate, head = q.get(timeout=120)
        out[rank] = (tmax, rate, head)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import synth
    wl = synth.workload("tiny")
    # every rank sees the slowest rank's time and the same whole-job rate
    assert out[0][0] == out[1][0] == 125.0
    units = 2 * wl.K * 2 * wl.nb * 10
    assert out[0][1] == out[1][1] == pytest.approx(units / 0.125)
    # independent series per rank
    assert not np.array_equal(out[0][2], out[1][2])


def test_reference_leg_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "3"], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
