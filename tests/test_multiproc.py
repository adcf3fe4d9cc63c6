"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): ranks own
disjoint blocks of models, and the step time is the max over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2603_16393_gb300 import inputs
    B = 3
    seed0 = bench.rank_seed0(rank, B)
    vt, _, _ = bench.workload_inputs(bench.WORKLOADS["70x70"], B, seed0)
    local = [10.0 + rank, 20.0 - rank, 1.0 * rank]
    mx = bench.max_over_ranks(local, world)
    # every rank sees the same maximum
    got = [None] * world
    dist.all_gather_object(got, (seed0, mx, float(vt.sum())))
    if rank == 0:
        out.put(got)
    dist.destroy_process_group()


def test_two_ranks_shard_models_and_take_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (s0, m0, v0), (s1, m1, v1) = got
    assert (s0, s1) == (0, 3)                 # disjoint seed blocks
    assert m0 == m1 == [11.0, 20.0, 1.0]      # element-wise max over ranks
    assert v0 != v1                           # different models per rank
