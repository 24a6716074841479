"""Replica bookkeeping of the benchmark under torch.distributed (gloo, world size 2, CPU):
each rank draws its own coil minibatches and the job time is the slowest rank's."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2408_02367_gb300 import synth
    ws, r, _ = bench.dist_env()
    draws = synth.coil_minibatches(8, 2, 5, seed=bench.rank_seed(synth.SEED_COILS_DRAW, r))
    t = 10.0 + 5.0 * r
    tmax = bench.max_over_ranks(t, dist, torch.device("cpu"))
    out[rank] = (ws, r, tmax, [d.tolist() for d in draws])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_draw_independently():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == 2 and res[1][0] == 2
    assert res[0][2] == res[1][2] == 15.0
    assert res[0][3] != res[1][3]
