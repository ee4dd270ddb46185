"""The multi-GPU path is replicas (voices are independent): rank r renders
batch indices r * steps + s and the reported time is the slowest rank's. The
host logic of that path is checked here on CPU with two gloo ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, steps, out):
    import torch.distributed as dist
    import bench
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": str(ws), "RANK": str(rank), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_env() == (ws, rank, rank)
    mine = torch.tensor([bench.rank_batch_index(s, ws, rank, steps) for s in range(steps)])
    gathered = [torch.zeros_like(mine) for _ in range(ws)]
    dist.all_gather(gathered, mine)
    slowest = bench.max_over_ranks(10.0 + rank, dist, torch.device("cpu"))
    out[rank] = (sorted(torch.cat(gathered).tolist()), slowest)
    dist.destroy_process_group()


def test_two_rank_replicas_cover_disjoint_batches_and_report_the_slowest():
    ws, steps = 2, 5
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(ws, _free_port(), steps, out), nprocs=ws, join=True)
    for rank in range(ws):
        indices, slowest = out[rank]
        assert indices == list(range(steps * ws))  # disjoint, nothing missed
        assert slowest == 10.0 + ws - 1
