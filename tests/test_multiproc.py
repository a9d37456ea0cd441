"""The multi-rank path of bench.py on CPU with the gloo backend (world size 2): each rank
takes its own query shard (weak scaling, no data-path collective) and the step time is the
maximum over ranks."""
import os
import socket

import numpy as np


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import meshgen
    wl = meshgen.workload(2, scale=2048 / 1048576)
    X, F = wl.single
    q = bench.rank_queries(wl, X.astype(np.float32), F, rank)
    t = bench.max_over_ranks(10.0 + rank, world)
    out[rank] = (t, len(q), float(q.v[:, 0].sum()), int(q.face.max() < len(F)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_shards_and_max_time():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0][0] == out[1][0] == 11.0          # max over ranks
    assert out[0][1] == out[1][1] == 2048          # equal shard sizes (weak scaling)
    assert out[0][2] != out[1][2]                  # distinct query batches
    assert out[0][3] == out[1][3] == 1
