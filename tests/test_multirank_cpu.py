"""The multi-GPU path of bench.py is replicas: each rank owns a shard of the
pair space and the ranks exchange only their times (MAX over ranks).  Run
here with two gloo ranks on CPU."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    n = 500
    p0 = bench.shard_start(rank, n)
    P = synth.generate(synth.SKEWED, bench.SEED, n, m=150, E=6, p0=p0)
    slowest = bench.max_over_ranks(10.0 + rank, dist)
    dist.barrier()
    out[rank] = (p0, slowest, bytes(P.reads[:150 * 3]))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    import synth
    assert res[0][0] == 0 and res[1][0] == 500          # disjoint shards
    assert res[0][1] == res[1][1] == 11.0                # both see the slowest rank
    whole = synth.generate(synth.SKEWED, 0x5EED0001, 503, m=150, E=6)
    assert res[1][2] == bytes(whole.reads[500 * 150:503 * 150])  # shard = slice of the whole
