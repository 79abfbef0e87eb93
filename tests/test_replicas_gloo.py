"""Multi-process plumbing of bench.py's replica mode on CPU (gloo, world size
2): barrier and the max-over-ranks step time, and distinct per-rank seeds."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo")
    import bench
    bench._barrier(world)
    m = bench._max_over_ranks(10.0 + rank, world)
    out[rank] = m
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert out[0] == 11.0 and out[1] == 11.0


def test_replica_population_seeds_differ():
    sys.path.insert(0, ROOT)
    import goac_synth as synth
    prob = synth.random_cubic_problem(n_side=4)
    a = synth.random_population(prob, 3, synth.SEED_BASE + 2 + 1000 * 0)
    b = synth.random_population(prob, 3, synth.SEED_BASE + 2 + 1000 * 1)
    assert (a != b).any()
