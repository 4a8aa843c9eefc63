"""Multi-GPU is replicas only (one independent chain per rank, no data-path collective).  The host logic of the
N > 1 bench path -- replica chain ids and the max-time / summed-moves reduction -- runs here as two gloo ranks
on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import inputs


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, moves = bench.reduce_max_sum(float(rank + 1), 10.0 * (rank + 1), world)
    out[rank] = (t, moves)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_max_time_sum_moves_two_ranks():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == (2.0, 30.0) and out[1] == (2.0, 30.0)


def test_replica_chain_ids_are_distinct_and_keep_inputs():
    import bench
    chains = [inputs.small_chain(40, seed=s, chain_id=s) for s in range(3)]
    seen = set()
    for rank in range(4):
        rep = bench.replica_chains(chains, rank)
        for a, b in zip(chains, rep):
            assert (a.pos == b.pos).all() and (a.q == b.q).all() and a.seed == b.seed
        ids = [c.chain_id for c in rep]
        assert not (seen & set(ids))
        seen |= set(ids)


def test_replicas_give_independent_draws():
    import oracle
    a = oracle.move_draws(0, 0, 12345)
    b = oracle.move_draws(0, 1, 12345)
    assert not np.array_equal(a, b)
