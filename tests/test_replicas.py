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


def _merge_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1602_05716_gb300 import replicas
    counts = np.full((3, 5), 10 * (rank + 1), np.uint64)
    counts[1, 2] = 2 ** 40 + rank  # large counts survive the int64 reduction
    merged, n_ref = replicas.merge_counts(counts, (3 + rank, 7 * rank))
    series = np.linspace(0.0, 1.0, 6) * (rank + 1) - 5.0 * rank
    stack = replicas.gather_series(series)
    out[rank] = (merged.tolist(), n_ref, stack.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_merge_counts_and_stack_series_two_ranks():
    """End of a replica run, two gloo ranks: g(r) and reference-ion counts summed, energy series stacked in rank
    order on every rank; the stack feeds the ensemble autocorrelation (Sec. 5.2's overline over processes)."""
    import oracle
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_merge_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    want = np.full((3, 5), 30, np.uint64)
    want[1, 2] = 2 ** 41 + 1
    s0 = np.linspace(0.0, 1.0, 6) - 0.0
    s1 = np.linspace(0.0, 1.0, 6) * 2 - 5.0
    for r in range(2):
        merged, n_ref, stack = out[r]
        assert (np.array(merged, np.uint64) == want).all()
        assert n_ref == (7, 7)
        assert np.array_equal(np.array(stack), np.stack([s0, s1]))
    C, _ = oracle.energy_autocorr(np.array(out[0][2]), 2)
    assert C[0] == 1.0


def test_merge_without_a_process_group_is_the_identity():
    from paper_1602_05716_gb300 import replicas
    c = np.arange(6, dtype=np.uint64).reshape(3, 2)
    m, n = replicas.merge_counts(c, (2, 3))
    assert (m == c).all() and n == (2, 3)
    assert replicas.gather_series([1.0, 2.0]).shape == (1, 2)


def test_interior_reference_counts_match_the_histogram_totals():
    """With r_max beyond every pair distance the histogram counts every ordered pair around each reference ion,
    so its class totals must be N_ref,+ (N_+ - 1), N_ref,+ N_- + N_ref,- N_+ and N_ref,- (N_- - 1), with the
    reference counts taken by the same interior rule (checked with and without a wall margin)."""
    import oracle
    from paper_1602_05716_gb300 import replicas
    ch = inputs.small_chain(300, phi=0.15, seed=44, two_one=True)
    oc = oracle.OracleChain.from_chain(ch)
    oc.sweep(2)
    x = oc.positions()
    n_p, n_m = int((ch.q > 0).sum()), int((ch.q < 0).sum())
    for margin in (0.0, 1.5, 3.0):
        counts = oc.gr_histogram(n_bins=8, r_max=2.0 * ch.R + 1.0, wall_margin=margin)
        rp, rm = replicas.interior_reference_counts(x, ch.q, ch.R, ch.sigma, margin)
        assert counts[0].sum() == rp * (n_p - 1)
        assert counts[1].sum() == rp * n_m + rm * n_p
        assert counts[2].sum() == rm * (n_m - 1)
        if margin > 0:
            assert rp + rm < n_p + n_m
