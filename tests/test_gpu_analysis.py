"""Sec. 5.2's analysis fed by the hot path itself: g(r) counts from the GPU chains, merged over two replicas by
the replicas' end-of-run exchange (two gloo ranks on the CPU), into the library's dressed-ion analysis.

A 3:-1 primitive-model electrolyte (the paper's valences, l_B = 7.117 A / 7.5 A = 0.949 sigma) at volume fraction
0.01: about 1.2 sigma Debye length, so the far-field window [2.5, 5.5] sigma lies several Debye lengths out yet
inside the histogram's 8 sigma.  Two replicas (chain ids 0 and 1) sweep together on the GPU; every 5 sweeps the
interior ions' pair counts (8 sigma from the wall, as the paper excludes ions near the wall) are accumulated per
replica.  The merged counts must equal the plain sum of the replicas' counts; the analysis must give finite
kappa_R, q_+^R > 0 > q_-^R and eps_R > 0, and both sides of Eq. RD must agree within four standard errors of their
difference, estimated from independent blocks of snapshots.
"""
import math
import os
import socket

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

N_BINS, R_MAX, MARGIN = 160, 8.0, 8.0
L_B = 7.117 / 7.5
WINDOW = (2.5, 5.5)


def _free_port():
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    port = sk.getsockname()[1]
    sk.close()
    return port


def _rank_merge(rank, port, per_rank, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    from paper_1602_05716_gb300 import replicas
    c, r = replicas.merge_counts(per_rank[rank][0], per_rank[rank][1])
    out[rank] = (c.tolist(), r)
    dist.barrier()
    dist.destroy_process_group()


def _merge_over_gloo(per_rank):
    """Each replica's counts on its own gloo rank (CPU processes, no GPU), summed by the end-of-run exchange."""
    import torch.multiprocessing as tmp
    mgr = tmp.get_context("spawn").Manager()
    out = mgr.dict()
    tmp.start_processes(_rank_merge, args=(_free_port(), per_rank, out), nprocs=2, start_method="spawn", join=True)
    c0, r0 = out[0]
    c1, r1 = out[1]
    assert c0 == c1 and r0 == r1
    return np.array(c0, dtype=np.uint64), tuple(r0)


def test_dressed_ion_analysis_from_gpu_chains():
    import paper_1602_05716_gb300 as pkg
    from paper_1602_05716_gb300 import replicas
    pkg.build()
    base = inputs.make_chain([(1000, 3.0), (3000, -1.0)], 0.01, L_B, 1.0, 1, seed=81)
    chains = []
    for cid in range(2):
        import copy
        c = copy.copy(base)
        c.chain_id = cid
        chains.append(c)
    s = pkg.System(chains)
    s.sweep(200)  # equilibration
    n_blocks, snaps_per_block, gap = 4, 50, 5
    blocks = np.zeros((n_blocks, 2, 3, N_BINS), np.uint64)
    nref = np.zeros((n_blocks, 2, 2), np.int64)
    for b in range(n_blocks):
        for _ in range(snaps_per_block):
            s.sweep(gap)
            for k in range(2):
                s.gr_histogram(chain=k, n_bins=N_BINS, r_max=R_MAX, wall_margin=MARGIN, counts=blocks[b, k])
                nref[b, k] += replicas.interior_reference_counts(s.positions(k), base.q, base.R, base.sigma, MARGIN)
    s.close()
    per_rank = [(blocks[:, k].sum(0), tuple(int(v) for v in nref[:, k].sum(0))) for k in range(2)]
    merged, nr = _merge_over_gloo(per_rank)
    assert (merged == per_rank[0][0] + per_rank[1][0]).all()
    assert nr == (per_rank[0][1][0] + per_rank[1][1][0], per_rank[0][1][1] + per_rank[1][1][1])

    V = 4.0 / 3.0 * math.pi * base.R ** 3
    dens_p, dens_m = 1000 / V, 3000 / V

    def analyse(counts, n_ref):
        return pkg.dressed_ion_analysis(counts, R_MAX, n_ref[0], n_ref[1], dens_p, dens_m, 3.0, -1.0, L_B, *WINDOW)

    res = analyse(merged, nr)
    print({k: v for k, v in res.items() if k != "g"})
    assert res["n_fit"] >= 3
    assert math.isfinite(res["kappa_R"]) and res["kappa_R"] > 0
    assert res["qR_p"][0] > 0 and res["qR_p"][1] > 0 and res["qR_m"][0] < 0 and res["qR_m"][1] < 0
    assert all(math.isfinite(e) and e > 0 for e in res["epsR_pm"])
    # Eq. RD within statistics: the spread of the difference over independent blocks (both replicas per block)
    diffs = []
    for b in range(n_blocks):
        rb = analyse(blocks[b].sum(0), tuple(int(v) for v in nref[b].sum(0)))
        diffs.append(rb["rd_lhs"] - rb["rd_rhs"])
    se = np.std(diffs, ddof=1) / math.sqrt(n_blocks)
    print("Eq. RD", res["rd_lhs"], res["rd_rhs"], "block differences", diffs)
    assert abs(res["rd_lhs"] - res["rd_rhs"]) <= 4.0 * se + 1e-12, (res["rd_lhs"], res["rd_rhs"], se)
