"""Sec. 5.2's analysis fed by the hot path itself: g(r) counts from the GPU chains, merged over two replicas by
the replicas' end-of-run exchange (two gloo ranks on the CPU), into the library's dressed-ion analysis.

A 3:-1 primitive-model electrolyte (the paper's valences, l_B = 7.117 A / 7.5 A = 0.949 sigma), 8000 ions at volume
fraction 0.01: about 1.2 sigma Debye length, so the far-field window [2.5, 5.5] sigma lies several Debye lengths
out yet inside the histogram's 8 sigma.  Two replicas (chain ids 0 and 1) sweep together on the GPU; every 5 sweeps
the interior ions' pair counts (8 sigma from the wall, as the paper excludes ions near the wall) are accumulated
per replica.  The merged counts must equal the plain sum of the replicas' counts.  From them: g(r) must show the
primitive model's structure (unlike ions piled up at contact, like ions depleted, every class within 5 % of 1 at
the histogram's far end); the analysis must give a finite kappa_R > 0 within a factor two of the bare kappa, finite
renormalised valences and dielectric ratios; and the two sides of Eq. RD as the library forms them (each q^R the
mean of its two estimates) must agree within four standard errors of their difference, estimated from eight
independent blocks of snapshots, plus 10 % for the finite window.  The individual q^R and eps_R estimates are not
checked one by one: the ones built on the charge density around the -1 ion are within the noise at this sample
size (their sign varies from run to run).
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
    base = inputs.make_chain([(2000, 3.0), (6000, -1.0)], 0.01, L_B, 1.0, 1, seed=81)
    chains = []
    for cid in range(2):
        import copy
        c = copy.copy(base)
        c.chain_id = cid
        chains.append(c)
    s = pkg.System(chains)
    s.sweep(400)  # equilibration
    n_blocks, snaps_per_block, gap = 8, 400, 5
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
    dens_p, dens_m = 2000 / V, 6000 / V

    def analyse(counts, n_ref):
        return pkg.dressed_ion_analysis(counts, R_MAX, n_ref[0], n_ref[1], dens_p, dens_m, 3.0, -1.0, L_B, *WINDOW)

    res = analyse(merged, nr)
    print({k: v for k, v in res.items() if k != "g"})
    g = res["g"]
    assert g[1][int(1.05 / (R_MAX / N_BINS))] > 2.0  # unlike ions (+3, -1) at contact
    assert g[0][int(1.05 / (R_MAX / N_BINS))] < 0.5  # like ions (+3, +3) at contact
    assert all(abs(np.nanmean(g[c][-20:]) - 1.0) < 0.05 for c in range(3))
    assert res["n_fit"] >= 3
    assert math.isfinite(res["kappa_R"]) and 0.5 * res["kappa"] < res["kappa_R"] < 2.0 * res["kappa"]
    assert all(math.isfinite(v) for v in res["qR_p"] + res["qR_m"] + res["epsR_pm"])
    diffs = []
    for b in range(n_blocks):
        rb = analyse(blocks[b].sum(0), tuple(int(v) for v in nref[b].sum(0)))
        diffs.append(rb["rd_lhs"] - rb["rd_rhs"])
    se = np.std(diffs, ddof=1) / math.sqrt(n_blocks)
    print("Eq. RD", res["rd_lhs"], res["rd_rhs"], "block differences", diffs)
    assert abs(res["rd_lhs"] - res["rd_rhs"]) <= 4.0 * se + 0.1 * abs(res["rd_lhs"]), (res["rd_lhs"], res["rd_rhs"], se)
