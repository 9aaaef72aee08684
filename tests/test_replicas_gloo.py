"""Multi-rank host logic on CPU (gloo, world size 2): replicas with disjoint shift
batches combine to exactly the estimate of one solve over the union of the shifts."""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2003_11183_gb300 import replicas
from oracle import sov


@pytest.fixture(scope="module", autouse=True)
def built_library():
    # the pooled estimate is the library's (tlrmvn_estimate_pooled, host code: no GPU needed)
    import __graft_entry__ as ge
    ge.build()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, per_shift, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = replicas.gather_and_combine(per_shift[rank])
    out[rank] = res
    dist.destroy_process_group()


def test_combine_equals_single_solve_estimate():
    rng = np.random.default_rng(0)
    logP = rng.normal(-50.0, 2.0, size=(6, 40))          # 6 shifts x 40 points, per-sample logs
    logp, err, ell = sov.estimate(logP.ravel(), 6, 40)   # one solve over all 6 shifts
    got = replicas.combine([ell[:2], ell[2:5], ell[5:]])  # three replicas
    assert abs(got[0] - logp) < 1e-12 and abs(got[1] - err) < 1e-12


def test_rank_seeds_disjoint():
    seeds = {replicas.rank_seed(7, r, 20) for r in range(8)}
    assert len(seeds) == 8


def test_two_rank_gloo_gather():
    rng = np.random.default_rng(1)
    per_shift = [rng.normal(-30, 1, 5), rng.normal(-30, 1, 7)]  # uneven shift counts per rank
    want = replicas.combine(per_shift)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, per_shift, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        for r in range(2):
            assert abs(out[r][0] - want[0]) < 1e-12 and abs(out[r][1] - want[1]) < 1e-12
