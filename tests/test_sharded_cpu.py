"""The sharded bisection on two gloo ranks (CPU): each rank counts electrons of its half of the
submatrices with the FP64 oracle; the all-reduced bisection must visit exactly the points of the
single-process bisection over all submatrices and stop at the same mu."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import nolsm_oracle as orc
from synth import make_system, SystemSpec


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _spec():
    return SystemSpec(3, 3, 2, cutoff=4.5, seed=31)


def _bracket(sysm, plan, subs):
    lo, hi = np.inf, -np.inf
    for J in subs:
        S = orc.gather(plan, J, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
        H = orc.gather(plan, J, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
        A = orc.overlap_inverse(S) @ H
        d = np.diag(A)
        R = np.sum(np.abs(A), axis=1) - np.abs(d)
        lo, hi = min(lo, float(np.min(d - R))), max(hi, float(np.max(d + R)))
    return lo, hi


def _rank(rank, world, port, out):
    import torch.distributed as dist
    from paper_2104_08245_gb300.sharded import bisect_allreduce
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sysm = make_system(_spec())
    plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    n = sysm.n_mol
    subs = list(range(n * rank // world, n * (rank + 1) // world))
    r = bisect_allreduce(lambda mu: orc.solve(sysm, mu, subs=subs, plan=plan).trace_DS,
                         _bracket(sysm, plan, subs), sysm.n_occ, 1e-5, 1e-10, 100)
    out[rank] = (r.status, r.mu, r.trace_DS, r.history)
    dist.destroy_process_group()


def test_two_rank_bisection_matches_single_process():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    sysm = make_system(_spec())
    plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    lo, hi = _bracket(sysm, plan, range(sysm.n_mol))
    ref = orc.find_mu(lambda mu: orc.solve(sysm, mu, plan=plan).trace_DS, sysm.n_occ, lo, hi,
                      tol_n=1e-5 * sysm.n_occ)
    for rank in range(world):
        status, mu, t, hist = out[rank]
        assert status == 0 and ref.ok
        assert hist == [m for m, _ in ref.history]
        assert mu == ref.mu
        assert t == pytest.approx(ref.trace_DS, abs=1e-9)
