"""The sharded bisection on two gloo ranks (CPU): each rank counts electrons of its half of the
submatrices with the FP64 oracle; the all-reduced bisection must visit exactly the points of the
single-process bisection over all submatrices and stop at the same mu. Failure detection, made on the
host: a rank that leaves between two bisection points makes the other rank's next sum fail with an
error (the group also has a 20 s timeout) instead of hanging."""
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
    import paper_2104_08245_gb300 as nl
    r = bisect_allreduce(lambda mu: orc.solve(sysm, mu, subs=subs, plan=plan).trace_DS,
                         _bracket(sysm, plan, subs), sysm.n_occ, nl.options("fp64", tol_n=1e-5, tol_mu=1e-10,
                                                                            max_bisect=100))
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


def _rank_that_leaves(rank, world, port, out):
    import datetime
    import torch.distributed as dist
    from paper_2104_08245_gb300.sharded import bisect_allreduce
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    points = []

    def count(mu):
        points.append(mu)
        if rank == 1 and len(points) == 2:
            os._exit(0)          # leaves between points, without joining the next sum
        return 0.0               # every rank below n_occ: the bisection keeps going

    try:
        import paper_2104_08245_gb300 as nl
        bisect_allreduce(count, (-1.0, 1.0), 10.0, nl.options("fp64", tol_n=1e-5, tol_mu=1e-10, max_bisect=50))
        out[rank] = "finished"
    except RuntimeError as e:    # the peer's exit (or the group's timeout) surfaces as an error, not a hang
        out[rank] = "detected: " + str(e).splitlines()[0][:80]


def test_a_rank_that_leaves_is_detected_by_the_others():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ctx = mp.start_processes(_rank_that_leaves, args=(world, port, out), nprocs=world, join=False,
                             start_method="spawn")
    for _ in range(120):                     # bounded wait: at most 120 x 1 s
        if ctx.join(timeout=1):
            break
    else:
        for p in ctx.processes:
            p.kill()
        pytest.fail("the remaining rank hung after its peer left")
    assert 1 not in out                      # rank 1 left without reporting
    assert out[0].startswith("detected")
