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


def test_each_rank_halo_holds_its_neighbourhoods():
    """A rank's extracted input (its halo) is the union of its molecules' N(J) from the oracle's plan, its
    owned range maps to a contiguous local range, and every owned T_J(S), T_J(H0) gathered from the halo equals
    the one gathered from the whole input; the halo is much smaller than the whole system."""
    from paper_2104_08245_gb300.sharded import extract_halo
    sysm = make_system(SystemSpec(6, 6, 6, seed=33))
    plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    world = 4
    for rank in range(world):
        j0, j1 = sysm.n_mol * rank // world, sysm.n_mol * (rank + 1) // world
        h = extract_halo(sysm, j0, j1)
        want = sorted({int(I) for J in range(j0, j1) for I in plan.nb_idx[plan.nb_ptr[J]:plan.nb_ptr[J + 1]]})
        assert list(h.mols) == want
        assert list(h.mols[h.l0:h.l1]) == list(range(j0, j1))
        hs = h.system
        lp = orc.build_plan(hs.nbf, hs.S.row_ptr, hs.S.col_idx, hs.H.row_ptr, hs.H.col_idx)
        for J in range(j0, j1, 7):
            L = J - j0 + h.l0
            for M, HM in ((sysm.S, hs.S), (sysm.H, hs.H)):
                full = orc.gather(plan, J, M.row_ptr, M.col_idx, M.blk_off, M.vals)
                part = orc.gather(lp, L, HM.row_ptr, HM.col_idx, HM.blk_off, HM.vals)
                assert np.array_equal(full, part)
        assert len(h.mols) < sysm.n_mol


def _rank_halo(rank, world, port, out):
    import torch.distributed as dist
    from paper_2104_08245_gb300.sharded import bisect_allreduce, extract_halo
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sysm = make_system(_spec())
    n = sysm.n_mol
    j0, j1 = n * rank // world, n * (rank + 1) // world
    h = extract_halo(sysm, j0, j1)            # this rank holds only its halo from here on
    hs = h.system
    lp = orc.build_plan(hs.nbf, hs.S.row_ptr, hs.S.col_idx, hs.H.row_ptr, hs.H.col_idx)
    subs = list(range(h.l0, h.l1))

    class _Local:
        pass
    loc = _Local()
    loc.S, loc.H, loc.nbf = hs.S, hs.H, hs.nbf
    lo, hi = _bracket(loc, lp, subs)
    import paper_2104_08245_gb300 as nl
    r = bisect_allreduce(lambda mu: orc.solve(loc, mu, subs=subs, plan=lp).trace_DS, (lo, hi), sysm.n_occ,
                         nl.options("fp64", tol_n=1e-5, tol_mu=1e-10, max_bisect=100))
    out[rank] = (r.status, r.mu, r.trace_DS, r.history, len(h.mols))
    dist.destroy_process_group()


def test_two_rank_bisection_on_halos_matches_single_process():
    """The same two-rank bisection with every rank holding only its halo: the same points and mu."""
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_halo, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    sysm = make_system(_spec())
    plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    lo, hi = _bracket(sysm, plan, range(sysm.n_mol))
    ref = orc.find_mu(lambda mu: orc.solve(sysm, mu, plan=plan).trace_DS, sysm.n_occ, lo, hi,
                      tol_n=1e-5 * sysm.n_occ)
    for rank in range(world):
        status, mu, t, hist, held = out[rank]
        assert status == 0 and ref.ok
        assert hist == [m for m, _ in ref.history]
        assert mu == ref.mu
        assert t == pytest.approx(ref.trace_DS, abs=1e-9)
