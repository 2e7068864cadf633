"""Chemical-potential bisection over submatrices sharded across processes.

Submatrices are independent (each molecule's columns are owned by one rank and written back locally),
so ranks split the molecules into contiguous ranges and exchange only numbers: the union of their
spectral brackets once, then per bisection point the FP64 sum of their partial electron counts. Every
decision of the bisection (Sec. "Simulation Details": mu by bisection for charge neutrality) is taken
by the library's nolsm_bisection_start / nolsm_bisection_update, the same calls nolsm_find_mu makes, so
the ranks visit the points a single process would. This module only all-reduces.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Callable, Optional, Tuple

from . import _abi


@dataclasses.dataclass
class ShardedMu:
    status: int        # 0 on success, 7 (no plateau) otherwise
    mu: float
    trace_DS: float
    steps: int
    history: list


def bisect_allreduce(count_local: Callable[[float], float], bracket_local: Tuple[float, float], n_occ: float,
                     opts, group=None, side_local: Optional[Callable[[bool], None]] = None) -> ShardedMu:
    """The bisection with the partial counts summed over the process group (FP64 all-reduce);
    side_local(raises_lo) is told which end of the bracket each point becomes. opts: nolsm_options
    (tol_n, tol_mu, max_bisect)."""
    import torch
    import torch.distributed as dist

    lib = _abi.load(build_if_missing=True)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else \
        torch.device("cpu")
    b = torch.tensor([-bracket_local[0], bracket_local[1]], dtype=torch.float64, device=dev)
    dist.all_reduce(b, op=dist.ReduceOp.MAX, group=group)
    st = _abi.NolsmBisection()
    rc = lib.nolsm_bisection_start(ctypes.byref(st), float(n_occ), -float(b[0]), float(b[1]))
    if rc != 0:
        raise RuntimeError(f"nolsm_bisection_start: {lib.nolsm_last_error().decode()}")
    hist = []
    mu = st.mu
    while st.state == _abi.BISECT_EVALUATE:
        mu = st.mu
        c = torch.tensor([count_local(mu)], dtype=torch.float64, device=dev)
        dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
        hist.append(mu)
        raises = ctypes.c_int32(0)
        rc = lib.nolsm_bisection_update(ctypes.byref(st), float(c.item()), ctypes.byref(opts), ctypes.byref(raises))
        if rc != 0:
            raise RuntimeError(f"nolsm_bisection_update: {lib.nolsm_last_error().decode()}")
        if st.state != _abi.BISECT_ACCEPTED and side_local is not None:
            side_local(bool(raises.value))
    status = 0 if st.state == _abi.BISECT_ACCEPTED else _abi.ERR_NO_PLATEAU
    return ShardedMu(status, mu, st.trace_DS, st.steps, hist)


def sharded_find_mu(plan, n_occ: float, opts, group=None) -> ShardedMu:
    """nolsm_find_mu for a plan whose options select this rank's range of submatrices: each point
    solves only the rank's submatrices with an eigenvalue left in the bracket (the union of the ranks'
    Gershgorin brackets holds every eigenvalue, so the counts at its ends are known)."""
    import paper_2104_08245_gb300 as nl
    lo, hi = nl.nolsm_spectral_bracket(plan, opts)
    nl.nolsm_bisect_begin(plan, opts, True)

    def count(mu):
        return nl.nolsm_bisect_point(plan, mu, opts)[1]

    def side(raises_lo):
        nl.nolsm_bisect_side(plan, opts, raises_lo)

    return bisect_allreduce(count, (lo, hi), n_occ, opts, group, side)
