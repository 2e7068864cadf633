"""Chemical-potential bisection over submatrices sharded across processes.

Submatrices are independent (each molecule's columns are owned by one rank and written back locally),
so ranks split the molecules into contiguous ranges and exchange only one number per bisection point:
the FP64 sum of their partial electron counts. The bisection rule is the one of nolsm_find_mu
(Sec. "Simulation Details": mu by bisection for charge neutrality): mu = (lo + hi)/2, f < 0 raises lo,
otherwise hi is lowered, stop at |f| <= tol_n * N_occ, on the bracket width tol_mu, or after
max_bisect points. The bracket is the union of the ranks' spectral brackets.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional, Tuple


@dataclasses.dataclass
class ShardedMu:
    status: int        # 0 on success, 7 (no plateau) otherwise
    mu: float
    trace_DS: float
    steps: int
    history: list


def bisect_allreduce(count_local: Callable[[float], float], bracket_local: Tuple[float, float], n_occ: float,
                     tol_n: float, tol_mu: float, max_steps: int, group=None,
                     side_local: Optional[Callable[[bool], None]] = None) -> ShardedMu:
    """The bisection with the partial counts summed over the process group (FP64 all-reduce);
    side_local(raises_lo) is told which end of the bracket each point becomes."""
    import torch
    import torch.distributed as dist

    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else \
        torch.device("cpu")
    b = torch.tensor([-bracket_local[0], bracket_local[1]], dtype=torch.float64, device=dev)
    dist.all_reduce(b, op=dist.ReduceOp.MAX, group=group)
    lo, hi = -float(b[0]), float(b[1])
    hist = []
    mu, t = 0.5 * (lo + hi), float("nan")
    status = 7
    for step in range(1, max_steps + 1):
        mu = 0.5 * (lo + hi)
        c = torch.tensor([count_local(mu)], dtype=torch.float64, device=dev)
        dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
        t = float(c.item())
        hist.append(mu)
        f = t - n_occ
        if abs(f) <= tol_n * abs(n_occ):
            status = 0
            break
        if side_local is not None:
            side_local(f < 0.0)
        if f < 0.0:
            lo = mu
        else:
            hi = mu
        if hi - lo <= tol_mu:
            break
    return ShardedMu(status, mu, t, len(hist), hist)


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

    return bisect_allreduce(count, (lo, hi), n_occ, opts.tol_n, opts.tol_mu,
                            opts.max_bisect if opts.max_bisect > 0 else 100, group, side)
