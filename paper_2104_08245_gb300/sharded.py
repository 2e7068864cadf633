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


@dataclasses.dataclass
class Halo:
    """The part of the input one rank needs for its molecules [j0, j1): the molecules of the union of their
    neighbourhoods N(J) (the halo, ascending global ids), the block rows of S and H0 of those molecules
    restricted to columns in the halo, renumbered 0 .. len(mols)-1; the rank's molecules are the local range
    [l0, l1)."""
    mols: "object"           # int32 [m]: global id of every local molecule
    l0: int
    l1: int
    system: "object"         # a synth-like object with nbf, S, H (BlockCSR-like), n_occ, occ, and the
                             # geometry of the halo's molecules (pos, onsite, cell, spec, dirs) when known


def extract_halo(system, j0: int, j1: int) -> Halo:
    """Host-side extraction of a rank's halo (once per geometry): N(J) is the merged pattern of S and H0 in
    block column J (the submatrix's rows, Sec. "The Non-Orthogonal Local Submatrix Method"); every submatrix
    of the rank needs the blocks (I, K) with I, K in N(J), which are among the halo's rows and columns. The
    pattern stays structurally symmetric (it is the full one restricted to the halo on both sides), so the
    plan built from it reproduces N(J), T_J(S) and T_J(H0) of every owned J exactly."""
    import numpy as np

    n = int(system.nbf.shape[0])
    # N(J) of the owned molecules from the symmetric patterns: block column J = block row J
    mols = np.unique(np.concatenate([system.S.col_idx[system.S.row_ptr[j0]:system.S.row_ptr[j1]],
                                     system.H.col_idx[system.H.row_ptr[j0]:system.H.row_ptr[j1]]])).astype(np.int32)
    loc = np.full(n, -1, dtype=np.int64)
    loc[mols] = np.arange(mols.shape[0])

    def ranges(starts, counts):
        """Concatenation of [starts[k], starts[k] + counts[k]) over k."""
        tot = int(np.sum(counts))
        if tot == 0:
            return np.zeros(0, dtype=np.int64)
        base = np.repeat(starts - np.concatenate([[0], np.cumsum(counts)[:-1]]), counts)
        return base + np.arange(tot, dtype=np.int64)

    def restrict(M):
        rp = M.row_ptr.astype(np.int64)
        ps = ranges(rp[mols], rp[mols + 1] - rp[mols])                  # the halo's block rows
        keep = ps[loc[M.col_idx[ps]] >= 0]                               # restricted to halo columns
        row_of = np.repeat(np.arange(mols.shape[0]), (rp[mols + 1] - rp[mols]))[loc[M.col_idx[ps]] >= 0]
        row_ptr = np.zeros(mols.shape[0] + 1, dtype=np.int64)
        np.cumsum(np.bincount(row_of, minlength=mols.shape[0]), out=row_ptr[1:])
        sizes = M.blk_off[keep + 1] - M.blk_off[keep]
        blk = np.zeros(keep.shape[0] + 1, dtype=np.int64)
        np.cumsum(sizes, out=blk[1:])
        vals = M.vals[ranges(M.blk_off[keep], sizes)]
        return type(M)(row_ptr.astype(np.int32), loc[M.col_idx[keep]].astype(np.int32), blk, vals)

    S, H = restrict(system.S), restrict(system.H)
    get = lambda k: getattr(system, k, None)
    sub = dataclasses.make_dataclass("HaloSystem", ["nbf", "S", "H", "occ", "n_occ", "pos", "onsite", "cell", "spec",
                                                    "dirs"])(
        system.nbf[mols].astype(np.int32), S, H, system.occ[mols] if get("occ") is not None else None,
        float(np.sum(system.occ[j0:j1])) if get("occ") is not None else 0.0,
        system.pos[mols] if get("pos") is not None else None,
        [system.onsite[int(g)] for g in mols] if get("onsite") is not None else None,
        get("cell"), get("spec"), get("dirs"))
    return Halo(mols, int(loc[j0]), int(loc[j1 - 1]) + 1, sub)
