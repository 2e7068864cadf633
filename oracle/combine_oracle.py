"""Submatrix combination heuristic, plain Python -- TEST INFRASTRUCTURE ONLY (same import rule as the
rest of ``oracle/``: tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``).

Sec. "Submatrix Combination Heuristics": submatrices T_i, T_j of dimensions n_i, n_j with n_{i^j} rows in
common merge into one submatrix of n_i + n_j - n_{i^j} rows; since the work per submatrix grows with the
cube of its dimension, the merge pays if and only if (Eq. combination_criterion)

    (n_i + n_j - n_{i^j})^3 < n_i^3 + n_j^3,

used as a strict acceptance test. Candidates j for i come from the row entries of T_i (the submatrices
of the molecules that are rows of T_i); they are taken in the order of n_{j\\i} = n_j - n_{i^j}, the rows T_j
would add, from 0 upwards; at each value the valid candidates are prioritised and merged; the procedure
stops by itself when no merge improves the cubic metric. The start is one submatrix per molecule (the
paper's one per atom; here all functions of a molecule share a submatrix).

Readings of points the section leaves open:

1. Dimensions are counted in basis functions (matrix rows), the merged row set of a group is the union
   of its molecules' N(J), and a group's candidates are the groups owning a molecule among its rows.
2. One sweep: every valid ordered pair (i, j) is listed once with its level n_{j\\i} and gain
   n_i^3 + n_j^3 - (merged)^3; the pairs are taken in the order (level ascending, gain descending,
   i ascending, j ascending); a pair merges if neither group has merged earlier in the same sweep (each
   group merges at most once per sweep, so every listed level and gain is exact when it is used). The
   merged group takes the smaller of the two ids (the smallest molecule index among its members).
3. Sweeps repeat until one merges nothing; then no two groups with neighbouring molecules satisfy the
   criterion.
4. All arithmetic is on integers (the cubes are exact), so the result is unique.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def criterion(n_i: int, n_j: int, n_common: int) -> bool:
    """Eq. combination_criterion: merging pays iff (n_i + n_j - n_common)^3 < n_i^3 + n_j^3."""
    return (n_i + n_j - n_common) ** 3 < n_i ** 3 + n_j ** 3


@dataclasses.dataclass
class CombineResult:
    group_of: np.ndarray   # int32 [n_mol]: id of the group of each molecule (its smallest member)
    members: dict          # group id -> sorted list of molecules
    rows: dict             # group id -> sorted list of molecules whose functions are the group's rows
    merges: list           # (i, j, n_i, n_j, n_common) in the order they were made
    sweeps: int
    sum_n3_before: int
    sum_n3_after: int
    sum_n2_before: int
    sum_n2_after: int


def dim(rows, nbf) -> int:
    return int(sum(int(nbf[m]) for m in rows))


def combine(nbf, nb_ptr, nb_idx) -> CombineResult:
    """The heuristic on the merged pattern N(J) = nb_idx[nb_ptr[J]:nb_ptr[J+1]] (one submatrix per J)."""
    nbf = [int(x) for x in nbf]
    n_mol = len(nbf)
    rows = {J: sorted(int(m) for m in nb_idx[nb_ptr[J]:nb_ptr[J + 1]]) for J in range(n_mol)}
    members = {J: [J] for J in range(n_mol)}
    group_of = list(range(n_mol))
    n3_0 = sum(dim(r, nbf) ** 3 for r in rows.values())
    n2_0 = sum(dim(r, nbf) ** 2 for r in rows.values())
    merges = []
    sweeps = 0
    while True:
        sweeps += 1
        pairs = []
        for i in sorted(rows):
            Ri = set(rows[i])
            n_i = dim(rows[i], nbf)
            cands = sorted({group_of[m] for m in rows[i]} - {i})
            for j in cands:
                n_j = dim(rows[j], nbf)
                common = dim(Ri.intersection(rows[j]), nbf)
                if criterion(n_i, n_j, common):
                    gain = n_i ** 3 + n_j ** 3 - (n_i + n_j - common) ** 3
                    pairs.append((n_j - common, -gain, i, j, n_i, n_j, common))
        pairs.sort()
        touched = set()
        merged = 0
        for level, neg_gain, i, j, n_i, n_j, common in pairs:
            if i in touched or j in touched:
                continue
            touched.add(i)
            touched.add(j)
            keep, gone = min(i, j), max(i, j)
            rows[keep] = sorted(set(rows[i]) | set(rows[j]))
            members[keep] = sorted(members[i] + members[j])
            for m in members[keep]:
                group_of[m] = keep
            del rows[gone], members[gone]
            merges.append((i, j, n_i, n_j, common))
            merged += 1
        if merged == 0:
            break
    n3_1 = sum(dim(r, nbf) ** 3 for r in rows.values())
    n2_1 = sum(dim(r, nbf) ** 2 for r in rows.values())
    return CombineResult(np.asarray(group_of, dtype=np.int32), members, rows, merges, sweeps, n3_0, n3_1, n2_0, n2_1)


# ============================================================================ merged submatrices

def gather_rows(system_matrix, nbf, mols) -> np.ndarray:
    """The dense submatrix of a block-CSR matrix over the rows and columns of the molecules ``mols``
    (ascending), blocks placed in that order; absent blocks are zero (Sec. "The Submatrix Method",
    step (i), for a merged row set)."""
    from .nolsm_oracle import _block
    offs = np.concatenate([[0], np.cumsum([int(nbf[m]) for m in mols])]).astype(np.int64)
    T = np.zeros((int(offs[-1]), int(offs[-1])), dtype=np.float64)
    for a, I in enumerate(mols):
        for c, K in enumerate(mols):
            blk = _block(system_matrix.row_ptr, system_matrix.col_idx, system_matrix.blk_off, system_matrix.vals,
                         nbf, int(I), int(K))
            if blk is not None:
                T[offs[a]:offs[a + 1], offs[c]:offs[c + 1]] = blk
    return T


@dataclasses.dataclass
class GroupedResult:
    D_cols: dict           # J -> centre columns of J from its group's T_G(D), on the rows of N(J)
    t_S: dict              # J -> sum over J's columns j and rows i of T_G(D)_ij T_G(S)_ij
    trace_DS: float
    D_vals: np.ndarray     # D in the merged pattern (block (I, J) for I in N(J), as the per-molecule solve)


def solve_grouped(system, mu: float, group_of, plan, tol: float = 1e-9, only=None) -> GroupedResult:
    """The density matrix from merged submatrices (Sec. "Submatrix Combination Heuristics": the columns of
    all molecules of a group share one submatrix T_G over the union of their rows):
    T_G(D) = 1/2 (I - sign(T_G(S)^-1 T_G(H0) - mu I)) T_G(S)^-1 (Eq. purification_submatrix), and the
    columns of each member J are written back on the rows of N(J), so that D keeps the merged pattern of S
    and H0 (reading: the paper notes that merging could keep a denser D; this keeps the output format).
    only: solve just the groups with these labels (their members' columns and traces; no written-back D)."""
    from .nolsm_oracle import submatrix_density, write_back_cols
    nbf = plan.nbf
    group_of = np.asarray(group_of)
    cols, tS = {}, {}
    total = 0.0
    labels = sorted(set(int(x) for x in group_of))
    if only is not None:
        labels = [g for g in labels if g in set(int(x) for x in only)]
    for g in labels:
        members = [int(J) for J in np.nonzero(group_of == g)[0]]
        rows = sorted(set(int(m) for J in members for m in plan.nb_idx[plan.nb_ptr[J]:plan.nb_ptr[J + 1]]))
        offs = dict(zip(rows, np.concatenate([[0], np.cumsum([int(nbf[m]) for m in rows])])[:-1].tolist()))
        S = gather_rows(system.S, nbf, rows)
        H = gather_rows(system.H, nbf, rows)
        r = submatrix_density(S, H, mu, 0, S.shape[0], tol)
        for J in members:
            c0, bJ = offs[J], int(nbf[J])
            nJ = [int(m) for m in plan.nb_idx[plan.nb_ptr[J]:plan.nb_ptr[J + 1]]]
            sel = np.concatenate([np.arange(offs[m], offs[m] + int(nbf[m])) for m in nJ])
            cols[J] = r.D_sub[sel, c0:c0 + bJ].copy()
            t = 0.0
            for j in range(c0, c0 + bJ):
                for i in range(S.shape[0]):
                    t += r.D_sub[i, j] * S[i, j]
            tS[J] = t
            total += t
    return GroupedResult(cols, tS, total, write_back_cols(plan, cols) if only is None else None)
