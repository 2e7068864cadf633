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
