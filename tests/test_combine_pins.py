"""Pins of the combination heuristic's oracle (Sec. "Submatrix Combination Heuristics",
Eq. combination_criterion) against facts fixed by hand or by the structure of the input:

* the criterion's consequences: a submatrix contained in another always merges, disjoint ones never,
  and for n_i = n_j = 100 the threshold lies where 200 - n_common crosses 100 * 2^(1/3) = 125.99;
* a three-molecule chain worked through by hand (the level order and the tie rule decide the pairs);
* a periodic cell that the cutoff spans (every submatrix the whole matrix: everything merges, in
  log2 sweeps) and isolated molecules (nothing merges);
* on an atom-resolved ions-in-water pattern: the groups partition the sites, a replay of the merge log
  from scratch reproduces every logged dimension, each merge passed the criterion, the cubic metric
  falls by exactly the logged gains, and no two final groups with neighbouring members would still
  pass the criterion (the stopping rule);
* planted mistakes (a criterion on squares, the common rows not subtracted) that the replay or the
  stopping-rule pin catches;
* the density from merged submatrices: singleton groups give the per-molecule solve exactly, and one
  group of every molecule gives the full matrix's density (LAPACK's generalized eigensolver).
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import combine_oracle as co
from oracle import nolsm_oracle as orc
from synth import SystemSpec, make_site_pattern, make_system, spec_ions_in_water_small, spec_tiny


def _pattern(sysm):
    p = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    return p.nbf, p.nb_ptr, p.nb_idx


@pytest.fixture(scope="module")
def ions():
    sp = make_site_pattern(spec_ions_in_water_small())
    return sp, co.combine(sp.nbf, sp.nb_ptr, sp.nb_idx)


def test_criterion_consequences():
    for n_i, n_j in ((1, 1), (7, 300), (250, 40)):
        assert co.criterion(n_i, n_j, min(n_i, n_j))      # one row set inside the other
        assert not co.criterion(n_i, n_j, 0)              # nothing in common
    assert not co.criterion(100, 100, 74)                 # 126^3 = 2,000,376 > 2,000,000
    assert co.criterion(100, 100, 75)                     # 125^3 = 1,953,125 < 2,000,000


def test_three_molecule_chain_by_hand():
    # N(0) = {0,1}, N(1) = {0,1,2}, N(2) = {1,2}, one function each: n = 2, 3, 2.
    # Sweep 1 lists (0,1) level 1, (1,0) level 0, (1,2) level 0, (2,1) level 1, all with gain
    # 8 + 27 - 27 = 8; (1,0) comes first (level 0, then i = 1, j = 0) and merges into group 0 = {0,1}
    # with rows {0,1,2}; (1,2) is skipped (group 1 merged in this sweep). Sweep 2 merges {0,1} and {2}
    # (common 2, merged n 3: 27 < 27 + 8). Sweep 3 finds nothing.
    r = co.combine([1, 1, 1], [0, 2, 5, 7], [0, 1, 0, 1, 2, 1, 2])
    assert r.merges == [(1, 0, 3, 2, 2), (0, 2, 3, 2, 2)]
    assert r.sweeps == 3
    assert list(r.group_of) == [0, 0, 0]
    assert (r.sum_n3_before, r.sum_n3_after) == (43, 27)


def test_whole_cell_merges_everything():
    sysm = make_system(spec_tiny(2))            # 8 molecules, every N(J) = all 8, n = 48
    r = co.combine(*_pattern(sysm))
    assert list(r.group_of) == [0] * 8
    assert r.sweeps == 4                        # 8 -> 4 -> 2 -> 1 groups, then a sweep with nothing
    assert (r.sum_n3_before, r.sum_n3_after) == (8 * 48 ** 3, 48 ** 3)


def test_isolated_molecules_never_merge():
    r = co.combine(*_pattern(make_system(SystemSpec(3, 3, 2, cutoff=1.5, seed=14))))
    assert r.merges == [] and r.sweeps == 1
    assert list(r.group_of) == list(range(18))


def _replay(nbf, nb_ptr, nb_idx, merges):
    rows = {J: set(int(m) for m in nb_idx[nb_ptr[J]:nb_ptr[J + 1]]) for J in range(len(nbf))}
    dim = lambda s: sum(int(nbf[m]) for m in s)
    gains = 0
    for i, j, n_i, n_j, common in merges:
        assert (dim(rows[i]), dim(rows[j]), dim(rows[i] & rows[j])) == (n_i, n_j, common)
        merged = n_i + n_j - common
        assert merged ** 3 < n_i ** 3 + n_j ** 3
        gains += n_i ** 3 + n_j ** 3 - merged ** 3
        keep, gone = min(i, j), max(i, j)
        rows[keep] = rows[i] | rows[j]
        del rows[gone]
    return rows, gains


def _stopping_rule_violations(nbf, r):
    dim = lambda s: sum(int(nbf[m]) for m in s)
    bad = 0
    for i, Ri in r.rows.items():
        nbr = {int(r.group_of[m]) for m in Ri} - {i}
        for j in nbr:
            n_i, n_j, c = dim(Ri), dim(r.rows[j]), dim(set(Ri) & set(r.rows[j]))
            bad += (n_i + n_j - c) ** 3 < n_i ** 3 + n_j ** 3
    return bad


def test_ions_in_water_invariants(ions):
    sp, r = ions
    n = sp.n_sites
    # partition, group ids = smallest member, rows = union of the members' neighbourhoods
    seen = sorted(m for ms in r.members.values() for m in ms)
    assert seen == list(range(n))
    for g, ms in r.members.items():
        assert g == min(ms) and all(r.group_of[m] == g for m in ms)
        union = sorted(set(int(x) for J in ms for x in sp.nb_idx[sp.nb_ptr[J]:sp.nb_ptr[J + 1]]))
        assert r.rows[g] == union
    rows, gains = _replay(sp.nbf, sp.nb_ptr, sp.nb_idx, r.merges)
    assert {g: sorted(s) for g, s in rows.items()} == r.rows
    assert r.sum_n3_before - r.sum_n3_after == gains
    assert _stopping_rule_violations(sp.nbf, r) == 0
    # the water molecules' three atoms share almost all rows: the metric falls noticeably
    assert r.sum_n3_before > 1.5 * r.sum_n3_after
    assert len(r.members) < n / 2


@pytest.mark.parametrize("mistake", ["squares", "no_common"])
def test_stopping_rule_catches_planted_mistakes(mistake, monkeypatch):
    sp = make_site_pattern(spec_ions_in_water_small())
    if mistake == "squares":
        monkeypatch.setattr(co, "criterion", lambda a, b, c: (a + b - c) ** 2 < a ** 2 + b ** 2)
    else:
        monkeypatch.setattr(co, "criterion", lambda a, b, c: (a + b) ** 3 < a ** 3 + b ** 3)
    r = co.combine(sp.nbf, sp.nb_ptr, sp.nb_idx)
    # squares merge too much (a logged merge fails the cube criterion on replay); without the common
    # rows nothing merges (pairs passing the criterion remain)
    try:
        _replay(sp.nbf, sp.nb_ptr, sp.nb_idx, r.merges)
        replay_ok = True
    except AssertionError:
        replay_ok = False
    assert not replay_ok or _stopping_rule_violations(sp.nbf, r) > 0


# ------------------------------------------------------------------ merged submatrices (the solve side)

def test_singleton_groups_reproduce_the_per_molecule_solve():
    sysm = make_system(SystemSpec(4, 4, 4, nbf="mixed", cutoff=4.5, seed=13))
    plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    ref = orc.solve(sysm, -0.8, plan=plan)
    g = co.solve_grouped(sysm, -0.8, list(range(sysm.n_mol)), plan)
    assert (g.D_vals == ref.D_vals).all()
    assert g.trace_DS == ref.trace_DS


@pytest.mark.parametrize("spec", [SystemSpec(4, 4, 4, seed=1001), SystemSpec(4, 4, 4, nbf="mixed", cutoff=4.5, seed=13)])
def test_one_group_gives_the_full_matrix_density(spec):
    """A group holding every molecule has the whole matrix as its submatrix: the written-back D is the
    S-orthogonal projector on the states below mu (LAPACK's generalized eigensolver) on D's pattern, and
    Tr(DS) is the number of those states."""
    sysm = make_system(spec)
    plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    S = orc.csr_to_dense(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
    H = orc.csr_to_dense(sysm.nbf, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
    eps, C = scipy.linalg.eigh(H, S)
    n_occ = int(sysm.n_occ)
    mu = 0.5 * (eps[n_occ - 1] + eps[n_occ])
    P = C[:, :n_occ] @ C[:, :n_occ].T
    g = co.solve_grouped(sysm, mu, [0] * sysm.n_mol, plan)
    D = orc.d_to_dense(plan, g.D_vals)
    mask = orc.d_to_dense(plan, np.ones_like(g.D_vals)) != 0
    assert np.max(np.abs((D - P)[mask])) < 1e-11
    assert np.all(D[~mask] == 0.0)
    assert g.trace_DS == pytest.approx(n_occ, abs=1e-9)
