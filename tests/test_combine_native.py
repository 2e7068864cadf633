"""The library's combination heuristic (nolsm_combine_submatrices, host code behind the C ABI; no GPU)
against the plain oracle: group assignments, group counts, sweeps and the cubic and quadratic metrics
must be identical (integer work). Also: the result does not depend on the number of threads, and a
malformed pattern is rejected."""
import numpy as np
import pytest

from oracle import combine_oracle as co
from oracle import nolsm_oracle as orc
from synth import (SystemSpec, make_site_pattern, make_system, spec_ions_in_water, spec_ions_in_water_small,
                   spec_small_fp64, spec_tiny)


@pytest.fixture(scope="module")
def nl():
    from paper_2104_08245_gb300 import build
    build.build()
    import paper_2104_08245_gb300 as nl
    return nl


def _sys_pattern(spec):
    s = make_system(spec)
    p = orc.build_plan(s.nbf, s.S.row_ptr, s.S.col_idx, s.H.row_ptr, s.H.col_idx)
    return p.nbf, p.nb_ptr, p.nb_idx


def _site_pattern(spec):
    sp = make_site_pattern(spec)
    return sp.nbf, sp.nb_ptr, sp.nb_idx


CASES = {
    "empty": lambda: (np.zeros(0, dtype=np.int32), np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32)),
    "one_molecule": lambda: (np.array([5]), np.array([0, 1]), np.array([0])),
    "chain": lambda: (np.array([1, 1, 1]), np.array([0, 2, 5, 7]), np.array([0, 1, 0, 1, 2, 1, 2])),
    "whole_cell": lambda: _sys_pattern(spec_tiny(2)),
    "isolated": lambda: _sys_pattern(SystemSpec(3, 3, 2, cutoff=1.5, seed=14)),
    "water_64": lambda: _sys_pattern(spec_small_fp64()),
    "mixed_6_23": lambda: _sys_pattern(SystemSpec(4, 4, 4, nbf="mixed", cutoff=4.5, seed=13)),
    "ions_in_water_632_sites": lambda: _site_pattern(spec_ions_in_water_small()),
    "ions_dense": lambda: _site_pattern(spec_ions_in_water_small(ion_fraction=0.2, seed=1303)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_native_matches_oracle(nl, name):
    nbf, nb_ptr, nb_idx = CASES[name]()
    ref = co.combine(nbf, nb_ptr, nb_idx)
    got = nl.nolsm_combine_submatrices(nbf, nb_ptr, nb_idx)
    assert np.array_equal(got.group_of, ref.group_of)
    assert got.n_groups == len(ref.members)
    assert got.sweeps == ref.sweeps
    assert (got.sum_n3_before, got.sum_n3_after) == (float(ref.sum_n3_before), float(ref.sum_n3_after))
    assert (got.sum_n2_before, got.sum_n2_after) == (float(ref.sum_n2_before), float(ref.sum_n2_after))


def test_threads_do_not_change_the_result(nl):
    nbf, nb_ptr, nb_idx = _site_pattern(spec_ions_in_water())      # about 12,000 atom sites
    one = nl.nolsm_combine_submatrices(nbf, nb_ptr, nb_idx, threads=1)
    many = nl.nolsm_combine_submatrices(nbf, nb_ptr, nb_idx, threads=8)
    assert np.array_equal(one.group_of, many.group_of) and one.sweeps == many.sweeps
    assert one.sum_n3_after == many.sum_n3_after
    # every group is named by its smallest member, and the metric fell
    g = one.group_of
    assert np.all(g <= np.arange(g.shape[0])) and np.all(g[g] == g)
    assert one.n_groups == np.unique(g).shape[0]
    assert one.sum_n3_after < one.sum_n3_before


@pytest.mark.parametrize("bad", ["unsorted", "no_self", "asymmetric", "out_of_range", "zero_nbf"])
def test_malformed_pattern_is_rejected(nl, bad):
    nbf = np.array([1, 1, 1])
    nb_ptr = np.array([0, 2, 5, 7])
    nb_idx = np.array([0, 1, 0, 1, 2, 1, 2])
    if bad == "unsorted":
        nb_idx = np.array([1, 0, 0, 1, 2, 1, 2])
    elif bad == "no_self":
        nb_ptr, nb_idx = np.array([0, 1, 4, 6]), np.array([1, 0, 1, 2, 1, 2])
    elif bad == "asymmetric":
        nb_ptr, nb_idx = np.array([0, 2, 4, 6]), np.array([0, 1, 0, 1, 1, 2])
    elif bad == "out_of_range":
        nb_idx = np.array([0, 1, 0, 1, 3, 1, 2])
    else:
        nbf = np.array([1, 0, 1])
    with pytest.raises(nl.NolsmError) as e:
        nl.nolsm_combine_submatrices(nbf, nb_ptr, nb_idx)
    assert e.value.status == 1          # NOLSM_ERR_ARG


def _random_pattern(rng, n, p, max_b):
    adj = rng.random((n, n)) < p
    adj = adj | adj.T
    np.fill_diagonal(adj, True)
    nb_ptr = np.concatenate([[0], np.cumsum(adj.sum(axis=0))]).astype(np.int32)
    nb_idx = np.concatenate([np.nonzero(adj[:, J])[0] for J in range(n)]).astype(np.int32)
    nbf = rng.integers(1, max_b + 1, size=n).astype(np.int32)
    return nbf, nb_ptr, nb_idx


@pytest.mark.parametrize("seed", range(12))
def test_native_matches_oracle_on_random_patterns(nl, seed):
    """Random symmetric patterns (any degree, 1..9 functions per molecule), including dense and almost
    empty ones: the same groups, sweeps and metrics as the oracle."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 60))
    p = float(rng.choice([0.02, 0.1, 0.3, 0.8]))
    nbf, nb_ptr, nb_idx = _random_pattern(rng, n, p, 9)
    ref = co.combine(nbf, nb_ptr, nb_idx)
    got = nl.nolsm_combine_submatrices(nbf, nb_ptr, nb_idx, threads=int(rng.integers(1, 5)))
    assert np.array_equal(got.group_of, ref.group_of)
    assert got.sweeps == ref.sweeps and got.n_groups == len(ref.members)
    assert (got.sum_n3_before, got.sum_n3_after) == (float(ref.sum_n3_before), float(ref.sum_n3_after))
