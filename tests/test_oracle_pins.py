"""Pins of the FP64 oracle against results fixed by the mathematics, not by the oracle itself.

* closed forms: scalar Newton-Schulz, diagonal matrices, a two-level dimer, isolated molecules;
* the generalized symmetric eigenproblem H c = eps S c solved by LAPACK (a different algorithm from
  the oracle's inverse + sign iteration): T_J(D) = C_< C_<^T;
* a periodic cell that the cutoff spans entirely, where every submatrix is the whole matrix and the
  write-back must reproduce the full density matrix, which is then symmetric, idempotent in the S
  metric and has Tr(DS) equal to the number of states below mu;
* brute-force neighbour search and plain-loop index maps for the submatrix construction;
* planted mistakes (applied to a copy of the oracle on the CPU) that the pins must catch.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import nolsm_oracle as orc
from synth import SystemSpec, make_system, spec_small_fp64, spec_tiny


def gen_projector(S, H, mu):
    """C_< C_<^T from LAPACK's generalized symmetric eigensolver, with the states below mu."""
    eps, C = scipy.linalg.eigh(H, S)
    Cocc = C[:, eps < mu]
    return Cocc @ Cocc.T, eps


def mid_gap_mu(eps, n_occ):
    eps = np.sort(eps)
    return 0.5 * (eps[n_occ - 1] + eps[n_occ])


@pytest.fixture(scope="module")
def small():
    return make_system(spec_small_fp64())


@pytest.fixture(scope="module")
def small_aniso():
    return make_system(spec_small_fp64(aniso=0.3, cutoff_h=5.0, seed=11))


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("x", [1e-3, 0.1, 0.5, 1.0, 1.5, 1.7, -1e-3, -0.7, -1.69])
def test_scalar_newton_schulz_converges_to_sign(x):
    X, k, ok = orc.sign_newton_schulz(np.array([[x]]), alpha=1.0, tol=1e-12)
    assert ok
    assert X[0, 0] == pytest.approx(math.copysign(1.0, x), abs=1e-15)


def test_sign_of_diagonal_matrix():
    d = np.array([-2.0, -0.3, 0.01, 0.4, 3.0])
    X, k, ok = orc.sign_newton_schulz(np.diag(d), tol=1e-12)
    assert ok
    assert np.max(np.abs(X - np.diag(np.sign(d)))) < 1e-14


def test_dimer_closed_form():
    # two functions: S = [[1,s],[s,1]], H = [[e,h],[h,e]] with h < 0. Bonding state (1,1)/sqrt(2(1+s))
    # has eps = (e+h)/(1+s); with one state occupied D = [[1,1],[1,1]] / (2(1+s)).
    s, e, h = 0.2, -0.5, -0.3
    S = np.array([[1.0, s], [s, 1.0]])
    H = np.array([[e, h], [h, e]])
    eb, ea = (e + h) / (1 + s), (e - h) / (1 - s)
    mu = 0.5 * (eb + ea)
    r = orc.submatrix_density(S, H, mu, 0, 2, tol=1e-12)
    assert np.max(np.abs(r.D_sub - np.full((2, 2), 1.0 / (2 * (1 + s))))) < 1e-14
    assert r.t_S == pytest.approx(1.0, abs=1e-14)
    assert r.t_H == pytest.approx(eb, abs=1e-14)


def test_identity_overlap_gives_ordinary_projector():
    rng = np.random.default_rng(3)
    M = rng.normal(size=(40, 40))
    H = 0.5 * (M + M.T)
    w, V = np.linalg.eigh(H)
    mu = 0.5 * (w[17] + w[18])
    r = orc.submatrix_density(np.eye(40), H, mu, 0, 40, tol=1e-12)
    P = V[:, :18] @ V[:, :18].T
    assert np.max(np.abs(r.D_sub - P)) < 1e-11


def test_isolated_molecules_give_step_function():
    # cutoff below the smallest spacing: N(J) = {J}, T_J(S) = I, T_J(H) = diag(on-site)
    sysm = make_system(SystemSpec(3, 3, 3, cutoff=1.5, seed=5))
    res = orc.solve(sysm, mu=-0.2, tol=1e-12)
    for J, r in res.subs.items():
        expect = np.diag((sysm.onsite[J] < -0.2).astype(float))
        assert np.array_equal(np.asarray(r.D_sub.shape), [6, 6])
        assert np.max(np.abs(r.D_sub - expect)) < 1e-14
    assert res.trace_DS == pytest.approx(4 * 27, abs=1e-12)


# ------------------------------------------------------------------ generalized eigenproblem

def test_submatrices_match_generalized_eigenproblem(small, small_aniso):
    for sysm in (small, small_aniso):
        plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
        for J in (0, 17, 63):
            S = orc.gather(plan, J, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
            H = orc.gather(plan, J, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
            eps = scipy.linalg.eigh(H, S, eigvals_only=True)
            n_occ = 4 * (plan.nb_ptr[J + 1] - plan.nb_ptr[J])
            mu = mid_gap_mu(eps, n_occ)
            r = orc.submatrix_density(S, H, mu, int(plan.sub_c0[J]), 6)
            P, _ = gen_projector(S, H, mu)
            assert r.converged
            assert np.max(np.abs(r.D_sub - P)) < 1e-11
            # projector algebra holds exactly for every submatrix
            assert np.max(np.abs(r.D_sub @ S @ r.D_sub - r.D_sub)) < 1e-11
            assert np.max(np.abs(r.D_sub - r.D_sub.T)) < 1e-11
            assert np.trace(r.D_sub @ S) == pytest.approx(int(np.sum(eps < mu)), abs=1e-10)


def test_inverse_is_an_inverse(small):
    plan = orc.build_plan(small.nbf, small.S.row_ptr, small.S.col_idx, small.H.row_ptr, small.H.col_idx)
    S = orc.gather(plan, 5, small.S.row_ptr, small.S.col_idx, small.S.blk_off, small.S.vals)
    Si = orc.overlap_inverse(S)
    assert np.max(np.abs(S @ Si - np.eye(S.shape[0]))) < 1e-13


# ------------------------------------------------------------------ whole cell

@pytest.mark.parametrize("aniso", [0.0, 0.35])
def test_whole_cell_reproduces_full_density_matrix(aniso):
    sysm = make_system(spec_tiny(2, aniso=aniso))
    n_mol = sysm.n_mol
    S = orc.csr_to_dense(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
    H = orc.csr_to_dense(sysm.nbf, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
    # the cutoff spans the cell: every block is stored
    assert sysm.S.nnzb == n_mol * n_mol
    eps = scipy.linalg.eigh(H, S, eigvals_only=True)
    n_occ = int(sysm.n_occ)
    mu = mid_gap_mu(eps, n_occ)
    res = orc.solve(sysm, mu, tol=1e-12)
    D = orc.d_to_dense(res.plan, res.D_vals)
    P, _ = gen_projector(S, H, mu)
    assert np.max(np.abs(D - P)) < 1e-11
    assert np.max(np.abs(D - D.T)) < 1e-11
    assert np.max(np.abs(D @ S @ D - D)) < 1e-11
    assert res.trace_DS == pytest.approx(n_occ, abs=1e-10)
    assert res.trace_DH == pytest.approx(float(np.sum(np.sort(eps)[:n_occ])), abs=1e-10)


# ------------------------------------------------------------------ submatrix construction

def test_pattern_matches_brute_force_neighbours(small_aniso):
    sysm = small_aniso
    pairs_s = set(orc.brute_force_pairs(sysm.pos, sysm.cell, sysm.spec.cutoff))
    pairs_h = set(orc.brute_force_pairs(sysm.pos, sysm.cell, sysm.spec.cutoff_h))
    got_s = {(I, int(J)) for I in range(sysm.n_mol)
             for J in sysm.S.col_idx[sysm.S.row_ptr[I]:sysm.S.row_ptr[I + 1]]}
    got_h = {(I, int(J)) for I in range(sysm.n_mol)
             for J in sysm.H.col_idx[sysm.H.row_ptr[I]:sysm.H.row_ptr[I + 1]]}
    assert got_s == pairs_s
    assert got_h == pairs_h
    assert pairs_h < pairs_s      # the shorter H cutoff stores fewer blocks


def test_plan_index_maps_by_plain_loops():
    sysm = make_system(SystemSpec(3, 3, 3, nbf="mixed", cutoff=4.0, cutoff_h=5.0, seed=21))
    plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    n = sysm.n_mol
    dist2 = lambda I, J: float(np.sum(((sysm.pos[J] - sysm.pos[I]) - sysm.cell *
                                       np.rint((sysm.pos[J] - sysm.pos[I]) / sysm.cell)) ** 2))
    for J in range(n):
        expect = [I for I in range(n) if dist2(I, J) < 5.0 ** 2]   # merged pattern = the longer cutoff
        got = list(plan.nb_idx[plan.nb_ptr[J]:plan.nb_ptr[J + 1]])
        assert got == expect
        offs = np.concatenate([[0], np.cumsum([sysm.nbf[I] for I in expect])])
        assert list(plan.nb_off[plan.nb_ptr[J]:plan.nb_ptr[J + 1]]) == list(offs[:-1])
        assert plan.sub_n[J] == offs[-1]
        assert plan.sub_c0[J] == offs[expect.index(J)]


def test_gather_places_blocks_by_hand(small_aniso):
    sysm = small_aniso
    plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    full = orc.csr_to_dense(sysm.nbf, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
    J = 9
    T = orc.gather(plan, J, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
    rows = np.concatenate([np.arange(6 * I, 6 * I + 6) for I in plan.nb_idx[plan.nb_ptr[J]:plan.nb_ptr[J + 1]]])
    assert np.array_equal(T, full[np.ix_(rows, rows)])
    assert np.max(np.abs(T - T.T)) == 0.0


# ------------------------------------------------------------------ chemical potential

def test_electron_count_is_monotone_with_a_plateau(small):
    plan = orc.build_plan(small.nbf, small.S.row_ptr, small.S.col_idx, small.H.row_ptr, small.H.col_idx)
    subs = list(range(0, 64, 7))
    mus = np.linspace(-0.6, 0.3, 10)
    counts = [orc.solve(small, mu, subs=subs, plan=plan).trace_DS for mu in mus]
    assert all(b >= a - 1e-9 for a, b in zip(counts, counts[1:]))


def test_find_mu_lands_in_the_gap_whole_cell():
    sysm = make_system(spec_tiny(2))
    S = orc.csr_to_dense(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
    H = orc.csr_to_dense(sysm.nbf, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
    eps = np.sort(scipy.linalg.eigh(H, S, eigvals_only=True))
    n_occ = int(sysm.n_occ)
    plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    res = orc.find_mu(lambda mu: orc.solve(sysm, mu, plan=plan, tol=1e-12).trace_DS, n_occ,
                      -3.0, 3.0, tol_n=1e-6)
    assert res.ok
    assert eps[n_occ - 1] < res.mu < eps[n_occ]
    # on the plateau the count is the integer number of states below mu
    assert res.trace_DS == pytest.approx(n_occ, abs=1e-9)
    for mu, f in res.history[:-1]:
        assert (f < 0) == (mu < eps[n_occ - 1]) or abs(f) < 1e-9


# ------------------------------------------------------------------ planted mistakes

def _eig_pin_error(S, H, mu, sub_fn):
    P, _ = gen_projector(S, H, mu)
    r = sub_fn(S, H, mu)
    return np.max(np.abs(r - P))


@pytest.mark.parametrize("mistake", ["drop_inverse", "transpose_product", "wrong_sign", "drop_mu",
                                     "wrong_half", "transpose_gather"])
def test_pins_catch_planted_mistakes(mistake, small_aniso):
    sysm = small_aniso
    plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    J = 3
    S = orc.gather(plan, J, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
    H = orc.gather(plan, J, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
    eps = scipy.linalg.eigh(H, S, eigvals_only=True)
    # a mu inside the occupied band (0 lies in the gap, where dropping mu would go unnoticed)
    mu = mid_gap_mu(eps, 4 * (plan.nb_ptr[J + 1] - plan.nb_ptr[J]) - 17)
    assert mu < -0.2
    n = S.shape[0]
    I = np.eye(n)

    def mutated(S, H, mu):
        Si = np.linalg.inv(S)
        if mistake == "drop_inverse":
            A = H - mu * I
        elif mistake == "transpose_product":
            A = H @ Si - mu * I
        elif mistake == "drop_mu":
            A = Si @ H
        elif mistake == "transpose_gather":
            # every 6x6 block read transposed (column-major instead of row-major)
            Ht = H.reshape(n // 6, 6, n // 6, 6).transpose(0, 3, 2, 1).reshape(n, n)
            A = Si @ Ht - mu * I
        else:
            A = Si @ H - mu * I
        X, _, _ = orc.sign_newton_schulz(A)
        if mistake == "wrong_sign":
            return 0.5 * (I + X) @ Si
        if mistake == "wrong_half":
            return (I - X) @ Si
        if mistake == "drop_inverse":
            return 0.5 * (I - X)
        return 0.5 * (I - X) @ Si

    def correct(S, H, mu):
        return orc.submatrix_density(S, H, mu, 0, n).D_sub

    assert _eig_pin_error(S, H, mu, correct) < 1e-11
    assert _eig_pin_error(S, H, mu, mutated) > 1e-3


def test_whole_cell_pin_catches_transposed_write_back(monkeypatch):
    sysm = make_system(spec_tiny(2, aniso=0.35))
    S = orc.csr_to_dense(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
    H = orc.csr_to_dense(sysm.nbf, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
    eps = scipy.linalg.eigh(H, S, eigvals_only=True)
    mu = mid_gap_mu(eps, int(sysm.n_occ))
    P, _ = gen_projector(S, H, mu)
    real = orc.write_back

    def transposed(plan, subs):
        D = real(plan, subs)
        off = orc.d_block_offsets(plan)
        for q in range(off.shape[0] - 1):
            D[off[q]:off[q + 1]] = D[off[q]:off[q + 1]].reshape(6, 6).T.reshape(-1)
        return D

    monkeypatch.setattr(orc, "write_back", transposed)
    res = orc.solve(sysm, mu, tol=1e-12)
    assert np.max(np.abs(orc.d_to_dense(res.plan, res.D_vals) - P)) > 1e-3
