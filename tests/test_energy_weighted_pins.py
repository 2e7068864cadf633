"""Pins of the oracle's energy-weighted density matrix W = D H0 D (NOLSM section; submatrix form
T_J(W) = T_J(D) T_J(H0) T_J(D)) against results the mathematics fixes, not the oracle itself:

* the generalized symmetric eigenproblem H c = eps S c (LAPACK): W = C_< diag(eps_<) C_<^T, and
  Tr(W S) = the sum of the eigenvalues below mu;
* a two-level dimer in closed form (W = eps_bonding D);
* a periodic cell that the cutoff spans, where the written-back W is the full matrix's W;
* the form the GPU library evaluates, W_c = T_J(S)^-1 T_J(H0) D_c (the projector 1/2 (I - sign)
  commutes with T_J(S)^-1 T_J(H0) and is idempotent), checked here against the definition;
* planted mistakes in a copy of the product on the CPU, which the eigenproblem pin must catch.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import nolsm_oracle as orc
from synth import make_system, spec_small_fp64, spec_tiny


def gen_weighted(S, H, mu):
    eps, C = scipy.linalg.eigh(H, S)
    occ = eps < mu
    return (C[:, occ] * eps[occ]) @ C[:, occ].T, eps


def mid_gap_mu(eps, n_occ):
    eps = np.sort(eps)
    return 0.5 * (eps[n_occ - 1] + eps[n_occ])


@pytest.fixture(scope="module")
def small_aniso():
    return make_system(spec_small_fp64(aniso=0.3, cutoff_h=5.0, seed=11))


def _sub(sysm, plan, J):
    S = orc.gather(plan, J, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
    H = orc.gather(plan, J, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
    return S, H


def test_dimer_closed_form():
    # S = [[1,s],[s,1]], H = [[e,h],[h,e]], bonding state occupied: D = [[1,1],[1,1]] / (2(1+s)) and
    # W = D H D = eps_b D with eps_b = (e+h)/(1+s)
    s, e, h = 0.2, -0.5, -0.3
    S = np.array([[1.0, s], [s, 1.0]])
    H = np.array([[e, h], [h, e]])
    eb, ea = (e + h) / (1 + s), (e - h) / (1 - s)
    r = orc.submatrix_density(S, H, 0.5 * (eb + ea), 0, 2, tol=1e-12)
    W = orc.submatrix_energy_weighted(r.D_sub, H)
    assert np.max(np.abs(W - eb * np.full((2, 2), 1.0 / (2 * (1 + s))))) < 1e-14


def test_submatrices_match_generalized_eigenproblem(small_aniso):
    sysm = small_aniso
    plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    for J in (0, 17, 63):
        S, H = _sub(sysm, plan, J)
        eps = scipy.linalg.eigh(H, S, eigvals_only=True)
        mu = mid_gap_mu(eps, 4 * (plan.nb_ptr[J + 1] - plan.nb_ptr[J]))
        r = orc.submatrix_density(S, H, mu, int(plan.sub_c0[J]), 6)
        W = orc.submatrix_energy_weighted(r.D_sub, H)
        Wref, _ = gen_weighted(S, H, mu)
        assert np.max(np.abs(W - Wref)) < 1e-11
        assert np.max(np.abs(W - W.T)) < 1e-11
        assert np.trace(W @ S) == pytest.approx(float(np.sum(eps[eps < mu])), abs=1e-10)


def test_energy_weighted_traces_and_columns(small_aniso):
    sysm = small_aniso
    plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    subs = [2, 40]
    res = orc.solve(sysm, -0.1, subs=subs, plan=plan)
    w = orc.energy_weighted(sysm, res)
    assert w.W_vals is None
    for J in subs:
        S, H = _sub(sysm, plan, J)
        Wref, _ = gen_weighted(S, H, -0.1)
        c0 = int(plan.sub_c0[J])
        assert np.max(np.abs(w.W_cols[J] - Wref[:, c0:c0 + 6])) < 1e-11
        assert w.t_S[J] == pytest.approx(float(np.sum(Wref[:, c0:c0 + 6] * S[:, c0:c0 + 6])), abs=1e-11)
    assert w.trace_WS == pytest.approx(sum(w.t_S.values()), abs=1e-13)


@pytest.mark.parametrize("aniso", [0.0, 0.35])
def test_whole_cell_reproduces_full_energy_weighted_matrix(aniso):
    sysm = make_system(spec_tiny(2, aniso=aniso))
    S = orc.csr_to_dense(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
    H = orc.csr_to_dense(sysm.nbf, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
    assert sysm.S.nnzb == sysm.n_mol ** 2
    eps = scipy.linalg.eigh(H, S, eigvals_only=True)
    n_occ = int(sysm.n_occ)
    mu = mid_gap_mu(eps, n_occ)
    res = orc.solve(sysm, mu, tol=1e-12)
    w = orc.energy_weighted(sysm, res)
    Wd = orc.d_to_dense(res.plan, w.W_vals)
    Wref, _ = gen_weighted(S, H, mu)
    assert np.max(np.abs(Wd - Wref)) < 1e-11
    # Tr(W S) = E_elec = Tr(D H0) = sum of the occupied eigenvalues
    assert w.trace_WS == pytest.approx(float(np.sum(np.sort(eps)[:n_occ])), abs=1e-10)
    assert w.trace_WS == pytest.approx(res.trace_DH, abs=1e-10)


def test_product_form_of_the_library_matches_the_definition(small_aniso):
    """W_c = A_J D_c with A_J = T_J(S)^-1 T_J(H0): P = 1/2 (I - sign(A_J - mu I)) commutes with A_J and
    P^2 = P, so D H D = P A_J P T_J(S)^-1 = A_J P T_J(S)^-1 = A_J D (at the converged sign)."""
    sysm = small_aniso
    plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    for J, mu in ((5, -0.1), (30, -0.4)):
        S, H = _sub(sysm, plan, J)
        c0 = int(plan.sub_c0[J])
        r = orc.submatrix_density(S, H, mu, c0, 6)
        W = orc.submatrix_energy_weighted(r.D_sub, H)
        A = orc.overlap_inverse(S) @ H
        assert np.max(np.abs(A @ r.D_cols - W[:, c0:c0 + 6])) < 1e-11


@pytest.mark.parametrize("mistake", ["drop_right_D", "overlap_for_H", "shifted_H"])
def test_pins_catch_planted_mistakes(mistake, small_aniso):
    sysm = small_aniso
    plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    J = 3
    S, H = _sub(sysm, plan, J)
    eps = scipy.linalg.eigh(H, S, eigvals_only=True)
    mu = mid_gap_mu(eps, 4 * (plan.nb_ptr[J + 1] - plan.nb_ptr[J]) - 17)
    r = orc.submatrix_density(S, H, mu, 0, S.shape[0])
    D = r.D_sub
    if mistake == "drop_right_D":
        W = D @ H
    elif mistake == "overlap_for_H":
        W = D @ S @ D
    else:                     # the shifted matrix of the sign iteration reused: W - mu D
        W = D @ (H - mu * S) @ D
    Wref, _ = gen_weighted(S, H, mu)
    assert np.max(np.abs(orc.submatrix_energy_weighted(D, H) - Wref)) < 1e-11
    assert np.max(np.abs(W - Wref)) > 1e-3
