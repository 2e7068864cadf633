"""Pins of the oracle's coupled Newton-Schulz inverse square root (Eqs. inv1-inv3) against the
mathematics: closed forms for diagonal matrices, the defining identity R S R = I with R symmetric, the
inverse from LAPACK (np.linalg.solve against the identity) and the inverse square root from LAPACK's
symmetric eigensolver on gathered overlap submatrices, and a planted mistake (Z dropped from V_k)."""
import numpy as np
import pytest

from oracle import inverse_oracle as inv
from oracle import nolsm_oracle as orc
from synth import make_system, spec_small_fp64, SystemSpec


def test_diagonal_closed_form():
    d = np.array([0.3, 0.9, 1.0, 1.7, 4.0])
    R, k, ok = inv.inverse_sqrt_ns(np.diag(d))
    assert ok
    assert np.max(np.abs(R - np.diag(1.0 / np.sqrt(d)))) < 1e-14


@pytest.mark.parametrize("spec", [spec_small_fp64(), SystemSpec(3, 3, 3, nbf="mixed", cutoff=4.5, seed=13)])
def test_overlap_submatrices(spec):
    sysm = make_system(spec)
    plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    for J in (0, sysm.n_mol // 2, sysm.n_mol - 1):
        S = orc.gather(plan, J, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
        R, k, ok = inv.inverse_sqrt_ns(S)
        assert ok and k < 60
        n = S.shape[0]
        assert np.max(np.abs(R - R.T)) < 1e-13
        assert np.max(np.abs(R @ S @ R - np.eye(n))) < 1e-12
        w, U = np.linalg.eigh(S)
        assert np.max(np.abs(R - (U / np.sqrt(w)) @ U.T)) < 1e-12
        Si, _, _ = inv.overlap_inverse_ns(S)
        assert np.max(np.abs(Si - np.linalg.solve(S, np.eye(n)))) < 1e-12


def test_planted_mistake_is_caught():
    sysm = make_system(spec_small_fp64())
    plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    S = orc.gather(plan, 7, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
    n = S.shape[0]
    c = float(np.max(np.sum(np.abs(S), axis=1)))
    Y, Z = S / c, np.eye(n)
    for _ in range(40):                   # V_k = Y_k instead of Z_k Y_k
        T = 3.0 * np.eye(n) - Y
        Y, Z = 0.5 * Y @ T, 0.5 * T @ Z
    R = Z / np.sqrt(c)
    assert np.max(np.abs(R @ S @ R - np.eye(n))) > 1e-3
