"""Coupled Newton-Schulz iteration for the inverse square root of the overlap submatrix, plain FP64 --
TEST INFRASTRUCTURE ONLY (same import rule as the rest of ``oracle/``).

Sec. "Efficient Iterative Matrix Function Solvers on GPU Tensor Cores", Eqs. inv1-inv3: with Y_0 = T_i(S),
Z_0 = I and V_k = Z_k Y_k,

    Y_{k+1} = 1/2 Y_k (3I - V_k),   Z_{k+1} = 1/2 (3I - V_k) Z_k,

Z_k tends to Y_0^{-1/2} and T_i(S)^{-1} = (Y_0^{-1/2})^2.

Readings (the section gives neither a scaling nor a stopping rule; it runs a fixed number of steps):
1. The iteration converges when the eigenvalues of Y_0 lie in (0, 2) (||I - Y_0|| < 1); the oracle starts
   from Y_0 = S / c with c = ||S||_inf (at least the largest eigenvalue of the symmetric positive definite S),
   so that the eigenvalues of Y_0 lie in (0, 1], and undoes the scale at the end:
   S^{-1/2} = Z / sqrt(c), S^{-1} = Z^2 / c.
2. The step whose input has ||I - V_k||_F / sqrt(n) <= tol is the last one (the same defect test as the
   sign iteration); ``max_iter`` caps the steps.
"""
from __future__ import annotations

import math

import numpy as np


def inverse_sqrt_ns(S: np.ndarray, tol: float = 1e-12, max_iter: int = 100):
    """(S^{-1/2}, steps, converged) by Eqs. inv1-inv2 on the scaled start of reading 1."""
    n = S.shape[0]
    c = float(np.max(np.sum(np.abs(S), axis=1)))
    I = np.eye(n)
    Y = S / c
    Z = I.copy()
    for k in range(1, max_iter + 1):
        V = Z @ Y
        defect = np.linalg.norm(I - V) / math.sqrt(n)
        T = 3.0 * I - V
        Y = 0.5 * (Y @ T)
        Z = 0.5 * (T @ Z)
        if defect <= tol:
            return Z / math.sqrt(c), k, True
    return Z / math.sqrt(c), max_iter, False


def overlap_inverse_ns(S: np.ndarray, tol: float = 1e-12, max_iter: int = 100):
    """(T_i(S)^{-1}, steps, converged) = (Y_0^{-1/2})^2 of Eq. inv3."""
    R, k, ok = inverse_sqrt_ns(S, tol, max_iter)
    return R @ R, k, ok
