"""FP64 CPU oracle of the NOLSM hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import or
run this module. The GPU library never calls it and shares no code with it; the only thing both sides
use is the seeded input generator in ``synth/``.

Every function is a plain, slow restatement of one step of the non-orthogonalised local submatrix
method (NOLSM) in float64, in the order the paper gives the steps:

* submatrix construction over the merged sparsity pattern of H0 and S  (Sec. "The Non-Orthogonal
  Local Submatrix Method", merged pattern; Sec. "The Submatrix Method", step (i));
* the overlap-submatrix inverse T_J(S)^-1                                  (Eq. purification_submatrix);
* spectral rescaling followed by the Newton-Schulz sign iteration
  X_{k+1} = 1/2 X_k (3I - X_k^2)                                           (Eq. NS1, NS2);
* T_J(D) = 1/2 (I - sign(T_J(S)^-1 T_J(H0) - mu I)) T_J(S)^-1              (Eq. purification_submatrix);
* write-back of the centre molecule's columns into the sparse D            (Sec. "The Submatrix
  Method", step (iii); columns of one molecule coalesced, Sec. "Simulation Details");
* E_elec = Tr(D H0) = sum_ij D_ij H0_ji and the electron count Tr(D S)     (Eq. e_elec);
* the energy-weighted density matrix W = D H0 D, in submatrix form
  T_J(W) = T_J(D) T_J(H0) T_J(D), its centre columns written back like D  (NOLSM section, the
  equation after Eq. e_elec and its submatrix form after Eq. purification_submatrix);
* the chemical potential by bisection on the electron count               (Sec. "Simulation Details").

Readings of points the paper leaves open (each one also listed in the design notes):

1. Scaling norm (the paper says only that the matrix is rescaled): alpha = ||A||_inf, the maximum
   absolute row sum, which bounds the spectral radius, so the scaled spectrum lies in [-1, 1].
2. Stopping rule (the paper runs a fixed, unstated number of steps): the step X_k -> X_{k+1} is the
   last one when the defect ||I - X_k^2||_F / sqrt(n) <= tol; quadratic convergence then leaves
   X_{k+1} within about tol^2 of the sign. Cap: ``max_iter`` steps.
3. Electron count: Eq. purification has no spin factor, so Tr(DS) counts occupied orbitals.
4. mu rule ("bisection-like"): plain bisection on f(mu) = Tr(DS) - N_occ from the caller's bracket;
   f < 0 raises lo, otherwise lowers hi; stop at the first |f| <= tol_n, or when hi - lo <= tol_mu,
   or after max_steps evaluations.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np


# ============================================================================ submatrix construction

@dataclasses.dataclass
class OraclePlan:
    """Integer maps of the submatrix construction (one submatrix per molecule J)."""
    nb_ptr: np.ndarray    # int32 [n_mol+1]; molecules of N(J) are nb_idx[nb_ptr[J]:nb_ptr[J+1]]
    nb_idx: np.ndarray    # int32; sorted ascending within each J
    nb_off: np.ndarray    # int32; local row offset of each molecule of N(J) inside T_J
    sub_n: np.ndarray     # int32 [n_mol]; submatrix dimension n_J
    sub_c0: np.ndarray    # int32 [n_mol]; local offset of J's own (centre) columns inside T_J
    nbf: np.ndarray       # int32 [n_mol]


def block_columns(n_mol: int, row_ptr: np.ndarray, col_idx: np.ndarray) -> list:
    """For every block column J, the set of block rows I holding a stored block (I, J)."""
    cols = [set() for _ in range(n_mol)]
    for I in range(n_mol):
        for p in range(int(row_ptr[I]), int(row_ptr[I + 1])):
            cols[int(col_idx[p])].add(I)
    return cols


def build_plan(nbf, S_row_ptr, S_col, H_row_ptr, H_col) -> OraclePlan:
    """Merged pattern: row I belongs to the submatrix of column J if S_IJ != 0 or H0_IJ != 0
    (Sec. "The Non-Orthogonal Local Submatrix Method"); all columns of molecule J share one
    submatrix (Sec. "Simulation Details"). Rows are ordered by molecule index, then function index."""
    nbf = np.asarray(nbf, dtype=np.int64)
    n_mol = nbf.shape[0]
    cs = block_columns(n_mol, S_row_ptr, S_col)
    ch = block_columns(n_mol, H_row_ptr, H_col)
    nb_ptr = [0]
    nb_idx, nb_off, sub_n, sub_c0 = [], [], [], []
    for J in range(n_mol):
        rows = sorted(cs[J] | ch[J])
        off = 0
        c0 = -1
        for I in rows:
            if I == J:
                c0 = off
            nb_idx.append(I)
            nb_off.append(off)
            off += int(nbf[I])
        nb_ptr.append(len(nb_idx))
        sub_n.append(off)
        sub_c0.append(c0)
    i32 = lambda v: np.asarray(v, dtype=np.int32)
    return OraclePlan(i32(nb_ptr), i32(nb_idx), i32(nb_off), i32(sub_n), i32(sub_c0), i32(nbf))


def _block(row_ptr, col_idx, blk_off, vals, nbf, I, K):
    """Stored block (I, K) as a dense b_I x b_K array, or None when the block is absent."""
    for p in range(int(row_ptr[I]), int(row_ptr[I + 1])):
        if int(col_idx[p]) == K:
            return vals[int(blk_off[p]):int(blk_off[p + 1])].reshape(int(nbf[I]), int(nbf[K]))
    return None


def gather(plan: OraclePlan, J: int, row_ptr, col_idx, blk_off, vals) -> np.ndarray:
    """T_J(M): keep the rows and columns of M that belong to N(J) (Sec. "The Submatrix Method",
    step (i)); positions without a stored block are zero."""
    lo, hi = int(plan.nb_ptr[J]), int(plan.nb_ptr[J + 1])
    mols = plan.nb_idx[lo:hi]
    offs = plan.nb_off[lo:hi]
    n = int(plan.sub_n[J])
    T = np.zeros((n, n), dtype=np.float64)
    for a, I in enumerate(mols):
        for c, K in enumerate(mols):
            blk = _block(row_ptr, col_idx, blk_off, vals, plan.nbf, int(I), int(K))
            if blk is not None:
                T[offs[a]:offs[a] + blk.shape[0], offs[c]:offs[c] + blk.shape[1]] = blk
    return T


# ============================================================================ dense matrix function

def overlap_inverse(S_sub: np.ndarray) -> np.ndarray:
    """T_J(S)^-1 (Eq. purification_submatrix), by an LAPACK solve against the identity."""
    return np.linalg.solve(S_sub, np.eye(S_sub.shape[0]))


def spectral_scale(A: np.ndarray) -> float:
    """alpha = ||A||_inf >= spectral radius of A (reading 1 of the module docstring)."""
    return float(np.max(np.sum(np.abs(A), axis=1)))


def sign_newton_schulz(A: np.ndarray, alpha: Optional[float] = None, tol: float = 1e-9,
                       max_iter: int = 100):
    """sign(A) by X_0 = A/alpha, X_{k+1} = 1/2 X_k (3I - X_k^2) (Eq. NS1, NS2).

    Returns (X, steps, converged). Stopping rule: reading 2 of the module docstring."""
    n = A.shape[0]
    if alpha is None:
        alpha = spectral_scale(A)
    I = np.eye(n)
    X = A / alpha
    for k in range(1, max_iter + 1):
        X2 = X @ X
        defect = np.linalg.norm(I - X2) / math.sqrt(n)
        X = 0.5 * (X @ (3.0 * I - X2))
        if defect <= tol:
            return X, k, True
    return X, max_iter, False


@dataclasses.dataclass
class SubResult:
    D_sub: np.ndarray      # full T_J(D), n_J x n_J
    D_cols: np.ndarray     # centre columns T_J(D)[:, c0:c0+b_J]
    t_S: float             # sum over centre columns j and rows i of T_J(D)_ij T_J(S)_ij
    t_H: float             # same with T_J(H0)
    steps: int
    converged: bool
    alpha: float


def submatrix_density(S_sub, H_sub, mu, c0, b, tol=1e-9, max_iter=100, alpha=None) -> SubResult:
    """T_J(D) = 1/2 (I - sign(T_J(S)^-1 T_J(H0) - mu I)) T_J(S)^-1 (Eq. purification_submatrix),
    its centre columns, and their contributions to Tr(D S) and Tr(D H0) (Eq. e_elec)."""
    n = S_sub.shape[0]
    Sinv = overlap_inverse(S_sub)
    A = Sinv @ H_sub - mu * np.eye(n)
    if alpha is None:
        alpha = spectral_scale(A)
    X, steps, ok = sign_newton_schulz(A, alpha, tol, max_iter)
    D = 0.5 * (np.eye(n) - X) @ Sinv
    cols = D[:, c0:c0 + b]
    t_S = 0.0
    t_H = 0.0
    for j in range(c0, c0 + b):
        for i in range(n):
            t_S += D[i, j] * S_sub[i, j]
            t_H += D[i, j] * H_sub[i, j]
    return SubResult(D, cols.copy(), t_S, t_H, steps, ok, alpha)


# ============================================================================ whole system

@dataclasses.dataclass
class OracleResult:
    plan: OraclePlan
    subs: dict             # J -> SubResult
    trace_DS: float
    trace_DH: float
    D_vals: Optional[np.ndarray]   # D in the merged pattern (block row I = N(I)), or None for a subset


def solve(system, mu: float, subs: Optional[Sequence[int]] = None, tol: float = 1e-9,
          max_iter: int = 100, plan: Optional[OraclePlan] = None) -> OracleResult:
    """Every submatrix (or the listed ones) at chemical potential mu, then the write-back."""
    if plan is None:
        plan = build_plan(system.nbf, system.S.row_ptr, system.S.col_idx,
                          system.H.row_ptr, system.H.col_idx)
    n_mol = plan.nbf.shape[0]
    todo = range(n_mol) if subs is None else [int(j) for j in subs]
    out = {}
    tS = 0.0
    tH = 0.0
    for J in todo:
        S_sub = gather(plan, J, system.S.row_ptr, system.S.col_idx, system.S.blk_off, system.S.vals)
        H_sub = gather(plan, J, system.H.row_ptr, system.H.col_idx, system.H.blk_off, system.H.vals)
        r = submatrix_density(S_sub, H_sub, mu, int(plan.sub_c0[J]), int(plan.nbf[J]), tol, max_iter)
        out[J] = r
        tS += r.t_S
        tH += r.t_H
    D_vals = write_back(plan, out) if subs is None else None
    return OracleResult(plan, out, tS, tH, D_vals)


@dataclasses.dataclass
class WResult:
    W_cols: dict           # J -> centre columns of T_J(W), n_J x b_J
    t_S: dict              # J -> sum over centre columns j and rows i of T_J(W)_ij T_J(S)_ij
    trace_WS: float        # sum of t_S over the submatrices
    W_vals: Optional[np.ndarray]   # W in the merged pattern of D, or None for a subset


def submatrix_energy_weighted(D_sub: np.ndarray, H_sub: np.ndarray) -> np.ndarray:
    """T_J(W) = T_J(D) T_J(H0) T_J(D) (NOLSM section, energy-weighted density matrix in submatrix
    form), as the two products the definition names."""
    return (D_sub @ H_sub) @ D_sub


def energy_weighted(system, res: OracleResult) -> WResult:
    """T_J(W) of every submatrix of an oracle solve, from its full T_J(D); the centre columns are
    written back into the merged pattern as for D (when ``res`` covers the whole system).
    Tr(W S) = Tr(D H0 D S) = Tr(D H0) for the full matrices when D S D = D, so the traces sum to an
    approximation of E_elec (Eq. e_elec)."""
    plan = res.plan
    cols, tS = {}, {}
    total = 0.0
    for J, r in res.subs.items():
        S_sub = gather(plan, J, system.S.row_ptr, system.S.col_idx, system.S.blk_off, system.S.vals)
        H_sub = gather(plan, J, system.H.row_ptr, system.H.col_idx, system.H.blk_off, system.H.vals)
        W = submatrix_energy_weighted(r.D_sub, H_sub)
        c0, b = int(plan.sub_c0[J]), int(plan.nbf[J])
        cols[J] = W[:, c0:c0 + b].copy()
        t = 0.0
        for j in range(c0, c0 + b):
            for i in range(W.shape[0]):
                t += W[i, j] * S_sub[i, j]
        tS[J] = t
        total += t
    W_vals = write_back_cols(plan, cols) if res.D_vals is not None else None
    return WResult(cols, tS, total, W_vals)


def d_block_offsets(plan: OraclePlan) -> np.ndarray:
    """Element offsets of the blocks of D stored in the merged pattern, block row I = N(I) in order,
    block (I, J) b_I x b_J row-major."""
    offs = [0]
    for I in range(plan.nbf.shape[0]):
        for p in range(int(plan.nb_ptr[I]), int(plan.nb_ptr[I + 1])):
            offs.append(offs[-1] + int(plan.nbf[I]) * int(plan.nbf[plan.nb_idx[p]]))
    return np.asarray(offs, dtype=np.int64)


def write_back(plan: OraclePlan, subs: dict) -> np.ndarray:
    """Column block J of D <- the centre columns of T_J(D), placed on the rows of N(J)
    (Sec. "The Submatrix Method", step (iii))."""
    return write_back_cols(plan, {J: r.D_cols for J, r in subs.items()})


def write_back_cols(plan: OraclePlan, cols: dict) -> np.ndarray:
    """The write-back of ``write_back`` for any per-submatrix centre columns (J -> n_J x b_J array):
    block (I, J) of the result, for I in N(J), is the rows of I in J's columns."""
    off = d_block_offsets(plan)
    D = np.zeros(int(off[-1]), dtype=np.float64)
    for J, C in cols.items():
        for p in range(int(plan.nb_ptr[J]), int(plan.nb_ptr[J + 1])):
            I = int(plan.nb_idx[p])
            bI = int(plan.nbf[I])
            rows = C[int(plan.nb_off[p]):int(plan.nb_off[p]) + bI, :]
            # slot of block (I, J) in block row I
            q = int(plan.nb_ptr[I]) + int(np.nonzero(plan.nb_idx[plan.nb_ptr[I]:plan.nb_ptr[I + 1]] == J)[0][0])
            D[off[q]:off[q + 1]] = rows.reshape(-1)
    return D


def d_to_dense(plan: OraclePlan, D_vals: np.ndarray) -> np.ndarray:
    """Dense N x N copy of a D stored in the merged pattern (tiny systems only)."""
    nbf = plan.nbf.astype(np.int64)
    start = np.concatenate([[0], np.cumsum(nbf)])
    off = d_block_offsets(plan)
    N = int(start[-1])
    M = np.zeros((N, N))
    for I in range(nbf.shape[0]):
        for p in range(int(plan.nb_ptr[I]), int(plan.nb_ptr[I + 1])):
            J = int(plan.nb_idx[p])
            M[start[I]:start[I + 1], start[J]:start[J + 1]] = \
                D_vals[off[p]:off[p + 1]].reshape(int(nbf[I]), int(nbf[J]))
    return M


def csr_to_dense(nbf, row_ptr, col_idx, blk_off, vals) -> np.ndarray:
    """Dense N x N copy of a block-CSR matrix (tiny systems only)."""
    nbf = np.asarray(nbf, dtype=np.int64)
    start = np.concatenate([[0], np.cumsum(nbf)])
    N = int(start[-1])
    M = np.zeros((N, N))
    for I in range(nbf.shape[0]):
        for p in range(int(row_ptr[I]), int(row_ptr[I + 1])):
            J = int(col_idx[p])
            M[start[I]:start[I + 1], start[J]:start[J + 1]] = \
                vals[int(blk_off[p]):int(blk_off[p + 1])].reshape(int(nbf[I]), int(nbf[J]))
    return M


# ============================================================================ chemical potential

@dataclasses.dataclass
class MuResult:
    mu: float
    trace_DS: float
    steps: int
    ok: bool
    history: list          # [(mu, f(mu))] in evaluation order


def find_mu(count, n_occ: float, lo: float, hi: float, tol_n: float, tol_mu: float = 1e-10,
            max_steps: int = 100) -> MuResult:
    """Bisection for charge neutrality Tr(D S) = N_occ (Sec. "Simulation Details"), reading 4.

    ``count(mu)`` returns Tr(D(mu) S)."""
    hist = []
    mu = 0.5 * (lo + hi)
    t = float("nan")
    for step in range(1, max_steps + 1):
        mu = 0.5 * (lo + hi)
        t = count(mu)
        f = t - n_occ
        hist.append((mu, f))
        if abs(f) <= tol_n:
            return MuResult(mu, t, step, True, hist)
        if f < 0.0:
            lo = mu
        else:
            hi = mu
        if hi - lo <= tol_mu:
            return MuResult(mu, t, step, False, hist)
    return MuResult(mu, t, max_steps, False, hist)


# ============================================================================ input checks

def brute_force_pairs(pos: np.ndarray, cell: np.ndarray, rc: float):
    """All ordered molecule pairs with minimum-image distance^2 < rc^2, by a plain double loop."""
    n = pos.shape[0]
    out = []
    for I in range(n):
        for J in range(n):
            d = pos[J] - pos[I]
            d = d - cell * np.rint(d / cell)
            if d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < rc * rc:
                out.append((I, J))
    return out
