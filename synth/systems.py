"""Seeded water-like test systems: a jittered cubic lattice of "molecules", each carrying b basis
functions, with overlap S and Hamiltonian H stored block-CSR over molecules.

Construction (the readings of the workload description, one per parameter):

* Lattice: cubic, spacing 3.1 Angstrom (the density of 32 water molecules in a 9.8 Angstrom cell,
  (9.8^3/32)^(1/3) = 3.1), periodic cell of ``n_axis * spacing`` per axis, uniform jitter
  U(-0.3, 0.3) Angstrom per coordinate.
* Optional local density field (+-20 %): a local length-scale factor s ~ U(1-a, 1+a) on a periodic
  coarse grid of ``density_cell`` lattice cells, trilinearly interpolated to the lattice sites. Along
  each axis the gap between consecutive sites scales with s and each lattice line is renormalised to
  the cell length, so the system stays periodic while the local number density follows s^-3. (Read
  on the number density instead, +-20 % gives submatrix dimensions of only about 140-200; on the
  length scale it gives the 120-300 span the workload asks for.)
* All b functions of a molecule sit at the molecule's position. Intra-molecular blocks: S = identity,
  H = diag(on-site energies). Inter-molecular blocks for minimum-image centre distance r < r_c
  (strict): S = exp(-0.5 r^2) and H = -0.2 exp(-r/1.5) for every entry, optionally modulated by a
  direction-dependent factor (1 + aniso (u_a - u_c) . r_hat) that keeps S and H symmetric while
  making the individual off-diagonal blocks non-symmetric (used by tests that must catch transposed
  operands). Blocks at r >= r_c are absent. Between molecules with b_I and b_J functions every
  inter-molecular entry carries the factor 1/sqrt(b_I b_J): with it, the block of S seen by the
  normalised all-ones vector of each molecule is exactly the Gaussian-kernel matrix exp(-0.5 r_IJ^2),
  which is positive definite for every geometry, so S is positive definite (up to the cutoff
  truncation of terms below exp(-18)). Without the factor, b coincident functions multiply the
  coupling by b and S turns indefinite wherever two molecules come close (the +-20 % density field
  produces contacts at 1.8 Angstrom).
* On-site energies: 6 functions per molecule use types [0,1,1,1,2,2] with -1.0, -0.5, +0.3 Ha and
  four occupied orbitals per molecule. 23 functions per molecule draw one energy per function slot
  from N(-0.5, 0.3) Ha once per system; their occupied count (not given for that workload) is the m
  in 2..8 with the widest gap between the m-th and (m+1)-th lowest drawn energies, so the system is
  an insulator like the 6-function one.

Block-CSR layout (shared input format): block row I lists the molecules J with a stored block (I, J)
in ascending order; block (I, J) is b_I x b_J, row-major, and blocks are concatenated in CSR order,
so block slot p starts at ``blk_off[p]`` with ``blk_off[p+1] - blk_off[p] = b_I * b_J``.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

ONSITE_6 = np.array([-1.0, -0.5, -0.5, -0.5, 0.3, 0.3])


@dataclasses.dataclass(frozen=True)
class SystemSpec:
    nx: int
    ny: int
    nz: int
    nbf: str = "6"              # "6", "23" or "mixed" (6 or 23 per molecule, probability 1/2)
    spacing: float = 3.1
    jitter: float = 0.3
    cutoff: float = 6.0         # cutoff of the S blocks
    cutoff_h: Optional[float] = None   # cutoff of the H blocks (None: same as S)
    density_amp: float = 0.0    # +- amplitude of the local length-scale factor
    density_cell: int = 4       # lattice cells per coarse density-grid cell
    aniso: float = 0.0
    s_exp: float = 0.5
    hop: float = -0.2
    hop_len: float = 1.5
    occ_per_mol: int = 4        # occupied orbitals of a 6-function molecule
    basis_mix: float = 0.0      # beta of the per-molecule basis transform B = I - beta v v^T (0: none)
    basis_mix_every: int = 1    # transform molecules 0, k, 2k, ... (k = basis_mix_every)
    seed: int = 0

    @property
    def n_mol(self) -> int:
        return self.nx * self.ny * self.nz


@dataclasses.dataclass
class BlockCSR:
    row_ptr: np.ndarray   # int32 [n_mol+1]
    col_idx: np.ndarray   # int32 [nnzb]
    blk_off: np.ndarray   # int64 [nnzb+1], element offset of each block in vals
    vals: np.ndarray      # float64 [blk_off[-1]]

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])


@dataclasses.dataclass
class System:
    spec: SystemSpec
    pos: np.ndarray       # float64 [n_mol, 3], in [0, L)
    cell: np.ndarray      # float64 [3]
    nbf: np.ndarray       # int32 [n_mol]
    onsite: list          # per molecule float64 arrays of length nbf[I]
    S: BlockCSR
    H: BlockCSR

    @property
    def n_mol(self) -> int:
        return int(self.nbf.shape[0])

    @property
    def n_basis(self) -> int:
        return int(self.nbf.sum())

    occ: Optional[np.ndarray] = None   # int32 [n_mol], occupied orbitals per molecule
    dirs: Optional[np.ndarray] = None  # float64 [2, 23, 3], direction vectors of the anisotropic modulation

    @property
    def n_occ(self) -> float:
        return float(np.sum(self.occ))


# ------------------------------------------------------------------------------------ geometry

def _density_positions(spec: SystemSpec, rng: np.random.Generator) -> np.ndarray:
    nx, ny, nz = spec.nx, spec.ny, spec.nz
    a = spec.spacing
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    if spec.density_amp <= 0.0:
        return np.stack([ii * a, jj * a, kk * a], axis=-1).reshape(-1, 3).astype(np.float64)
    dc = spec.density_cell
    gx, gy, gz = -(-nx // dc), -(-ny // dc), -(-nz // dc)
    coarse = rng.uniform(1.0 - spec.density_amp, 1.0 + spec.density_amp, size=(gx, gy, gz))

    def interp(fi, fj, fk):
        i0, j0, k0 = np.floor(fi).astype(int), np.floor(fj).astype(int), np.floor(fk).astype(int)
        ti, tj, tk = fi - i0, fj - j0, fk - k0
        out = 0.0
        for di in (0, 1):
            wi = ti if di else 1.0 - ti
            for dj in (0, 1):
                wj = tj if dj else 1.0 - tj
                for dk in (0, 1):
                    wk = tk if dk else 1.0 - tk
                    out = out + wi * wj * wk * coarse[(i0 + di) % gx, (j0 + dj) % gy, (k0 + dk) % gz]
        return out

    # the coarse grid spans the whole periodic lattice (gx coarse cells over nx sites, about dc sites each)
    w = interp(ii * gx / nx, jj * gy / ny, kk * gz / nz)     # local length-scale factor s
    dims = (nx, ny, nz)
    coords = []
    for ax in range(3):
        n = dims[ax]
        L = n * a
        gap = 0.5 * (w + np.roll(w, -1, axis=ax))            # gap from site s to s+1 along ax
        cum = np.cumsum(gap, axis=ax) - gap                    # exclusive prefix sum
        tot = np.sum(gap, axis=ax, keepdims=True)
        coords.append(cum / tot * L)
    return np.stack(coords, axis=-1).reshape(-1, 3).astype(np.float64)


def _min_image(d: np.ndarray, cell: np.ndarray) -> np.ndarray:
    return d - cell * np.rint(d / cell)


def minimum_image_pairs(pos: np.ndarray, cell: np.ndarray, rc: float, chunk: int = 2048):
    """All ordered pairs (I, J), I == J included, with minimum-image distance^2 < rc^2 (strict).

    Returns (I, J, d) with d = minimum-image vector from I to J, sorted by (I, J). Uses a periodic
    cell list when every axis holds at least three cells of edge >= rc, else brute force.
    """
    n = pos.shape[0]
    rc2 = rc * rc
    m = np.floor(cell / rc).astype(int)
    out_i, out_j, out_d = [], [], []
    if np.all(m >= 3):
        csize = cell / m
        cidx = np.minimum((pos / csize).astype(int), m - 1)
        cflat = (cidx[:, 0] * m[1] + cidx[:, 1]) * m[2] + cidx[:, 2]
        order = np.argsort(cflat, kind="stable")
        ncell = int(m.prod())
        counts = np.bincount(cflat, minlength=ncell)
        starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
        offsets = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)])
        for lo in range(0, n, chunk):
            I = np.arange(lo, min(n, lo + chunk))
            for off in offsets:
                nc = (cidx[I] + off) % m
                nf = (nc[:, 0] * m[1] + nc[:, 1]) * m[2] + nc[:, 2]
                cnt = counts[nf]
                if cnt.sum() == 0:
                    continue
                ii = np.repeat(I, cnt)
                base = np.repeat(starts[nf], cnt)
                within = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
                jj = order[base + within]
                d = _min_image(pos[jj] - pos[ii], cell)
                r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
                keep = r2 < rc2
                out_i.append(ii[keep]); out_j.append(jj[keep]); out_d.append(d[keep])
    else:
        for lo in range(0, n, chunk):
            I = np.arange(lo, min(n, lo + chunk))
            d = _min_image(pos[None, :, :] - pos[I, None, :], cell)
            r2 = d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2]
            ii, jj = np.nonzero(r2 < rc2)
            out_i.append(I[ii]); out_j.append(jj); out_d.append(d[ii, jj])
    I = np.concatenate(out_i).astype(np.int64)
    J = np.concatenate(out_j).astype(np.int64)
    D = np.concatenate(out_d)
    key = np.lexsort((J, I))
    return I[key], J[key], D[key]


# ------------------------------------------------------------------------------------ matrices

def _build_blocks(I, J, d, nbf, onsite, dirs, value_fn, diag_fn, n_mol):
    """Block-CSR with blocks value_fn(r, dhat, b_I, b_J, I) for I != J and diag_fn(I) for I == J."""
    counts = np.bincount(I, minlength=n_mol)
    row_ptr = np.zeros(n_mol + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    bI = nbf[I].astype(np.int64)
    bJ = nbf[J].astype(np.int64)
    sizes = bI * bJ
    blk_off = np.zeros(I.shape[0] + 1, dtype=np.int64)
    np.cumsum(sizes, out=blk_off[1:])
    vals = np.zeros(int(blk_off[-1]), dtype=np.float64)
    r = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2])
    off = I != J
    for b1 in np.unique(bI):
        for b2 in np.unique(bJ):
            sel = np.nonzero(off & (bI == b1) & (bJ == b2))[0]
            if sel.size == 0:
                continue
            dhat = d[sel] / r[sel, None]
            blocks = value_fn(r[sel], dhat, int(b1), int(b2), dirs)      # [k, b1, b2]
            idx = blk_off[sel][:, None] + np.arange(b1 * b2)[None, :]
            vals[idx] = blocks.reshape(sel.size, -1)
    for p in np.nonzero(~off)[0]:
        b = int(bI[p])
        vals[blk_off[p]:blk_off[p + 1]] = diag_fn(int(I[p]), b).reshape(-1)
    return BlockCSR(row_ptr.astype(np.int32), J.astype(np.int32), blk_off, vals)


def make_system(spec: SystemSpec) -> System:
    rng = np.random.default_rng(spec.seed)
    n = spec.n_mol
    cell = np.array([spec.nx, spec.ny, spec.nz], dtype=np.float64) * spec.spacing
    pos = _density_positions(spec, rng)
    pos = pos + rng.uniform(-spec.jitter, spec.jitter, size=pos.shape)
    pos = np.mod(pos, cell)

    eps23 = rng.normal(-0.5, 0.3, size=23)
    if spec.nbf == "6":
        nbf = np.full(n, 6, dtype=np.int32)
    elif spec.nbf == "23":
        nbf = np.full(n, 23, dtype=np.int32)
    elif spec.nbf == "mixed":
        nbf = np.where(rng.random(n) < 0.5, 6, 23).astype(np.int32)
    else:
        raise ValueError(f"unknown nbf mode {spec.nbf!r}")
    onsite = [ONSITE_6 if b == 6 else eps23 for b in nbf]
    srt = np.sort(eps23)
    m23 = int(2 + np.argmax(srt[2:9] - srt[1:8]))      # widest gap after the m-th level, m in 2..8
    occ = np.where(nbf == 6, spec.occ_per_mol, m23).astype(np.int32)
    # fixed per-slot direction vectors for the optional anisotropic modulation (S: 0, H: 1)
    dirs = rng.normal(size=(2, 23, 3))

    rc_h = spec.cutoff if spec.cutoff_h is None else spec.cutoff_h

    def s_val(r, dhat, b1, b2, dirs):
        base = (1.0 / np.sqrt(b1 * b2)) * np.exp(-spec.s_exp * r * r)[:, None, None]
        if spec.aniso == 0.0:
            return np.broadcast_to(base, (r.shape[0], b1, b2)).copy()
        ua = dhat @ dirs[0, :b1].T          # [k, b1]
        uc = dhat @ dirs[0, :b2].T          # [k, b2]
        return base * (1.0 + spec.aniso * (ua[:, :, None] - uc[:, None, :]))

    def h_val(r, dhat, b1, b2, dirs):
        base = (1.0 / np.sqrt(b1 * b2)) * (spec.hop * np.exp(-r / spec.hop_len))[:, None, None]
        if spec.aniso == 0.0:
            return np.broadcast_to(base, (r.shape[0], b1, b2)).copy()
        ua = dhat @ dirs[1, :b1].T
        uc = dhat @ dirs[1, :b2].T
        return base * (1.0 + spec.aniso * (ua[:, :, None] - uc[:, None, :]))

    I, J, d = minimum_image_pairs(pos, cell, max(spec.cutoff, rc_h))
    r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
    sel_s = r2 < spec.cutoff * spec.cutoff
    sel_h = r2 < rc_h * rc_h
    S = _build_blocks(I[sel_s], J[sel_s], d[sel_s], nbf, onsite, dirs, s_val,
                      lambda i, b: np.eye(b), n)
    H = _build_blocks(I[sel_h], J[sel_h], d[sel_h], nbf, onsite, dirs, h_val,
                      lambda i, b: np.diag(onsite[i]), n)
    if spec.basis_mix != 0.0:
        _mix_basis(S, nbf, spec)
        _mix_basis(H, nbf, spec)
    return System(spec=spec, pos=pos, cell=cell, nbf=nbf, onsite=onsite, S=S, H=H, occ=occ, dirs=dirs)


def _mix_basis(M: BlockCSR, nbf: np.ndarray, spec: SystemSpec) -> None:
    """Replaces the basis of every basis_mix_every-th molecule I by a linear combination of its functions,
    B_I = I - beta v v^T with v = (1, 2, ..., b_I) / |(1, 2, ..., b_I)|, in place: block (I, J) becomes
    B_I M_IJ B_J (B symmetric, identity for untouched molecules). The same congruence of S and H leaves the
    generalized eigenvalues, hence the gap and mu, unchanged, while the overlap's condition number grows
    like 1 / (1 - beta)^2: a non-orthogonal basis with nearly dependent functions."""
    def B(I):
        b = int(nbf[I])
        if I % spec.basis_mix_every != 0:
            return None
        v = np.arange(1.0, b + 1.0)
        v /= np.linalg.norm(v)
        return np.eye(b) - spec.basis_mix * np.outer(v, v)
    n = nbf.shape[0]
    Bs = [B(I) for I in range(n)]
    for I in range(n):
        for p in range(int(M.row_ptr[I]), int(M.row_ptr[I + 1])):
            J = int(M.col_idx[p])
            if Bs[I] is None and Bs[J] is None:
                continue
            blk = M.vals[M.blk_off[p]:M.blk_off[p + 1]].reshape(int(nbf[I]), int(nbf[J]))
            if Bs[I] is not None:
                blk = Bs[I] @ blk
            if Bs[J] is not None:
                blk = blk @ Bs[J]
            M.vals[M.blk_off[p]:M.blk_off[p + 1]] = blk.ravel()


# ------------------------------------------------------------------------------------ named workloads

def spec_small_fp64(**kw) -> SystemSpec:
    """64 molecules (4x4x4), 6 functions each, FP64 end to end."""
    return SystemSpec(4, 4, 4, **{"seed": 1001, **kw})


def spec_batched_uneven(**kw) -> SystemSpec:
    """32,768 molecules (32x32x32) with a +-20 % local density field."""
    return SystemSpec(32, 32, 32, **{"density_amp": 0.2, "seed": 1002, **kw})


def spec_batched_uneven_4096(**kw) -> SystemSpec:
    """4,096 molecules (16x16x16) with the same +-20 % field: a smaller case of the same workload."""
    return SystemSpec(16, 16, 16, **{"density_amp": 0.2, "seed": 1012, **kw})


def spec_streamed_bf16(**kw) -> SystemSpec:
    """262,144 molecules (64x64x64), 6 functions each."""
    return SystemSpec(64, 64, 64, **{"seed": 1003, **kw})


def spec_streamed_4096(**kw) -> SystemSpec:
    """4,096 molecules (16x16x16), 6 functions each: a smaller case of the 262,144-molecule workload (same recipe,
    its own seed), for profiling."""
    return SystemSpec(16, 16, 16, **{"seed": 1013, **kw})


def spec_split_valence(**kw) -> SystemSpec:
    """16,384 molecules (32x32x16), 23 functions each."""
    return SystemSpec(32, 32, 16, **{"nbf": "23", "seed": 1004, **kw})


def spec_mixed(**kw) -> SystemSpec:
    """65,536 molecules (64x32x32), 6 or 23 functions per molecule."""
    return SystemSpec(64, 32, 32, **{"nbf": "mixed", "seed": 1005, **kw})


def spec_tiny(n=2, **kw) -> SystemSpec:
    """n^3 molecules; with n = 2 the 6 Angstrom cutoff spans the whole periodic cell."""
    return SystemSpec(n, n, n, **{"seed": 7, **kw})
