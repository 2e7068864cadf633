"""Seeded atom-resolved sparsity patterns (inputs only: positions, functions per site, the pattern).

The combination heuristic works on the pattern of the submatrices, nothing else. The paper applies it
where every atom starts with a submatrix of its own and species differ (its HIV-1 capsid system: large
submatrices around sodium ions, small ones around the atoms of water and protein), not to the
molecule-coalesced water of the main workload. This module makes a stand-in of that kind:

* the water lattice of ``systems.py`` (3.1 Angstrom spacing, jitter U(-0.3, 0.3)) with each molecule
  resolved into three sites: O at the lattice site with ``o_nbf`` functions, two H at 0.96 Angstrom
  from it, 104.5 degrees apart, in a random orientation, with ``h_nbf`` functions each;
* a fraction ``ion_fraction`` of the lattice sites holding an ion instead (``ion_nbf`` functions);
* function counts as in the paper's Sec. "Simulation Details": two per hydrogen, four for every other
  element of its systems but sulfur (so four for O and for a sodium ion);
* a pair of sites (a, b) is in the pattern when their minimum-image distance is below
  (r_a + r_b) / 2 (strict), r = ``rc`` for water atoms and ``rc_ion`` for ions, so ions get large
  submatrices; every site is its own neighbour.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .systems import minimum_image_pairs


@dataclasses.dataclass(frozen=True)
class SiteSpec:
    nx: int
    ny: int
    nz: int
    ion_fraction: float = 0.0
    o_nbf: int = 4
    h_nbf: int = 2
    ion_nbf: int = 4
    rc: float = 6.0
    rc_ion: float = 10.0
    spacing: float = 3.1
    jitter: float = 0.3
    seed: int = 0


@dataclasses.dataclass
class SitePattern:
    spec: SiteSpec
    pos: np.ndarray       # float64 [n_sites, 3]
    cell: np.ndarray      # float64 [3]
    species: np.ndarray   # int8 [n_sites]: 0 O, 1 H, 2 ion
    nbf: np.ndarray       # int32 [n_sites]
    nb_ptr: np.ndarray    # int32 [n_sites + 1]
    nb_idx: np.ndarray    # int32: neighbours of site J in ascending order, J included

    @property
    def n_sites(self) -> int:
        return int(self.nbf.shape[0])


def make_site_pattern(spec: SiteSpec) -> SitePattern:
    rng = np.random.default_rng(spec.seed)
    a = spec.spacing
    cell = np.array([spec.nx, spec.ny, spec.nz], dtype=np.float64) * a
    ii, jj, kk = np.meshgrid(np.arange(spec.nx), np.arange(spec.ny), np.arange(spec.nz), indexing="ij")
    lat = np.stack([ii, jj, kk], axis=-1).reshape(-1, 3).astype(np.float64) * a
    lat = lat + rng.uniform(-spec.jitter, spec.jitter, size=lat.shape)
    ion = rng.random(lat.shape[0]) < spec.ion_fraction
    # a random orthonormal frame per water molecule places its two H atoms
    q = rng.normal(size=(lat.shape[0], 3, 3))
    frames = np.linalg.qr(q)[0]
    half = np.deg2rad(104.5) / 2
    h1 = 0.96 * (np.cos(half) * frames[:, :, 0] + np.sin(half) * frames[:, :, 1])
    h2 = 0.96 * (np.cos(half) * frames[:, :, 0] - np.sin(half) * frames[:, :, 1])
    pos, species = [], []
    for m in range(lat.shape[0]):
        if ion[m]:
            pos.append(lat[m]); species.append(2)
        else:
            pos.extend([lat[m], lat[m] + h1[m], lat[m] + h2[m]]); species.extend([0, 1, 1])
    pos = np.mod(np.asarray(pos), cell)
    species = np.asarray(species, dtype=np.int8)
    nbf = np.choose(species, [spec.o_nbf, spec.h_nbf, spec.ion_nbf]).astype(np.int32)
    radius = np.where(species == 2, spec.rc_ion, spec.rc)
    I, J, d = minimum_image_pairs(pos, cell, float(radius.max()))
    r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
    lim = 0.5 * (radius[I] + radius[J])
    keep = r2 < lim * lim
    I, J = I[keep], J[keep]
    nb_ptr = np.zeros(pos.shape[0] + 1, dtype=np.int64)
    np.cumsum(np.bincount(J, minlength=pos.shape[0]), out=nb_ptr[1:])
    order = np.lexsort((I, J))                 # column J, rows I ascending
    return SitePattern(spec, pos, cell, species, nbf, nb_ptr.astype(np.int32), I[order].astype(np.int32))


def spec_ions_in_water(**kw) -> SiteSpec:
    """4,096 lattice sites (16x16x16), 2 % ions: about 12,000 atom sites."""
    return SiteSpec(16, 16, 16, **{"ion_fraction": 0.02, "seed": 1301, **kw})


def spec_ions_in_water_small(**kw) -> SiteSpec:
    """216 lattice sites (6x6x6), 3 % ions: about 630 atom sites (fast enough for the plain oracle)."""
    return SiteSpec(6, 6, 6, **{"ion_fraction": 0.03, "seed": 1302, **kw})


# on-site energies (Ha) of the site species' functions: O (4), H (2), ion (4)
ONSITE_SITE = {0: np.array([-1.0, -0.5, -0.5, -0.5]), 1: np.array([-0.4, 0.3]), 2: np.array([-1.2, 0.2, 0.2, 0.2])}


def site_system(sp: SitePattern, s_exp: float = 0.5, hop: float = -0.2, hop_len: float = 1.5):
    """S and H0 on an atom-resolved pattern: the blocks of the pattern's pairs filled by the element model of
    systems.py (S = exp(-s_exp r^2) / sqrt(b_a b_b), H0 = hop exp(-r / hop_len) / sqrt(b_a b_b) between
    different sites, S = identity and H0 = diag(on-site energies of the species) on a site), so that S is
    positive definite for every geometry as in the molecule systems. Returns a systems.System whose
    "molecules" are the sites (spec carries the model's parameters; functions of other species than the
    molecule systems' have other on-site energies, ONSITE_SITE)."""
    from .systems import System, SystemSpec, _build_blocks, _min_image
    n = sp.n_sites
    J = np.repeat(np.arange(n), np.diff(sp.nb_ptr))          # column molecule of every (row, column) pair
    I = sp.nb_idx.astype(np.int64)
    key = np.lexsort((J, I))                                 # rows I ascending, then columns
    I, J = I[key], J[key].astype(np.int64)
    d = _min_image(sp.pos[J] - sp.pos[I], sp.cell)
    onsite = [ONSITE_SITE[int(s)] for s in sp.species]
    spec = SystemSpec(sp.spec.nx, sp.spec.ny, sp.spec.nz, s_exp=s_exp, hop=hop, hop_len=hop_len, seed=sp.spec.seed)

    def s_val(r, dhat, b1, b2, dirs):
        base = (1.0 / np.sqrt(b1 * b2)) * np.exp(-s_exp * r * r)[:, None, None]
        return np.broadcast_to(base, (r.shape[0], b1, b2)).copy()

    def h_val(r, dhat, b1, b2, dirs):
        base = (1.0 / np.sqrt(b1 * b2)) * (hop * np.exp(-r / hop_len))[:, None, None]
        return np.broadcast_to(base, (r.shape[0], b1, b2)).copy()

    S = _build_blocks(I, J, d, sp.nbf, onsite, None, s_val, lambda i, b: np.eye(b), n)
    H = _build_blocks(I, J, d, sp.nbf, onsite, None, h_val, lambda i, b: np.diag(onsite[i]), n)
    # occupied orbitals: every O function, the lower H and ion functions (a gap of 0.45 Ha on the 632-site
    # system between -0.29 and +0.16 Ha; two per O would put the Fermi level inside O's threefold level)
    occ = np.choose(sp.species, [4, 1, 1]).astype(np.int32)
    return System(spec=spec, pos=sp.pos, cell=sp.cell, nbf=sp.nbf.astype(np.int32), onsite=onsite, S=S, H=H,
                  occ=occ)
