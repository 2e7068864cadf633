"""Merged submatrices solved on the GPU (Sec. "Submatrix Combination Heuristics", Eq.
combination_criterion), against the FP64 oracle's grouped solve (oracle/combine_oracle.py: solve_grouped).

The inputs are atom-resolved: the water lattice with every molecule resolved into O and two H sites and a
fraction of the lattice sites holding an ion (synth/sites.py), S and H0 filled by the element model of the
molecule systems. The groups come from the library's combination heuristic on the pattern (groups wider
than the 64 centre columns a submatrix takes are split in member order, the same split on both sides). On
a sample of groups (the largest sixteen and eight more), the grouped plan must give, through
nolsm_scatter_density, the oracle's columns of every member on its rows within the path's tolerance (FP64
1e-9, BF16X3 1e-4) and the groups' partial traces; one group per site must reproduce the per-site plan; the
grouped solve must need less work (sum of n^3) than the per-site one, in the ratio the heuristic reports."""
import numpy as np
import pytest

from oracle import combine_oracle as co
from oracle import nolsm_oracle as orc
from synth import SiteSpec, make_site_pattern, site_system, spec_ions_in_water_small

pytestmark = pytest.mark.gpu

PATTERNS = {"3pct_ions": spec_ions_in_water_small(), "20pct_ions": SiteSpec(6, 6, 6, ion_fraction=0.2, seed=1303)}


@pytest.fixture(scope="module")
def nl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08245_gb300 import build
    build.build()
    import paper_2104_08245_gb300 as nl
    return nl


def split_wide_groups(group_of, nbf, limit=64):
    """Groups wider than `limit` functions cut, in member order, into consecutive parts of at most `limit`
    (each part labelled by its smallest member)."""
    g = np.asarray(group_of).copy()
    for lab in np.unique(g):
        mem = np.nonzero(g == lab)[0]
        if nbf[mem].sum() <= limit:
            continue
        start, width = mem[0], 0
        for J in mem:
            if width + nbf[J] > limit:
                start, width = J, 0
            g[J] = start
            width += nbf[J]
    return g


def setup(nl, name):
    sp = make_site_pattern(PATTERNS[name])
    sysm = site_system(sp)
    po = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    cr = nl.nolsm_combine_submatrices(sp.nbf, sp.nb_ptr, sp.nb_idx)
    groups = split_wide_groups(cr.group_of, sp.nbf)
    return sp, sysm, po, cr, groups


def quiet_mu(sysm):
    """A chemical potential far from every eigenvalue of the whole system (LAPACK), between the occupied and
    the virtual states when possible: the tests check arithmetic, not the ill-conditioned sign near an
    eigenvalue."""
    import scipy.linalg
    S = orc.csr_to_dense(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
    H = orc.csr_to_dense(sysm.nbf, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
    eps = scipy.linalg.eigh(H, S, eigvals_only=True)
    gaps = np.diff(eps)
    k = int(np.argmax(gaps[len(eps) // 4: 3 * len(eps) // 4])) + len(eps) // 4
    return 0.5 * (eps[k] + eps[k + 1])


def sample_groups(groups, nbf, k_large=16, k_rand=8, seed=3):
    labels, inv = np.unique(groups, return_inverse=True)
    width = np.bincount(inv, weights=nbf)
    order = np.argsort(-width, kind="stable")
    pick = set(int(labels[i]) for i in order[:k_large])
    rng = np.random.default_rng(seed)
    pick |= set(int(x) for x in rng.choice(labels, size=min(k_rand, len(labels)), replace=False))
    return sorted(pick), labels


def group_cond(sysm, po, groups, pick):
    """Condition numbers of the picked groups' overlaps T_G(S) (gathered by the oracle, LAPACK eigenvalues)."""
    out = []
    for g in pick:
        members = [int(J) for J in np.nonzero(groups == g)[0]]
        rows = sorted(set(int(m) for J in members for m in po.nb_idx[po.nb_ptr[J]:po.nb_ptr[J + 1]]))
        ev = np.linalg.eigvalsh(co.gather_rows(sysm.S, sysm.nbf, rows))
        out.append(ev[-1] / ev[0])
    return np.asarray(out)


def member_error(po, D, ref, members):
    off = orc.d_block_offsets(po)
    err = 0.0
    for J in members:
        cols = ref.D_cols[J]
        bJ = int(po.nbf[J])
        for p in range(po.nb_ptr[J], po.nb_ptr[J + 1]):
            I = int(po.nb_idx[p])
            q = po.nb_ptr[I] + int(np.nonzero(po.nb_idx[po.nb_ptr[I]:po.nb_ptr[I + 1]] == J)[0][0])
            bI = int(po.nbf[I])
            got = D[off[q]:off[q + 1]].reshape(bI, bJ)
            err = max(err, float(np.max(np.abs(got - cols[po.nb_off[p]:po.nb_off[p] + bI, :]))))
    return err


@pytest.mark.parametrize("name", list(PATTERNS))
def test_grouped_solve_matches_the_oracle(nl, name):
    sp, sysm, po, cr, groups = setup(nl, name)
    mu = quiet_mu(sysm)
    pick, labels = sample_groups(groups, sp.nbf)
    ref = co.solve_grouped(sysm, mu, groups, po, only=pick)
    members = [J for J in range(sp.n_sites) if int(groups[J]) in set(pick)]
    mplan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    gplan = nl.nolsm_build_grouped(mplan, groups)
    info = gplan.info()
    assert info.grouped == 1 and info.n_mol == len(labels)
    gidx = {int(l): k for k, l in enumerate(labels)}     # groups are numbered by their smallest member
    # the FP64 path takes submatrices up to 775 rows (its factorisation panel). With larger merged ones the
    # FP32 mode stands in for it; its 1e-6 target (n-scaled) holds for overlaps of condition number up to 10,
    # and the ion groups' merged overlaps have 13 to 29 (LAPACK on the oracle's gathered T_G(S)), so there it
    # is held to the BF16X3 target. (The library's lower estimate of the condition number from the FP32
    # Cholesky factor's diagonal gives 1.5 to 2.8 for these groups: it keeps them in the mode without
    # counting them in ill_conditioned_kept.)
    kappa = group_cond(sysm, po, groups, pick)
    large = info.max_n > 775
    first = ("fp32", 1e-4) if large else ("fp64", 1e-9)
    for prec, tol in (first, ("bf16x3", 1e-4)):
        gplan.stats_reset()
        r = nl.nolsm_solve_batch(gplan, mu, nl.options(prec))
        if large and prec == "fp32":
            kept = gplan.stats()["ill_conditioned_kept"]
            print(f"{name}: condition numbers of the sampled groups' overlaps {kappa.min():.1f}..{kappa.max():.1f}; "
                  f"{kept} groups above 775 rows counted as kept in FP32 mode")
        D = gplan.scatter().cpu().numpy()
        err = member_error(po, D, ref, members)
        tS = r.sub_t_S.cpu().numpy()
        terr = max(abs(tS[gidx[g]] - sum(ref.t_S[J] for J in members if int(groups[J]) == g)) for g in pick)
        print(f"{name}: {sp.n_sites} sites in {info.n_mol} groups (n {info.min_n}..{info.max_n}), {prec}: "
              f"max|dD| = {err:.3e} on {len(pick)} groups ({len(members)} sites), max group trace error {terr:.3e}")
        assert err <= tol
        assert terr <= max(tol, 1e-12) * 10
        assert np.all(r.sub_status.cpu().numpy() == 0)


def test_one_group_per_site_reproduces_the_per_site_plan(nl):
    sp, sysm, po, cr, groups = setup(nl, "3pct_ions")
    mu = quiet_mu(sysm)
    mplan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    gplan = nl.nolsm_build_grouped(mplan, np.arange(sp.n_sites))
    nl.nolsm_solve_batch(mplan, mu, nl.options("fp64"))
    nl.nolsm_solve_batch(gplan, mu, nl.options("fp64"))
    D1 = mplan.scatter().cpu().numpy()
    D2 = gplan.scatter().cpu().numpy()
    err = float(np.max(np.abs(D1 - D2)))
    print(f"singleton groups vs per-site plan: max|dD| = {err:.3e}")
    assert err <= 1e-12   # the same submatrices, rows reordered (the centre site first)


def test_grouped_work_and_find_mu(nl):
    """The groups' sum of n^3 is the heuristic's reported value, below the per-site one; the bisection runs
    on the groups (BF16X3), and at its final mu the sampled groups' columns match the oracle's grouped solve
    at that mode's tolerance."""
    sp, sysm, po, cr, groups = setup(nl, "3pct_ions")
    mplan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    gplan = nl.nolsm_build_grouped(mplan, cr.group_of)
    assert gplan.info().sum_n3 == pytest.approx(cr.sum_n3_after, rel=1e-12)
    assert mplan.info().sum_n3 == pytest.approx(cr.sum_n3_before, rel=1e-12)
    m = gplan.find_mu(float(np.sum(sysm.occ)), 0.0, 0.0, nl.options("bf16x3"))
    pick, _ = sample_groups(cr.group_of, sp.nbf, k_large=8, k_rand=4)
    ref = co.solve_grouped(sysm, m.mu, cr.group_of, po, only=pick)
    members = [J for J in range(sp.n_sites) if int(cr.group_of[J]) in set(pick)]
    D = gplan.scatter().cpu().numpy()
    err = member_error(po, D, ref, members)
    print(f"grouped find_mu (BF16X3): {m.steps} points, mu {m.mu:.6f}, status {m.status}, sampled max|dD| {err:.3e}")
    assert err <= 1e-4


def test_too_wide_groups_are_refused(nl):
    sp, sysm, po, cr, groups = setup(nl, "20pct_ions")
    mplan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    with pytest.raises(nl.NolsmError) as e:
        nl.nolsm_build_grouped(mplan, cr.group_of)   # the heuristic's groups, one of them 80 functions wide
    assert e.value.status == nl._abi.ERR_UNSUPPORTED
