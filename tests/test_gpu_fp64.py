"""Parity of the FP64 GPU path (through the C ABI) with the FP64 CPU oracle.

Integer maps bit-exact; D element by element within 1e-9; traces; the mu-bisection sequence; the
whole-cell case against LAPACK's generalized eigensolver; submatrix ranges; malformed input and a
non-positive-definite overlap made on the host (no GPU fault is provoked)."""
import numpy as np
import pytest
import scipy.linalg

from oracle import nolsm_oracle as orc
from synth import SystemSpec, make_system, spec_small_fp64, spec_tiny

pytestmark = pytest.mark.gpu

TOL_D = 1e-9


@pytest.fixture(scope="module")
def nl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08245_gb300 import build
    build.build()
    import paper_2104_08245_gb300 as nl
    return nl


def oracle_plan(sysm):
    return orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)


VARIANTS = {
    "small": spec_small_fp64(),
    "aniso_cutoffs": spec_small_fp64(aniso=0.3, cutoff_h=5.0, seed=11),
    "h_longer": SystemSpec(4, 4, 3, cutoff=4.5, cutoff_h=6.0, aniso=0.2, seed=12),
    "mixed_nbf": SystemSpec(3, 3, 3, nbf="mixed", cutoff=4.5, seed=13),
    "isolated": SystemSpec(3, 3, 2, cutoff=1.5, seed=14),
    "one_molecule": SystemSpec(1, 1, 1, seed=15),
}


@pytest.mark.parametrize("name", list(VARIANTS))
def test_plan_maps_are_bit_exact(nl, name):
    sysm = make_system(VARIANTS[name])
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    m = {k: v.cpu().numpy() for k, v in plan.maps().items()}
    ref = oracle_plan(sysm)
    assert np.array_equal(m["nb_ptr"], ref.nb_ptr)
    assert np.array_equal(m["nb_idx"], ref.nb_idx)
    assert np.array_equal(m["nb_off"], ref.nb_off)
    assert np.array_equal(m["sub_n"], ref.sub_n)
    assert np.array_equal(m["sub_c0"], ref.sub_c0)
    assert np.array_equal(m["d_blk_off"], orc.d_block_offsets(ref))
    info = plan.info()
    assert info.max_n == ref.sub_n.max() and info.min_n == ref.sub_n.min()


@pytest.mark.parametrize("name", list(VARIANTS))
def test_fp64_density_matches_oracle(nl, name):
    sysm = make_system(VARIANTS[name])
    mu = -0.1
    ref = orc.solve(sysm, mu)
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    r = nl.nolsm_solve_batch(plan, mu, nl.options("fp64"))
    D = plan.scatter().cpu().numpy()
    assert D.shape == ref.D_vals.shape
    assert np.max(np.abs(D - ref.D_vals)) <= TOL_D
    n = sysm.n_mol
    tS = np.array([ref.subs[J].t_S for J in range(n)])
    tH = np.array([ref.subs[J].t_H for J in range(n)])
    assert np.max(np.abs(r.sub_t_S.cpu().numpy() - tS)) <= TOL_D
    assert np.max(np.abs(r.sub_t_H.cpu().numpy() - tH)) <= TOL_D
    assert r.trace_DS == pytest.approx(ref.trace_DS, rel=1e-12, abs=1e-12)
    assert r.trace_DH == pytest.approx(ref.trace_DH, rel=1e-12, abs=1e-12)
    steps = np.array([ref.subs[J].steps for J in range(n)])
    assert np.max(np.abs(r.iters.cpu().numpy() - steps)) <= 1
    assert np.all(r.sub_status.cpu().numpy() == 0)


@pytest.mark.parametrize("aniso", [0.0, 0.35])
def test_whole_cell_matches_full_generalized_eigenproblem(nl, aniso):
    sysm = make_system(spec_tiny(2, aniso=aniso))
    S = orc.csr_to_dense(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
    H = orc.csr_to_dense(sysm.nbf, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
    eps, C = scipy.linalg.eigh(H, S)
    n_occ = int(sysm.n_occ)
    mu = 0.5 * (eps[n_occ - 1] + eps[n_occ])
    P = C[:, :n_occ] @ C[:, :n_occ].T
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    r = nl.nolsm_solve_batch(plan, mu, nl.options("fp64"))
    D = orc.d_to_dense(oracle_plan(sysm), plan.scatter().cpu().numpy())
    assert np.max(np.abs(D - P)) <= TOL_D
    assert r.trace_DS == pytest.approx(n_occ, abs=1e-9)
    assert r.trace_DH == pytest.approx(float(np.sum(eps[:n_occ])), abs=1e-9)


def test_find_mu_follows_the_oracle_sequence(nl):
    sysm = make_system(spec_small_fp64())
    plan_o = oracle_plan(sysm)
    tol_n = 1e-5
    ref = orc.find_mu(lambda mu: orc.solve(sysm, mu, plan=plan_o).trace_DS, sysm.n_occ, -2.0, 2.0,
                      tol_n=tol_n * sysm.n_occ)
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    got = plan.find_mu(sysm.n_occ, -2.0, 2.0, nl.options("fp64", tol_n=tol_n))
    assert got.status == 0 and ref.ok
    assert got.steps == ref.steps
    assert np.array_equal(np.array(got.history), np.array([m for m, _ in ref.history]))
    assert got.mu == ref.mu
    assert got.trace_DS == pytest.approx(ref.trace_DS, abs=1e-9)
    D = plan.scatter().cpu().numpy()
    assert np.max(np.abs(D - orc.solve(sysm, ref.mu, plan=plan_o).D_vals)) <= TOL_D


def test_submatrix_range_solves_and_writes_only_that_range(nl):
    import torch
    sysm = make_system(spec_small_fp64())
    mu = -0.1
    ref = orc.solve(sysm, mu)
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    r = nl.nolsm_solve_batch(plan, mu, nl.options("fp64", sub_begin=10, sub_end=30))
    assert r.trace_DS == pytest.approx(sum(ref.subs[J].t_S for J in range(10, 30)), rel=1e-12)
    info = plan.info()
    D = torch.full((info.d_nvals,), float("nan"), dtype=torch.float64, device="cuda")
    D = plan.scatter(D).cpu().numpy()
    po = oracle_plan(sysm)
    off = orc.d_block_offsets(po)
    for I in range(sysm.n_mol):
        for p in range(po.nb_ptr[I], po.nb_ptr[I + 1]):
            J = po.nb_idx[p]
            blk = D[off[p]:off[p + 1]]
            if 10 <= J < 30:
                assert np.max(np.abs(blk - ref.D_vals[off[p]:off[p + 1]])) <= TOL_D
            else:
                assert np.all(np.isnan(blk))


def test_overlap_not_positive_definite_is_reported(nl):
    sysm = make_system(spec_small_fp64())
    # host-made fault: the overlap diagonal block of molecule 5 is negated
    p = int(np.nonzero(sysm.S.col_idx[sysm.S.row_ptr[5]:sysm.S.row_ptr[6]] == 5)[0][0]) + sysm.S.row_ptr[5]
    sysm.S.vals[sysm.S.blk_off[p]:sysm.S.blk_off[p + 1]] *= -1.0
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    r = nl.nolsm_solve_batch(plan, -0.1, nl.options("fp64"), check=False)
    assert r.status == nl._abi.ERR_NOT_SPD
    st = r.sub_status.cpu().numpy()
    po = oracle_plan(sysm)
    for J in range(sysm.n_mol):
        has5 = 5 in po.nb_idx[po.nb_ptr[J]:po.nb_ptr[J + 1]]
        assert (st[J] == nl._abi.ERR_NOT_SPD) == has5


def test_malformed_input_is_rejected(nl):
    sysm = make_system(spec_small_fp64())
    bad = make_system(spec_small_fp64())
    a, b = bad.S.row_ptr[3], bad.S.row_ptr[4]
    bad.S.col_idx[a:b] = bad.S.col_idx[a:b][::-1].copy()      # unsorted row
    with pytest.raises(nl.NolsmError) as e:
        nl.nolsm_build_submatrices(nl.DeviceSystem(bad))
    assert e.value.status == nl._abi.ERR_ARG
    asym = make_system(spec_small_fp64())
    # drop block (0, J) from row 0 of H only, keeping (J, 0): structurally asymmetric
    row = list(asym.H.col_idx[asym.H.row_ptr[0]:asym.H.row_ptr[1]])
    J = row[-1]
    keep = np.ones(asym.H.col_idx.shape[0], dtype=bool)
    keep[asym.H.row_ptr[1] - 1] = False
    blk = np.ones(asym.H.vals.shape[0], dtype=bool)
    blk[asym.H.blk_off[asym.H.row_ptr[1] - 1]:asym.H.blk_off[asym.H.row_ptr[1]]] = False
    asym.H.col_idx = asym.H.col_idx[keep]
    asym.H.vals = asym.H.vals[blk]
    asym.H.row_ptr = asym.H.row_ptr.copy()
    asym.H.row_ptr[1:] -= 1
    with pytest.raises(nl.NolsmError) as e:
        nl.nolsm_build_submatrices(nl.DeviceSystem(asym))
    assert e.value.status == nl._abi.ERR_ARG
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    with pytest.raises(nl.NolsmError):
        nl.nolsm_solve_batch(plan, -0.1, nl.options("fp64", sub_begin=50, sub_end=40))
    with pytest.raises(nl.NolsmError):
        nl.nolsm_scatter_density(plan)      # nothing solved yet


def test_fp64_sampled_at_full_size(nl):
    """The 32,768-molecule uneven system: full plan bit-exact on sampled molecules, and D of a
    contiguous range of submatrices (a few hundred) against the oracle on sampled columns."""
    from synth import spec_batched_uneven
    sysm = make_system(spec_batched_uneven())
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    m = {k: v.cpu().numpy() for k, v in plan.maps().items()}
    po = oracle_plan(sysm)
    assert np.array_equal(m["nb_ptr"], po.nb_ptr) and np.array_equal(m["nb_idx"], po.nb_idx)
    assert np.array_equal(m["sub_n"], po.sub_n) and np.array_equal(m["sub_c0"], po.sub_c0)
    j0, j1 = 5000, 5304
    mu = -0.1
    r = nl.nolsm_solve_batch(plan, mu, nl.options("fp64", sub_begin=j0, sub_end=j1))
    D = plan.scatter().cpu().numpy()
    off = m["d_blk_off"]
    rng = np.random.default_rng(7)
    sample = sorted(rng.choice(np.arange(j0, j1), size=12, replace=False))
    ref = orc.solve(sysm, mu, subs=sample, plan=po)
    for J in sample:
        cols = ref.subs[J].D_cols
        for p in range(po.nb_ptr[J], po.nb_ptr[J + 1]):
            I = po.nb_idx[p]
            q = po.nb_ptr[I] + int(np.nonzero(po.nb_idx[po.nb_ptr[I]:po.nb_ptr[I + 1]] == J)[0][0])
            got = D[off[q]:off[q + 1]].reshape(6, 6)
            want = cols[po.nb_off[p]:po.nb_off[p] + 6, :]
            assert np.max(np.abs(got - want)) <= TOL_D
        assert r.sub_t_S.cpu().numpy()[J] == pytest.approx(ref.subs[J].t_S, abs=TOL_D)
