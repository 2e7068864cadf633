"""Parity of the energy-weighted density matrix T_J(W) = T_J(D) T_J(H0) T_J(D) (NOLSM section) computed
on the GPU (nolsm_energy_weighted, through the C ABI) with the FP64 oracle's product of the definition.

Tolerances: the FP64 path 1e-9 (the D target). The tensor-core modes multiply the FP32 A_J by D_c in
FP32, so |dW_c| <= ||A_J||_inf max|dD_c| + the FP32 rounding of the product; the test allows
2 ||A_J||_inf times the mode's D tolerance, ||A_J||_inf = max absolute row sum of T_J(S)^-1 T_J(H0)
over the checked submatrices (from the oracle)."""
import numpy as np
import pytest
import scipy.linalg

from oracle import nolsm_oracle as orc
from synth import SystemSpec, make_system, spec_small_fp64, spec_tiny

pytestmark = pytest.mark.gpu

TOL_W_FP64 = 1e-9
TOL_D = {"fp32": 1e-6, "bf16x3": 1e-4, "fp16": 1e-4}


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


def a_norm(sysm, plan, subs):
    """max over subs of ||T_J(S)^-1 T_J(H0)||_inf."""
    out = 0.0
    for J in subs:
        S = orc.gather(plan, J, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
        H = orc.gather(plan, J, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
        out = max(out, orc.spectral_scale(orc.overlap_inverse(S) @ H))
    return out


def w_error(plan_o, wref, W, subs):
    """max|dW| over the blocks of W written by the listed submatrices."""
    off = orc.d_block_offsets(plan_o)
    err = 0.0
    for J in subs:
        cols = wref.W_cols[J]
        bJ = int(plan_o.nbf[J])
        for p in range(plan_o.nb_ptr[J], plan_o.nb_ptr[J + 1]):
            I = int(plan_o.nb_idx[p])
            bI = int(plan_o.nbf[I])
            q = plan_o.nb_ptr[I] + int(np.nonzero(plan_o.nb_idx[plan_o.nb_ptr[I]:plan_o.nb_ptr[I + 1]] == J)[0][0])
            got = W[off[q]:off[q + 1]].reshape(bI, bJ)
            err = max(err, float(np.max(np.abs(got - cols[plan_o.nb_off[p]:plan_o.nb_off[p] + bI, :]))))
    return err


VARIANTS = {
    "small": spec_small_fp64(),
    "aniso_cutoffs": spec_small_fp64(aniso=0.3, cutoff_h=5.0, seed=11),
    "mixed_nbf": SystemSpec(3, 3, 3, nbf="mixed", cutoff=4.5, seed=13),   # b = 23: three column passes
    "isolated": SystemSpec(3, 3, 2, cutoff=1.5, seed=14),
    "one_molecule": SystemSpec(1, 1, 1, seed=15),
}


@pytest.mark.parametrize("name", list(VARIANTS))
def test_fp64_energy_weighted_matches_oracle(nl, name):
    sysm = make_system(VARIANTS[name])
    mu = -0.1
    ref = orc.solve(sysm, mu)
    wref = orc.energy_weighted(sysm, ref)
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    nl.nolsm_solve_batch(plan, mu, nl.options("fp64"))
    W, tw = plan.energy_weighted()
    W = W.cpu().numpy()
    assert W.shape == wref.W_vals.shape
    assert float(np.max(np.abs(W - wref.W_vals))) <= TOL_W_FP64
    assert tw == pytest.approx(wref.trace_WS, rel=1e-10, abs=1e-10)


@pytest.mark.parametrize("aniso", [0.0, 0.35])
def test_whole_cell_matches_generalized_eigenproblem(nl, aniso):
    sysm = make_system(spec_tiny(2, aniso=aniso))
    S = orc.csr_to_dense(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
    H = orc.csr_to_dense(sysm.nbf, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
    eps, C = scipy.linalg.eigh(H, S)
    n_occ = int(sysm.n_occ)
    mu = 0.5 * (eps[n_occ - 1] + eps[n_occ])
    Wref = (C[:, :n_occ] * eps[:n_occ]) @ C[:, :n_occ].T
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    nl.nolsm_solve_batch(plan, mu, nl.options("fp64"))
    W, tw = plan.energy_weighted()
    Wd = orc.d_to_dense(oracle_plan(sysm), W.cpu().numpy())
    assert float(np.max(np.abs(Wd - Wref))) <= TOL_W_FP64
    assert tw == pytest.approx(float(np.sum(eps[:n_occ])), abs=1e-9)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fp16"])
def test_tensor_modes_match_oracle(nl, prec):
    sysm = make_system(spec_small_fp64())
    po = oracle_plan(sysm)
    mu = -0.1
    ref = orc.solve(sysm, mu, plan=po)
    wref = orc.energy_weighted(sysm, ref)
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    nl.nolsm_solve_batch(plan, mu, nl.options(prec))
    W, tw = plan.energy_weighted()
    err = float(np.max(np.abs(W.cpu().numpy() - wref.W_vals)))
    tol = 2.0 * a_norm(sysm, po, range(sysm.n_mol)) * TOL_D[prec]
    print(f"{prec}: max|dW| = {err:.3e} (tolerance {tol:.2e}), Tr(WS) {tw:.9f} vs {wref.trace_WS:.9f}")
    assert err <= tol
    assert abs(tw - wref.trace_WS) <= 1e-5 * abs(wref.trace_WS)


def test_range_writes_only_its_blocks(nl):
    sysm = make_system(spec_small_fp64(aniso=0.3, cutoff_h=5.0, seed=11))
    po = oracle_plan(sysm)
    mu = -0.1
    o = nl.options("bf16x3")
    o.sub_begin, o.sub_end = 10, 30
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    nl.nolsm_solve_batch(plan, mu, o)
    import torch
    W = torch.full((plan.info().d_nvals,), 7.0, dtype=torch.float64, device=plan.dsys.nbf.device)
    plan.energy_weighted(W)
    W = W.cpu().numpy()
    subs = list(range(10, 30))
    wref = orc.energy_weighted(sysm, orc.solve(sysm, mu, subs=subs, plan=po))
    assert w_error(po, wref, W, subs) <= 2.0 * a_norm(sysm, po, subs) * TOL_D["bf16x3"]
    # blocks (I, J) of the other columns J keep the sentinel
    off = orc.d_block_offsets(po)
    written = np.zeros(W.shape, dtype=bool)
    for J in subs:
        for p in range(po.nb_ptr[J], po.nb_ptr[J + 1]):
            I = int(po.nb_idx[p])
            q = po.nb_ptr[I] + int(np.nonzero(po.nb_idx[po.nb_ptr[I]:po.nb_ptr[I + 1]] == J)[0][0])
            written[off[q]:off[q + 1]] = True
    assert np.all(W[~written] == 7.0)


def test_errors_are_reported(nl):
    sysm = make_system(spec_small_fp64())
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    with pytest.raises(nl.NolsmError) as e:
        plan.energy_weighted()
    assert e.value.status == 9          # NOLSM_ERR_NO_SOLUTION
    o = nl.options("bf16x3")
    o.symmetric_form = 1
    nl.nolsm_solve_batch(plan, -0.1, o)
    with pytest.raises(nl.NolsmError) as e:
        plan.energy_weighted()
    assert e.value.status == 8          # NOLSM_ERR_UNSUPPORTED: the symmetric form keeps no A_J


def test_full_size_after_find_mu_sampled(nl):
    """32,768 molecules with the density field: mu by the GPU bisection (BF16X3, every submatrix in one
    launch, as the benchmark runs it), then W of all submatrices; 64 sampled submatrices (with the
    smallest and the largest) against the oracle at that mu."""
    from synth import spec_batched_uneven
    sysm = make_system(spec_batched_uneven())
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    po = oracle_plan(sysm)
    m = plan.find_mu(float(np.sum(sysm.occ)), 0.0, 0.0, nl.options("bf16x3"))
    assert m.status == 0
    W, tw = plan.energy_weighted()
    W = W.cpu().numpy()
    rng = np.random.default_rng(17)
    subs = sorted({int(np.argmin(po.sub_n)), int(np.argmax(po.sub_n))} |
                  set(int(j) for j in rng.choice(sysm.n_mol, size=62, replace=False)))
    wref = orc.energy_weighted(sysm, orc.solve(sysm, m.mu, subs=subs, plan=po))
    err = w_error(po, wref, W, subs)
    tol = 2.0 * a_norm(sysm, po, subs) * TOL_D["bf16x3"]
    print(f"full size bf16x3 after find_mu: sampled max|dW| = {err:.3e} (tolerance {tol:.2e})")
    assert err <= tol
    assert np.isfinite(tw)
    st = plan.stats()
    assert st["ms_energy_weighted"] > 0.0
