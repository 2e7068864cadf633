"""Matrix elements generated on the device from the geometry (Sec. "Minimization of Communication").

A plan built from the block patterns alone (no S or H0 values on the device) with nolsm_plan_set_elements
generates T_J(S) and T_J(H0) from the positions, the cell, the on-site energies and the synthetic model's
parameters. It must give what the same plan gives from the stored block-CSR values that synth/ computed
with the same formula in numpy: the prepared FP64 A_J and the centre columns of T_J(S)^-1 within a few
units of FP64 rounding (the two sides round exp differently by at most an ulp or two; everything else is
evaluated in the same order), and the density of the FP64 and tensor-core paths against the FP64 oracle at
each path's tolerance. Variants: the direction modulation with different S and H0 cutoffs (the two
patterns differ, so presence must come from each pattern), and molecules with 6 or 23 functions."""
import numpy as np
import pytest

from oracle import nolsm_oracle as orc
from synth import SystemSpec, make_system, spec_small_fp64

pytestmark = pytest.mark.gpu

CASES = {
    "water64": spec_small_fp64(),
    "aniso_cutoffs": spec_small_fp64(aniso=0.3, cutoff_h=5.0, seed=11),
    "mixed_nbf": SystemSpec(3, 3, 3, nbf="mixed", cutoff=4.5, seed=13),
}


@pytest.fixture(scope="module")
def nl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08245_gb300 import build
    build.build()
    import paper_2104_08245_gb300 as nl
    return nl


def generated_plan(nl, sysm):
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm, values=False))
    nl.nolsm_plan_set_elements(plan, nl.ElementModel(sysm))
    return plan


@pytest.mark.parametrize("name", list(CASES))
def test_generated_elements_prepare_like_the_stored_ones(nl, name):
    sysm = make_system(CASES[name])
    gen = generated_plan(nl, sysm)
    ref = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    o = nl.options("fp64")
    A_g, Q_g, ps_g, _ = nl.nolsm_plan_get_prepared(gen, o)
    A_r, Q_r, ps_r, _ = nl.nolsm_plan_get_prepared(ref, o)
    assert np.array_equal(ps_g.cpu().numpy(), ps_r.cpu().numpy())
    eA = float((A_g - A_r).abs().max() / A_r.abs().max())
    eQ = float((Q_g - Q_r).abs().max() / Q_r.abs().max())
    print(f"{name}: generated vs stored elements: max|dA|/max|A| = {eA:.2e}, max|dQ|/max|Q| = {eQ:.2e}")
    assert eA <= 1e-13 and eQ <= 1e-13


@pytest.mark.parametrize("name", list(CASES))
def test_generated_elements_solve_to_the_oracle(nl, name):
    sysm = make_system(CASES[name])
    po = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    import scipy.linalg
    ev = []
    for J in range(sysm.n_mol):
        S = orc.gather(po, J, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
        H = orc.gather(po, J, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
        ev.append(scipy.linalg.eigh(H, S, eigvals_only=True))
    ev = np.concatenate(ev)
    mu = max(np.linspace(-0.6, 0.1, 15), key=lambda m: float(np.min(np.abs(ev - m))))   # away from eigenvalues
    ref = orc.solve(sysm, mu, plan=po)
    gen = generated_plan(nl, sysm)
    for prec, tol in (("fp64", 1e-9), ("fp32", 1e-6), ("bf16x3", 1e-4)):
        r = nl.nolsm_solve_batch(gen, mu, nl.options(prec))
        D = gen.scatter().cpu().numpy()
        err = float(np.max(np.abs(D - ref.D_vals)))
        print(f"{name} {prec}, generated elements: max|dD| = {err:.3e}")
        assert err <= tol * max(1.0, float(np.max(np.abs(ref.D_vals))))
        assert abs(r.trace_DS - ref.trace_DS) <= max(tol, 1e-12) * abs(ref.trace_DS) * 10
        assert np.all(r.sub_status.cpu().numpy() == 0)


def test_generated_elements_drive_the_learned_features(nl):
    """The on-site statistics of the learned predictor's features come from the model's on-site energies."""
    sysm = make_system(spec_small_fp64())
    gen = generated_plan(nl, sysm)
    ref = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    o = nl.options("bf16x3")
    fg = nl.nolsm_features(gen, -0.1, o)
    fr = nl.nolsm_features(ref, -0.1, o)
    assert float((fg - fr).abs().max()) <= 1e-6


def test_a_plan_without_values_needs_a_model(nl):
    sysm = make_system(spec_small_fp64())
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm, values=False))
    with pytest.raises(nl.NolsmError) as e:
        nl.nolsm_solve_batch(plan, -0.1, nl.options("fp64"))
    assert e.value.status == nl._abi.ERR_ARG
