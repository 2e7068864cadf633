"""Parity of the tensor-core (tcgen05) sign-iteration path with the FP64 CPU oracle.

Tolerances come from the workload targets: the FP32 mode (three-term FP16 split, about 22 bits)
max|dD| <= 1e-6; the BF16X3 and plain FP16 modes max|dD| <= 1e-4 with relative Tr(DH) error <= 1e-5. The plain BF16
and FP8 modes cannot reach 1e-4 (a rounding error made in any step persists in the occupied-virtual
block of the sign, and their 8 and 4 significant bits leave too much of it: the CPU pin of
tests/test_precision_readings.py): their measured errors are held to about twice the values measured on
GB300 (regressions fail), and the 1e-4 target itself is a strict expected failure for them."""
import numpy as np
import pytest

from oracle import nolsm_oracle as orc
from synth import SystemSpec, make_system, spec_small_fp64

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-6, "bf16x3": 1e-4, "fp16": 1e-4}
TOL_TR_DH = 1e-5


@pytest.fixture(scope="module")
def nl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08245_gb300 import build
    build.build()
    import paper_2104_08245_gb300 as nl
    return nl


def d_error(plan_o, ref, D, subs=None):
    """max|dD| over the blocks of D written by the listed submatrices (all if None)."""
    if subs is None:
        return float(np.max(np.abs(D - ref.D_vals)))
    off = orc.d_block_offsets(plan_o)
    err = 0.0
    for J in subs:
        cols = ref.subs[J].D_cols
        bJ = int(plan_o.nbf[J])
        for p in range(plan_o.nb_ptr[J], plan_o.nb_ptr[J + 1]):
            I = int(plan_o.nb_idx[p])
            bI = int(plan_o.nbf[I])
            q = plan_o.nb_ptr[I] + int(np.nonzero(plan_o.nb_idx[plan_o.nb_ptr[I]:plan_o.nb_ptr[I + 1]] == J)[0][0])
            got = D[off[q]:off[q + 1]].reshape(bI, bJ)
            err = max(err, float(np.max(np.abs(got - cols[plan_o.nb_off[p]:plan_o.nb_off[p] + bI, :]))))
    return err


@pytest.fixture(scope="module")
def small_ref():
    sysm = make_system(spec_small_fp64())
    return sysm, orc.solve(sysm, -0.1)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fp16"])
def test_split_modes_match_oracle(nl, small_ref, prec):
    sysm, ref = small_ref
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    r = nl.nolsm_solve_batch(plan, -0.1, nl.options(prec))
    D = plan.scatter().cpu().numpy()
    err = d_error(None, ref, D)
    print(f"{prec}: max|dD| = {err:.3e}")
    assert err <= TOL[prec]
    assert abs(r.trace_DH - ref.trace_DH) / abs(ref.trace_DH) <= TOL_TR_DH
    assert abs(r.trace_DS - ref.trace_DS) / abs(ref.trace_DS) <= TOL_TR_DH
    assert np.all(r.sub_status.cpu().numpy() == 0)
    steps = np.array([ref.subs[J].steps for J in range(sysm.n_mol)])
    it = r.iters.cpu().numpy()
    assert np.all(it >= steps - 2) and np.all(it <= steps + 4)


def test_plain_bf16_is_reported_not_hidden(nl, small_ref):
    sysm, ref = small_ref
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    r = nl.nolsm_solve_batch(plan, -0.1, nl.options("bf16"))
    D = plan.scatter().cpu().numpy()
    err = d_error(None, ref, D)
    print(f"bf16 + 2 refinement steps: max|dD| = {err:.3e}")
    assert 1e-6 < err < 3e-4          # measured on GB300: 1.2e-4
    assert np.all(r.sub_status.cpu().numpy() == 0)


def fp8_report(nl, sysm, ref, mu, po=None, subs=None):
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    r = nl.nolsm_solve_batch(plan, mu, nl.options("fp8e4m3"))
    D = plan.scatter().cpu().numpy()
    err = d_error(po, ref, D, subs)
    it = r.iters.cpu().numpy()
    assert np.all(r.sub_status.cpu().numpy() == 0)
    return r, err, it


def test_fp8_mode_is_reported_not_hidden(nl, small_ref):
    """E4M3 products (symmetric form, 2^7 operand scale) until the defect reaches 0.1, then three
    FP32-mode steps. The E4M3 rounding of the iterates persists like the BF16 one, 5 bits coarser
    (measured on GB300: max|dD| 4.9e-3, relative Tr(DH) 1.7e-5, 8 steps like the FP64 oracle)."""
    sysm, ref = small_ref
    r, err, it = fp8_report(nl, sysm, ref, -0.1)
    rel = abs(r.trace_DH - ref.trace_DH) / abs(ref.trace_DH)
    print(f"fp8e4m3 + 3 refinement steps: max|dD| = {err:.3e}, rel Tr(DH) = {rel:.3e}, "
          f"steps {it.min()}..{it.max()}")
    assert 1e-6 < err < 1e-2          # measured on GB300: 4.9e-3
    assert rel < 5e-5                 # measured: 1.7e-5
    steps = np.array([ref.subs[J].steps for J in range(sysm.n_mol)])
    assert np.all(it <= steps + 3)


def test_fp8_mode_larger_than_one_tile(nl):
    """n about 430: four 128-byte K slices, column blocks of 256 + 192, the ping-pong X planes."""
    sysm = make_system(SystemSpec(6, 6, 6, cutoff=8.0, seed=17))
    po = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    subs = [0, 37, 101, 215]
    ref = orc.solve(sysm, -0.1, subs=subs, plan=po)
    _, err, it = fp8_report(nl, sysm, ref, -0.1, po, subs)
    print(f"n~430 fp8e4m3: max|dD| = {err:.3e}, steps {it.min()}..{it.max()}")
    assert err < 2e-2


def test_fp8_mode_full_size_sampled(nl):
    """4,096 molecules of the uneven workload (n = 138..240: K padding from n64 up to whole 128-byte
    slices), 24 sampled submatrices against the oracle."""
    from synth import spec_batched_uneven_4096
    sysm = make_system(spec_batched_uneven_4096())
    po = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    rng = np.random.default_rng(9)
    subs = sorted(int(j) for j in rng.choice(sysm.n_mol, size=24, replace=False))
    ref = orc.solve(sysm, -0.35, subs=subs, plan=po)
    r, err, it = fp8_report(nl, sysm, ref, -0.35, po, subs)
    tH = r.sub_t_H.cpu().numpy()
    rel = max(abs(tH[J] - ref.subs[J].t_H) / abs(ref.subs[J].t_H) for J in subs)
    print(f"full size fp8e4m3: sampled max|dD| = {err:.3e}, max rel t_H = {rel:.3e}, "
          f"mean steps {it.mean():.2f}")
    # measured on GB300: 2.9e-2 and 3.4e-3 (the E4M3 floor, amplified by the overlap's conditioning)
    assert err < 6e-2
    assert rel < 7e-3


@pytest.mark.xfail(strict=True, reason="out of reach by the analysis pinned in test_precision_readings.py: "
                   "measured max|dD| 1.7e-4 (plain BF16) and 1.6e-2 (E4M3) on 96 sampled submatrices of the "
                   "262,144-molecule workload")
@pytest.mark.parametrize("prec", ["bf16", "fp8e4m3"])
def test_the_1e4_target_is_out_of_reach_for(nl, prec):
    """The workload's max|dD| <= 1e-4 target for the single-product 8-bit-mantissa modes, on 64 sampled
    submatrices of the 4,096-molecule uneven system: expected to fail (strict)."""
    from synth import spec_batched_uneven_4096
    sysm = make_system(spec_batched_uneven_4096())
    po = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    rng = np.random.default_rng(21)
    subs = sorted(int(j) for j in rng.choice(sysm.n_mol, size=64, replace=False))
    ref = orc.solve(sysm, -0.35, subs=subs, plan=po)
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    nl.nolsm_solve_batch(plan, -0.35, nl.options(prec))
    err = d_error(po, ref, plan.scatter().cpu().numpy(), subs)
    print(f"{prec}: sampled max|dD| = {err:.3e} against the 1e-4 target")
    assert err <= 1e-4


def test_fp8_needs_refinement_and_symmetric_form(nl, small_ref):
    sysm, _ = small_ref
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    with pytest.raises(nl.NolsmError) as e:
        nl.nolsm_solve_batch(plan, -0.1, nl.options("fp8e4m3", refine_steps=0))
    assert e.value.status == nl._abi.ERR_UNSUPPORTED


VARIANTS = {
    "aniso_cutoffs": spec_small_fp64(aniso=0.3, cutoff_h=5.0, seed=11),
    "mixed_nbf": SystemSpec(3, 3, 3, nbf="mixed", cutoff=4.5, seed=13),
    "isolated": SystemSpec(3, 3, 2, cutoff=1.5, seed=14),
    "one_molecule": SystemSpec(1, 1, 1, seed=15),
}


def well_separated_mu(sysm, candidates):
    """The candidate mu farthest from every submatrix eigenvalue (LAPACK generalized eigensolver):
    these tests check arithmetic, so they avoid the ill-conditioned sign near an eigenvalue."""
    import scipy.linalg
    po = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    ev = []
    for J in range(sysm.n_mol):
        S = orc.gather(po, J, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
        H = orc.gather(po, J, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
        ev.append(scipy.linalg.eigh(H, S, eigvals_only=True))
    ev = np.concatenate(ev)
    return max(candidates, key=lambda m: float(np.min(np.abs(ev - m))))


@pytest.mark.parametrize("name", list(VARIANTS))
def test_fp32_mode_variants(nl, name):
    sysm = make_system(VARIANTS[name])
    mu = well_separated_mu(sysm, np.linspace(-0.6, 0.1, 15))
    ref = orc.solve(sysm, mu)
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    r = nl.nolsm_solve_batch(plan, mu, nl.options("fp32"))
    D = plan.scatter().cpu().numpy()
    err = d_error(None, ref, D)
    print(f"{name}: fp32-mode max|dD| = {err:.3e}")
    assert err <= 1e-6 * max(1.0, float(np.max(np.abs(ref.D_vals))))
    assert abs(r.trace_DS - ref.trace_DS) <= 1e-6 * abs(ref.trace_DS)


def test_submatrices_larger_than_one_tile(nl):
    """n about 430 (8 A cutoff): 4 row blocks of 128 and column blocks of 256 + 192."""
    sysm = make_system(SystemSpec(6, 6, 6, cutoff=8.0, seed=17))
    mu = -0.1
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    info = plan.info()
    assert info.max_n > 256
    r = nl.nolsm_solve_batch(plan, mu, nl.options("fp32"))
    D = plan.scatter().cpu().numpy()
    po = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    subs = [0, 37, 101, 215]
    ref = orc.solve(sysm, mu, subs=subs, plan=po)
    err = d_error(po, ref, D, subs)
    print(f"n~{info.max_n}: fp32-mode max|dD| = {err:.3e}")
    # the 1e-6 target is stated for n up to 300; rounding errors of the products grow like sqrt(n)
    assert err <= 1e-6 * np.sqrt(info.max_n / 300.0)
    tS = r.sub_t_S.cpu().numpy()
    for J in subs:
        assert tS[J] == pytest.approx(ref.subs[J].t_S, rel=1e-6)


def test_full_size_sampled(nl):
    """32,768 molecules with the density field, every submatrix in one launch (the benchmark's
    launch configuration); 512 sampled submatrices (the smallest and largest among them) against the
    oracle."""
    from synth import spec_batched_uneven
    sysm = make_system(spec_batched_uneven())
    mu = -0.1
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    po = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    rng = np.random.default_rng(7)
    subs = set(int(j) for j in rng.choice(sysm.n_mol, size=510, replace=False))
    subs |= {int(np.argmax(po.sub_n)), int(np.argmin(po.sub_n))}
    subs = sorted(subs)
    ref = orc.solve(sysm, mu, subs=subs, plan=po)
    for prec in ("fp32", "bf16x3", "fp16"):
        r = nl.nolsm_solve_batch(plan, mu, nl.options(prec))
        D = plan.scatter().cpu().numpy()
        err = d_error(po, ref, D, subs)
        tH = r.sub_t_H.cpu().numpy()
        rel = max(abs(tH[J] - ref.subs[J].t_H) / abs(ref.subs[J].t_H) for J in subs)
        print(f"full size {prec}: sampled max|dD| = {err:.3e}, max rel t_H = {rel:.3e}")
        assert err <= TOL[prec]
        assert rel <= TOL_TR_DH
        assert np.all(r.sub_status.cpu().numpy() == 0)


def test_not_spd_reported_on_tensor_path(nl):
    sysm = make_system(spec_small_fp64())
    p = int(np.nonzero(sysm.S.col_idx[sysm.S.row_ptr[5]:sysm.S.row_ptr[6]] == 5)[0][0]) + sysm.S.row_ptr[5]
    sysm.S.vals[sysm.S.blk_off[p]:sysm.S.blk_off[p + 1]] *= -1.0
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    r = nl.nolsm_solve_batch(plan, -0.1, nl.options("bf16x3"), check=False)
    assert r.status == nl._abi.ERR_NOT_SPD
    assert np.sum(r.sub_status.cpu().numpy() == nl._abi.ERR_NOT_SPD) > 0


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_symmetric_form_matches_oracle(nl, small_ref, prec):
    """The symmetric form M = L^-1 T_J(H0) L^-T (same spectrum, symmetric iterates, D_c = L^-T U) gives
    the same densities as the standard form within the mode's tolerance."""
    sysm, ref = small_ref
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    r = nl.nolsm_solve_batch(plan, -0.1, nl.options(prec, symmetric_form=1))
    D = plan.scatter().cpu().numpy()
    err = d_error(None, ref, D)
    print(f"{prec} symmetric form: max|dD| = {err:.3e}")
    assert err <= TOL[prec]
    assert abs(r.trace_DH - ref.trace_DH) / abs(ref.trace_DH) <= TOL_TR_DH
    assert abs(r.trace_DS - ref.trace_DS) / abs(ref.trace_DS) <= TOL_TR_DH
    assert np.all(r.sub_status.cpu().numpy() == 0)


def test_symmetric_form_full_size_sampled(nl):
    from synth import spec_batched_uneven_4096
    sysm = make_system(spec_batched_uneven_4096())
    mu = -0.35
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    po = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    rng = np.random.default_rng(8)
    subs = sorted(int(j) for j in rng.choice(sysm.n_mol, size=24, replace=False))
    ref = orc.solve(sysm, mu, subs=subs, plan=po)
    r = nl.nolsm_solve_batch(plan, mu, nl.options("fp32", symmetric_form=1))
    D = plan.scatter().cpu().numpy()
    err = d_error(po, ref, D, subs)
    print(f"symmetric form, 4096 molecules: sampled max|dD| = {err:.3e}")
    assert err <= TOL["fp32"]
    assert np.all(r.sub_status.cpu().numpy() == 0)


def test_split_valence_sampled(nl):
    """512 molecules with 23 functions each: n = 598..713, so five or six row blocks, three column tiles,
    up to twelve K slices, the ping-pong X planes, and three column groups of b in the centre-column
    phase. mu from the GPU bisection; 6 sampled submatrices against the oracle at that mu in the FP32,
    BF16X3 and E4M3 modes."""
    sysm = make_system(SystemSpec(8, 8, 8, nbf="23", seed=1104))
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    po = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    m = plan.find_mu(float(np.sum(sysm.occ)), 0.0, 0.0, nl.options("fp32"))
    rng = np.random.default_rng(11)
    subs = sorted({int(np.argmin(po.sub_n)), int(np.argmax(po.sub_n))} |
                  set(int(j) for j in rng.choice(sysm.n_mol, size=4, replace=False)))
    ref = orc.solve(sysm, m.mu, subs=subs, plan=po)
    n_max = int(po.sub_n.max())
    for prec, tol in (("fp32", 1e-6 * np.sqrt(n_max / 300.0)), ("bf16x3", 1e-4), ("fp8e4m3", 1e-2)):
        r = nl.nolsm_solve_batch(plan, m.mu, nl.options(prec))
        D = plan.scatter().cpu().numpy()
        err = d_error(po, ref, D, subs)
        it = r.iters.cpu().numpy()
        print(f"23 functions, n {po.sub_n.min()}..{n_max}, mu {m.mu:.4f}: {prec} sampled max|dD| = {err:.3e}, "
              f"steps {it.min()}..{it.max()}")
        assert err <= tol
        assert np.all(r.sub_status.cpu().numpy() == 0)


def test_split_valence_n_above_900(nl):
    """23 functions per molecule with a 6.8 A cutoff: n = 805..1058 (the 700-1000 span of the split-valence
    workload and past it): up to nine row blocks, five column tiles, seventeen K slices. mu from the GPU
    bisection; the smallest, the largest and two random submatrices against the oracle at that mu, in the
    FP32, BF16X3 and FP16 modes and in BF16X3 with the tensor-core inverse square root."""
    sysm = make_system(SystemSpec(8, 8, 8, nbf="23", cutoff=6.8, seed=1104))
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    po = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
    assert po.sub_n.max() >= 1000 and po.sub_n.min() >= 700
    m = plan.find_mu(float(np.sum(sysm.occ)), 0.0, 0.0, nl.options("bf16x3"))
    assert m.status == 0
    rng = np.random.default_rng(12)
    subs = sorted({int(np.argmin(po.sub_n)), int(np.argmax(po.sub_n))} |
                  set(int(j) for j in rng.choice(sysm.n_mol, size=2, replace=False)))
    ref = orc.solve(sysm, m.mu, subs=subs, plan=po)
    n_max = int(po.sub_n.max())
    for prec, inv, tol in (("fp32", 0, 1e-6 * np.sqrt(n_max / 300.0)), ("bf16x3", 0, 1e-4), ("fp16", 0, 1e-4),
                           ("bf16x3", 1, 1e-4)):
        r = nl.nolsm_solve_batch(plan, m.mu, nl.options(prec, inverse=inv))
        D = plan.scatter().cpu().numpy()
        err = d_error(po, ref, D, subs)
        it = r.iters.cpu().numpy()
        print(f"23 functions, n {po.sub_n.min()}..{n_max}, mu {m.mu:.4f}: {prec} (inverse {inv}) sampled "
              f"max|dD| = {err:.3e}, steps {it.min()}..{it.max()}")
        assert err <= tol
        assert np.all(r.sub_status.cpu().numpy() == 0)


def test_submatrix_ranges_are_bit_identical_on_tensor_path(nl):
    """Solving the system in two ranges (the streamed configuration's batches) gives, submatrix by
    submatrix, the same bits as one solve of every submatrix: each submatrix's arithmetic does not depend
    on the launch that carries it."""
    from synth import spec_batched_uneven_4096
    sysm = make_system(spec_batched_uneven_4096())
    mu = -0.35
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    nl.nolsm_solve_batch(plan, mu, nl.options("bf16x3"))
    D_all = plan.scatter().cpu().numpy()
    plan2 = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    half = sysm.n_mol // 2 + 7
    D_rng = None
    for j0, j1 in ((0, half), (half, sysm.n_mol)):   # each range written back after its solve
        r = nl.nolsm_solve_batch(plan2, mu, nl.options("bf16x3", sub_begin=j0, sub_end=j1))
        assert r.status == 0
        D_rng = plan2.scatter(D_rng)
    assert np.array_equal(D_all, D_rng.cpu().numpy())


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 1e-6)])
def test_find_mu_solves_only_bracketed_submatrices(nl, prec, tol):
    """A system without a common gap (6 and 23 functions mixed) makes the bisection take many points;
    from the second one on, only submatrices with an eigenvalue left in the bracket are solved. At the
    final mu the density is as close to the oracle's as a solve of every submatrix at that mu (kept
    blocks come from an earlier mu of the same bracket, where the same D holds)."""
    sysm = make_system(VARIANTS["mixed_nbf"])
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    plan.stats_reset()
    m = plan.find_mu(float(sysm.n_occ), 0.0, 0.0, nl.options(prec))
    solved = plan.stats()["sub_solves"]
    D = plan.scatter().cpu().numpy()
    plan2 = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    r = nl.nolsm_solve_batch(plan2, m.mu, nl.options(prec), check=False)
    D2 = plan2.scatter().cpu().numpy()
    ref = orc.solve(sysm, m.mu)
    e_kept = float(np.max(np.abs(D - ref.D_vals)))
    e_fresh = float(np.max(np.abs(D2 - ref.D_vals)))
    print(f"{prec}: {m.steps} bisection points, {solved} submatrix solves of {m.steps * sysm.n_mol}; "
          f"max|dD| {e_kept:.3e} (kept blocks) vs {e_fresh:.3e} (every block solved at the final mu)")
    assert m.steps > 2
    assert solved < m.steps * sysm.n_mol
    assert e_kept <= e_fresh + tol
    assert abs(m.trace_DS - ref.trace_DS) <= abs(r.trace_DS - ref.trace_DS) + tol * sysm.n_mol


def test_sharded_bisection_with_one_rank_matches_find_mu(nl):
    """The point-by-point bisection API (begin / point / side) driven by the multi-rank loop of
    sharded.py on a one-rank gloo group takes the same points, mu and Tr(DS) as nolsm_find_mu, and solves
    as few submatrices."""
    import torch.distributed as dist
    from paper_2104_08245_gb300.sharded import sharded_find_mu
    sysm = make_system(VARIANTS["mixed_nbf"])
    opts = nl.options("fp64")
    plan = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    plan.stats_reset()
    m = plan.find_mu(float(sysm.n_occ), 0.0, 0.0, opts)
    solved_single = plan.stats()["sub_solves"]
    D = plan.scatter().cpu().numpy()
    plan2 = nl.nolsm_build_submatrices(nl.DeviceSystem(sysm))
    plan2.stats_reset()
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:29531", rank=0, world_size=1)
    try:
        r = sharded_find_mu(plan2, float(sysm.n_occ), opts)
    finally:
        dist.destroy_process_group()
    solved_sharded = plan2.stats()["sub_solves"]
    D2 = plan2.scatter().cpu().numpy()
    print(f"{r.steps} points; solves {solved_sharded} (sharded loop) vs {solved_single} (find_mu)")
    assert r.history == m.history
    assert r.mu == m.mu and r.trace_DS == m.trace_DS
    assert solved_sharded == solved_single
    assert np.array_equal(D, D2)
