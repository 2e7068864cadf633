"""Parity of the bound sources (power iteration, learned predictor) and of the predictor's network
(forward, gradient, Adam) with the FP64 CPU oracles, and the learned predictor's effect on a solve:
same densities, never an unconverged acceptance, fewer Newton-Schulz steps than the Gershgorin scale."""
import dataclasses

import numpy as np
import pytest

from oracle import bounds_oracle as bo
from oracle import mlp_oracle as mo
from oracle import nolsm_oracle as orc
from synth import make_system, spec_batched_uneven_4096

pytestmark = pytest.mark.gpu

MU = -0.35


@pytest.fixture(scope="module")
def nl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08245_gb300 import build
    build.build()
    import paper_2104_08245_gb300 as nl
    return nl


@pytest.fixture(scope="module")
def system():
    return make_system(spec_batched_uneven_4096())


@pytest.fixture(scope="module")
def oracle_plan(system):
    S, H = system.S, system.H
    return orc.build_plan(np.asarray(system.nbf), S.row_ptr, S.col_idx, H.row_ptr, H.col_idx)


def _oracle_A(system, plan_o, J):
    S, H = system.S, system.H
    tS = orc.gather(plan_o, J, S.row_ptr, S.col_idx, S.blk_off, S.vals)
    tH = orc.gather(plan_o, J, H.row_ptr, H.col_idx, H.blk_off, H.vals)
    return np.linalg.solve(tS, tH), tH


def _f32(p):
    return {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}


# ------------------------------------------------------------------------------------ network

def test_mlp_forward_matches_oracle(nl):
    import torch
    p = _f32(mo.init_params(seed=5))
    rng = np.random.default_rng(0)
    x = rng.normal(size=(1000, 7)).astype(np.float32)
    m = nl.Mlp(seed=1)
    m.set_params(mo.pack(p))
    y = m.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    y_ref, _ = mo.forward(p, x.astype(np.float64))
    err = float(np.max(np.abs(y - y_ref)))
    print(f"forward max|dy| = {err:.2e}")
    assert err <= 2e-5 * max(1.0, float(np.max(np.abs(y_ref))))


def test_mlp_gradient_matches_oracle(nl):
    import torch
    p = _f32(mo.init_params(seed=6))
    rng = np.random.default_rng(1)
    B = 1000   # 31 chunks of 32 and a ragged chunk of 8
    x = rng.normal(size=(B, 7)).astype(np.float32)
    t = rng.normal(size=(B, 3)).astype(np.float32)
    m = nl.Mlp(seed=1)
    m.set_params(mo.pack(p))
    g, loss = m.gradient(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    y, cache = mo.forward(p, x.astype(np.float64))
    g_ref = mo.backward(p, cache, y, t.astype(np.float64))
    loss_ref = mo.loss(y, t.astype(np.float64))
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    gu = mo.unpack(g)
    for k in mo.ORDER:
        scale = max(float(np.max(np.abs(g_ref[k]))), 1e-6)
        err = float(np.max(np.abs(gu[k] - g_ref[k])))
        print(f"grad {k}: max abs err {err:.2e} (scale {scale:.2e})")
        assert err <= 2e-5 * scale + 1e-7


def test_adam_step_matches_oracle(nl):
    import torch
    p = _f32(mo.init_params(seed=7))
    rng = np.random.default_rng(2)
    x = torch.from_numpy(rng.normal(size=(300, 7)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.normal(size=(300, 3)).astype(np.float32)).cuda()
    m = nl.Mlp(seed=1)
    m.set_params(mo.pack(p))
    state = {}
    ref = {k: v.copy() for k, v in p.items()}
    for _ in range(3):
        g, _ = m.gradient(x, t)
        m.adam_step(1e-3)
        mo.adam_step(ref, mo.unpack(g.astype(np.float64)), state, lr=1e-3)
    got = mo.unpack(m.get_params())
    for k in mo.ORDER:
        err = float(np.max(np.abs(got[k] - ref[k])))
        assert err <= 1e-6, (k, err)


def test_mlp_init_is_glorot(nl):
    m = nl.Mlp(seed=123)
    p = mo.unpack(m.get_params())
    for k, (fi, fo) in {"W1": (7, 128), "W2": (128, 128), "W3": (128, 3)}.items():
        lim = np.sqrt(6.0 / (fi + fo))
        w = p[k]
        assert np.all(np.abs(w) <= lim) and abs(float(np.mean(w))) < 0.1 * lim
        assert float(np.var(w)) == pytest.approx(lim * lim / 3.0, rel=0.15)
    for k in ("b1", "b2", "b3"):
        assert np.all(p[k] == 0.0)
    assert not np.array_equal(m.get_params(), nl.Mlp(seed=124).get_params())


def test_mlp_training_fits_a_teacher(nl):
    import torch
    rng = np.random.default_rng(3)
    x = rng.normal(size=(4096, 7)).astype(np.float32)
    A = rng.normal(size=(7, 16)) / np.sqrt(7)
    Bm = rng.normal(size=(16, 3)) / 4
    t = (np.tanh(x @ A) @ Bm).astype(np.float32)
    m = nl.Mlp(seed=9)
    losses = m.train(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), epochs=30, batch=256, lr=3e-3)
    print("training loss", losses[0], "->", losses[-1])
    assert losses[-1] < 0.05 * losses[0]


# ------------------------------------------------------------------------------------ features and bounds

@pytest.fixture(scope="module")
def plan(nl, system):
    return nl.nolsm_build_submatrices(nl.DeviceSystem(system))


def test_features_match_oracle(nl, system, oracle_plan, plan):
    f = nl.nolsm_features(plan, MU, nl.options("fp32")).cpu().numpy()
    rng = np.random.default_rng(4)
    for J in rng.choice(system.n_mol, 24, replace=False):
        A, tH = _oracle_A(system, oracle_plan, int(J))
        n_nb = int(oracle_plan.nb_ptr[J + 1] - oracle_plan.nb_ptr[J])
        ref = mo.features(A, tH, n_nb, MU)
        got = f[J]
        assert got[0] == pytest.approx(ref[0], rel=1e-6) and got[3] == pytest.approx(ref[3], rel=1e-6)
        assert got[6] == pytest.approx(ref[6], rel=1e-6)
        assert got[4] == pytest.approx(ref[4], rel=1e-5, abs=1e-6)
        assert got[5] == pytest.approx(ref[5], rel=1e-4, abs=1e-6)
        scale = max(abs(ref[1]), abs(ref[2]))
        assert abs(got[1] - ref[1]) <= 3e-5 * scale and abs(got[2] - ref[2]) <= 3e-5 * scale


def test_power_bounds_match_oracle_and_contain_spectrum(nl, system, oracle_plan, plan):
    o = nl.options("fp32")
    lam_p = nl.nolsm_power_bounds(plan, o).cpu().numpy()
    f = nl.nolsm_features(plan, MU, o).cpu().numpy()
    rng = np.random.default_rng(5)
    for J in rng.choice(system.n_mol, 16, replace=False):
        A, _ = _oracle_A(system, oracle_plan, int(J))
        lo_g, hi_g = float(f[J, 1]), float(f[J, 2])      # the library's Gershgorin interval as the shift
        ref = bo.power_bounds(A, lo_g, hi_g, iters=30)
        w = ref[1] - ref[0]
        assert abs(lam_p[J, 0] - ref[0]) <= 1e-4 * w and abs(lam_p[J, 1] - ref[1]) <= 1e-4 * w
        ev = np.linalg.eigvals(A).real
        assert lam_p[J, 0] <= ev.min() + 1e-6 and lam_p[J, 1] >= ev.max() - 1e-6
        assert lam_p[J, 1] - lam_p[J, 0] < hi_g - lo_g


def _solve(nl, plan, bound, mu=MU):
    plan.stats_reset()
    r = nl.nolsm_solve_batch(plan, mu, nl.options("fp32", bound_source=bound))
    return r, plan.scatter().cpu().numpy(), plan.stats()


def test_power_source_same_density_fewer_steps(nl, plan):
    r_g, D_g, _ = _solve(nl, plan, nl.BOUND_GERSHGORIN)
    r_p, D_p, st = _solve(nl, plan, nl.BOUND_POWER)
    assert np.all(r_p.sub_status.cpu().numpy() == 0)
    diff = float(np.max(np.abs(D_p - D_g)))
    it_g, it_p = r_g.iters.cpu().numpy().mean(), r_p.iters.cpu().numpy().mean()
    print(f"power vs Gershgorin: max|dD| {diff:.2e}, mean steps {it_p:.2f} vs {it_g:.2f}, reruns {st['reruns']}")
    assert diff <= 2e-6
    assert it_p < it_g
    assert abs(r_p.trace_DS - r_g.trace_DS) <= 1e-6 * abs(r_g.trace_DS)


def test_untrained_network_is_never_accepted_unconverged(nl, plan):
    m = nl.Mlp(seed=0)
    m.set_params(np.zeros(nl.MLP_PARAMS, dtype=np.float32))   # predicts a zero-width interval and 0 steps
    nl.nolsm_plan_set_mlp(plan, m)
    r_g, D_g, _ = _solve(nl, plan, nl.BOUND_GERSHGORIN)
    r_m, D_m, st = _solve(nl, plan, nl.BOUND_MLP)
    nl.nolsm_plan_set_mlp(plan, None)
    print(f"zero network: reruns {st['reruns']}, max|dD| {float(np.max(np.abs(D_m - D_g))):.2e}")
    assert np.all(r_m.sub_status.cpu().numpy() == 0)
    assert st["reruns"] > 0
    assert float(np.max(np.abs(D_m - D_g))) <= 2e-6


def test_trained_network_saves_steps_on_fresh_molecules(nl, system, plan):
    import torch
    o = nl.options("fp32")
    xs, ts = [], []
    for mu in (-0.45, -0.40, -0.35, -0.30, -0.25):
        x, t = nl.nolsm_training_data(plan, mu, o)
        xs.append(x)
        ts.append(t)
    x = torch.cat(xs)
    t = torch.cat(ts)
    m = nl.Mlp(seed=11)
    losses = m.train(x, t, epochs=60, batch=512, lr=2e-3)
    print(f"training on {x.shape[0]} samples: loss {losses[0]:.3e} -> {losses[-1]:.3e}")
    assert losses[-1] < 0.1 * losses[0]
    fresh = make_system(dataclasses.replace(spec_batched_uneven_4096(), seed=2012))
    p2 = nl.nolsm_build_submatrices(nl.DeviceSystem(fresh))
    nl.nolsm_plan_set_mlp(p2, m)
    r_g, D_g, _ = _solve(nl, p2, nl.BOUND_GERSHGORIN)
    r_p, _, _ = _solve(nl, p2, nl.BOUND_POWER)
    r_m, D_m, st = _solve(nl, p2, nl.BOUND_MLP)
    it_g, it_m = r_g.iters.cpu().numpy().mean(), r_m.iters.cpu().numpy().mean()
    it_p = r_p.iters.cpu().numpy().mean()
    diff = float(np.max(np.abs(D_m - D_g)))
    # the power-iteration interval (its own fallback) takes fewer steps still: the network's gain is over the
    # interval that needs no extra kernel, not over the power iteration (reported, not asserted)
    print(f"fresh molecules: mean steps learned {it_m:.3f} vs Gershgorin {it_g:.3f} vs power {it_p:.3f}, "
          f"reruns {st['reruns']}, max|dD| {diff:.2e}")
    assert np.all(r_m.sub_status.cpu().numpy() == 0)
    assert diff <= 2e-6
    assert it_m < it_g
    assert st["reruns"] <= 0.05 * fresh.n_mol
