"""Pins of the FP64 MLP oracle: central finite differences of the loss (the definition of the
gradient), closed-form forward passes, Adam's first step, and spectral bounds from the features."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    p = mo.init_params(seed=1)
    x = rng.normal(size=(9, mo.N_FEATURES))
    t = rng.normal(size=(9, mo.N_OUT))
    y, cache = mo.forward(p, x)
    g = mo.backward(p, cache, y, t)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = mo.loss(mo.forward(p, x)[0], t)
            flat[idx] = old - h
            lm = mo.loss(mo.forward(p, x)[0], t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert g[k].reshape(-1)[idx] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_forward_closed_forms():
    p = mo.init_params(seed=2)
    for k in ("W1", "W2", "W3"):
        p[k][:] = 0.0
    p["b3"][:] = [1.5, -2.0, 0.25]
    y, _ = mo.forward(p, np.ones((4, mo.N_FEATURES)))
    assert np.array_equal(y, np.tile([1.5, -2.0, 0.25], (4, 1)))
    # one active path: x0 -> unit 0 -> unit 0 -> output 1
    p["W1"][0, 0] = 0.5
    p["W2"][0, 0] = 2.0
    p["W3"][0, 1] = 3.0
    x = np.zeros((1, mo.N_FEATURES))
    x[0, 0] = 0.8
    y, _ = mo.forward(p, x)
    assert y[0, 1] == pytest.approx(-2.0 + 3.0 * np.tanh(2.0 * np.tanh(0.4)), abs=1e-15)


def test_adam_first_step_moves_by_lr_times_sign():
    p = {"w": np.array([1.0, -1.0, 0.5])}
    g = {"w": np.array([0.3, -2.0, 1e-3])}
    st = {}
    mo.adam_step(p, g, st, lr=0.01, eps=1e-12)
    assert np.allclose(p["w"], [1.0 - 0.01, -1.0 + 0.01, 0.5 - 0.01], atol=1e-9)


def test_gershgorin_features_bound_the_spectrum():
    rng = np.random.default_rng(4)
    M = rng.normal(size=(30, 30))
    S = np.eye(30) + 0.05 * (M @ M.T) / 30
    H = 0.5 * (M + M.T)
    A = np.linalg.solve(S, H)
    f = mo.features(A, H, 5, -0.1)
    ev = np.linalg.eigvals(A).real
    assert f[1] <= ev.min() + 1e-12 and ev.max() <= f[2] + 1e-12
    assert f[0] == pytest.approx(0.3) and f[6] == -0.1
