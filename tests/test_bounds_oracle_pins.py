"""Pins of the bound-source oracle (power iteration, learned interval, guarded scale) against the
spectrum computed by LAPACK and against the Newton-Schulz map's own fixed-point behaviour."""
import math

import numpy as np
import pytest

from oracle import bounds_oracle as bo
from oracle import mlp_oracle as mo


def _sym(n, lo, hi, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    d = np.concatenate([[lo, hi], rng.uniform(lo + 0.3 * (hi - lo), hi - 0.3 * (hi - lo), size=n - 2)])
    return (Q * d) @ Q.T, lo, hi


def test_gershgorin_closed_form_and_containment():
    A = np.array([[1.0, -2.0], [0.5, 3.0]])
    assert bo.gershgorin(A) == (min(1 - 2, 3 - 0.5), max(1 + 2, 3 + 0.5))
    B, lo, hi = _sym(40, -1.3, 0.7, 1)
    g = bo.gershgorin(B)
    assert g[0] <= lo and g[1] >= hi


def test_power_bounds_contain_and_track_the_spectrum():
    B, lo, hi = _sym(60, -1.0, 0.4, 2)
    g = bo.gershgorin(B)
    plo, phi = bo.power_bounds(B, *g, iters=30)
    assert plo <= lo and phi >= hi                       # contains the spectrum
    assert g[0] <= plo and phi <= g[1]                   # clipped to Gershgorin
    w = hi - lo
    assert phi - plo <= 1.10 * w + 1e-9                  # 5 % widening on each side of near-exact estimates
    assert abs(plo - (lo - 0.05 * w)) < 0.02 * w and abs(phi - (hi + 0.05 * w)) < 0.02 * w


def test_power_bounds_on_a_generalised_pencil():
    # A = S^-1 H is not symmetric but similar to L^-1 H L^-T: real spectrum, same bounds
    rng = np.random.default_rng(3)
    n = 50
    M = rng.normal(size=(n, n)) * 0.05
    S = np.eye(n) + M @ M.T
    H, _, _ = _sym(n, -1.2, 0.5, 4)
    A = np.linalg.solve(S, H)
    ev = np.sort(np.linalg.eigvals(A).real)
    g = bo.gershgorin(A)
    plo, phi = bo.power_bounds(A, *g, iters=60)
    assert plo <= ev[0] + 1e-9 and phi >= ev[-1] - 1e-9


def test_learned_interval_mapping():
    (lo, hi), bud = bo.learned_interval([0.5, -1.0, 0.5], (-2.0, 2.0), 100)
    assert lo == pytest.approx(-1.0 - 0.015) and hi == pytest.approx(0.5 + 0.015)
    assert bud == math.ceil(1.5 * 8.0) + 3
    (lo, hi), bud = bo.learned_interval([-5.0, 5.0, 10.0], (-1.0, 1.0), 30)
    assert (lo, hi) == (-1.0, 1.0) and bud == 30        # clipped to Gershgorin, budget capped
    (lo, hi), bud = bo.learned_interval([0.0, 0.0, 0.0], (-1.0, 1.0), 100)
    assert lo < hi and bud == 4 + 1                      # degenerate width 1e-6, budget floor ceil(1.5) + 3


def _ns(X, steps):
    I = np.eye(X.shape[0])
    for _ in range(steps):
        X = 0.5 * X @ (3 * I - X @ X)
    return X


def test_guarded_scale_keeps_every_sign():
    B, lo, hi = _sym(30, -1.0, 0.8, 5)
    ev = np.linalg.eigvalsh(B)
    mu = -0.05
    g = bo.gershgorin(B)
    bad = (mu - 1e-3, mu + 1e-3)                         # a learned interval far too narrow
    a_raw = bo.alpha(bad, mu)
    a = bo.scale_alpha(bad, g, mu)
    assert a >= bo.alpha(g, mu) / 1.7
    assert np.max(np.abs(ev - mu)) / a < math.sqrt(3)    # every scaled eigenvalue inside (-sqrt3, sqrt3)
    X = _ns((B - mu * np.eye(30)) / a, 60)
    S_ref = np.sign(ev - mu)
    assert np.allclose(np.sort(np.linalg.eigvalsh(0.5 * (X + X.T))), np.sort(S_ref), atol=1e-8)
    # without the guard the same interval flips signs: the defect test alone would accept it
    with np.errstate(all="ignore"):
        X_bad = _ns((B - mu * np.eye(30)) / a_raw, 8)
    with np.errstate(all="ignore"):
        assert not np.all(np.isfinite(X_bad)) or not np.allclose(X_bad @ X_bad, np.eye(30), atol=1e-3) or \
            not np.allclose(np.sort(np.linalg.eigvalsh(0.5 * (X_bad + X_bad.T))), np.sort(S_ref), atol=1e-3)


def test_sign_flip_beyond_sqrt3():
    # the reason for the guard: x in (sqrt(3), sqrt(5)) maps to the other sign and can converge there
    x = np.array([[1.9]])
    X = _ns(x, 40)
    assert X[0, 0] == pytest.approx(-1.0, abs=1e-12)


def test_pack_unpack_roundtrip():
    p = mo.init_params(seed=3)
    flat = mo.pack(p)
    assert flat.size == 7 * 128 + 128 + 128 * 128 + 128 + 128 * 3 + 3 == 17923
    q = mo.unpack(flat)
    for k in p:
        assert np.array_equal(p[k], q[k])
