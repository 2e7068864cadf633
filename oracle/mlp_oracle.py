"""FP64 CPU oracle of the learned spectral-bound predictor -- TEST INFRASTRUCTURE ONLY.

The predictor has no counterpart in the paper; the paper only requires that the matrix be rescaled
before the sign iteration (Sec. "Linear-Scaling Electronic Structure Calculations", after Eq. NS2) and
runs a fixed number of steps (Sec. "Efficient Iterative Matrix Function Solvers on GPU Tensor Cores").
The predictor supplies both per submatrix: spectral bounds of A = T_J(S)^-1 T_J(H0) and a step count.

Network: three dense layers, width 128, tanh after the first two, linear output:
    h1 = tanh(x W1 + b1), h2 = tanh(h1 W2 + b2), y = h2 W3 + b3
Weights are stored [fan_in, fan_out] row-major. Loss: L = 1/(2B) sum_b sum_o (y_bo - t_bo)^2.
Optimiser: Adam with bias correction.

Features of submatrix J (all cheap, O(n^2) at most), in this order:
    0: n_J / 100
    1: Gershgorin lower bound of A (min_i A_ii - sum_{j != i} |A_ij|)
    2: Gershgorin upper bound of A (max_i A_ii + sum_{j != i} |A_ij|)
    3: |N(J)| / 32                  (local density: molecules in the neighbourhood)
    4: mean of diag T_J(H0)
    5: standard deviation of diag T_J(H0)
Targets: lowest and highest eigenvalue of A, and the Newton-Schulz step count / 16 at the chemical
potential the step count was recorded at (which is appended as feature 6).
"""
from __future__ import annotations

import math

import numpy as np

N_FEATURES = 7
WIDTH = 128
N_OUT = 3


def init_params(n_in=N_FEATURES, width=WIDTH, n_out=N_OUT, seed=0) -> dict:
    """Glorot-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)

    def glorot(a, b):
        lim = math.sqrt(6.0 / (a + b))
        return rng.uniform(-lim, lim, size=(a, b))

    return {"W1": glorot(n_in, width), "b1": np.zeros(width),
            "W2": glorot(width, width), "b2": np.zeros(width),
            "W3": glorot(width, n_out), "b3": np.zeros(n_out)}


def forward(p: dict, x: np.ndarray):
    """Returns y and the activations needed by ``backward``."""
    h1 = np.tanh(x @ p["W1"] + p["b1"])
    h2 = np.tanh(h1 @ p["W2"] + p["b2"])
    y = h2 @ p["W3"] + p["b3"]
    return y, (x, h1, h2)


def loss(y: np.ndarray, t: np.ndarray) -> float:
    return float(0.5 * np.sum((y - t) ** 2) / y.shape[0])


def backward(p: dict, cache, y: np.ndarray, t: np.ndarray) -> dict:
    """Gradients of ``loss`` by the chain rule, layer by layer from the output."""
    x, h1, h2 = cache
    B = y.shape[0]
    dy = (y - t) / B
    g = {"W3": h2.T @ dy, "b3": dy.sum(axis=0)}
    dh2 = dy @ p["W3"].T
    dz2 = dh2 * (1.0 - h2 * h2)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"].T
    dz1 = dh1 * (1.0 - h1 * h1)
    g["W1"] = x.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_step(p: dict, g: dict, state: dict, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8) -> None:
    """One Adam update in place; ``state`` holds m, v and the step counter t."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m *= beta1
        m += (1.0 - beta1) * g[k]
        v *= beta2
        v += (1.0 - beta2) * g[k] * g[k]
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        p[k] -= lr * mhat / (np.sqrt(vhat) + eps)


def features(A: np.ndarray, H_sub: np.ndarray, n_nb: int, mu: float) -> np.ndarray:
    """Feature vector of one submatrix (order in the module docstring)."""
    d = np.diag(A)
    R = np.sum(np.abs(A), axis=1) - np.abs(d)
    hd = np.diag(H_sub)
    return np.array([A.shape[0] / 100.0, float(np.min(d - R)), float(np.max(d + R)), n_nb / 32.0,
                     float(np.mean(hd)), float(np.std(hd)), mu])


ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def pack(p: dict) -> np.ndarray:
    """Flat parameter vector in the library's order W1, b1, W2, b2, W3, b3 (row-major)."""
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in ORDER])


def unpack(flat, n_in=N_FEATURES, width=WIDTH, n_out=N_OUT) -> dict:
    shapes = {"W1": (n_in, width), "b1": (width,), "W2": (width, width), "b2": (width,),
              "W3": (width, n_out), "b3": (n_out,)}
    out, o = {}, 0
    flat = np.asarray(flat, dtype=np.float64)
    for k in ORDER:
        m = int(np.prod(shapes[k]))
        out[k] = flat[o:o + m].reshape(shapes[k]).copy()
        o += m
    assert o == flat.size
    return out
