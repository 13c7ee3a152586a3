"""FP64 oracle of the surrogate network -- plain numpy, written out.

TEST INFRASTRUCTURE ONLY (same rule as ``oracle.py``).  The surrogate is not
in the paper: it maps a patient's parameters and the controller's gains to
the five time-in-range fractions (Sec. IV-A) that the closed-loop simulation
(Sec. III) would produce, so that many controller tunings (the hyperparameters
p_kappa, p_mu of Eq. 3) can be screened before the full simulation picks the
best.

Network: features x (F) -> Z1 = x W1^T + b1, H1 = relu(Z1) -> Z2 = H1 W2^T + b2,
H2 = relu(Z2) -> Z3 = H2 W3^T + b3, p = softmax(Z3) over the 5 ranges.
Loss: mean over the batch of the cross-entropy -sum_i t_i log p_i against the
simulated fractions t.  Optimiser: AdamW (Loshchilov & Hutter) with bias
correction and decoupled weight decay on the weight matrices only.
"""
from __future__ import annotations

import numpy as np

NBINS = 5


def init(n_in: int, hidden: int, seed: int) -> dict:
    """He-uniform weights, zero biases (FP64)."""
    rng = np.random.default_rng(seed)

    def he(fan_out, fan_in):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, size=(fan_out, fan_in))

    return {"W1": he(hidden, n_in), "b1": np.zeros(hidden),
            "W2": he(hidden, hidden), "b2": np.zeros(hidden),
            "W3": he(NBINS, hidden), "b3": np.zeros(NBINS)}


def forward(params: dict, x: np.ndarray) -> dict:
    z1 = x @ params["W1"].T + params["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ params["W3"].T + params["b3"]
    zmax = z3.max(axis=1, keepdims=True)
    e = np.exp(z3 - zmax)
    p = e / e.sum(axis=1, keepdims=True)
    return {"x": x, "z1": z1, "h1": h1, "z2": z2, "h2": h2, "z3": z3, "p": p}


def loss(cache: dict, t: np.ndarray) -> float:
    return float(-(t * np.log(cache["p"])).sum(axis=1).mean())


def backward(params: dict, cache: dict, t: np.ndarray) -> dict:
    """Gradients of the mean cross-entropy, by the chain rule layer by layer."""
    b = t.shape[0]
    # d/dz3 of -sum t log softmax(z3) = p * sum(t) - t  (sum(t) = 1 for fractions)
    dz3 = (cache["p"] * t.sum(axis=1, keepdims=True) - t) / b
    g = {"W3": dz3.T @ cache["h2"], "b3": dz3.sum(axis=0)}
    dh2 = dz3 @ params["W3"]
    dz2 = dh2 * (cache["z2"] > 0)
    g["W2"] = dz2.T @ cache["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ params["W2"]
    dz1 = dh1 * (cache["z1"] > 0)
    g["W1"] = dz1.T @ cache["x"]
    g["b1"] = dz1.sum(axis=0)
    return g


def adamw_step(params: dict, grads: dict, state: dict, step: int, lr: float,
               beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
               weight_decay: float = 0.01) -> None:
    """In place; step counts from 1."""
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1.0 - beta1) * grads[k]
        v[...] = beta2 * v + (1.0 - beta2) * grads[k] * grads[k]
        mhat = m / (1.0 - beta1 ** step)
        vhat = v / (1.0 - beta2 ** step)
        if k.startswith("W"):
            params[k] -= lr * weight_decay * params[k]
        params[k] -= lr * mhat / (np.sqrt(vhat) + eps)


def predict(params: dict, x: np.ndarray) -> np.ndarray:
    return forward(params, x)["p"]
