"""Pins of the surrogate-network oracle (oracle/mlp.py), no GPU needed.

* analytic gradients = central finite differences of the loss (independent of
  the backward code);
* Gibbs' inequality: the cross-entropy is minimal, equal to the entropy of t,
  when the softmax equals t;
* the first AdamW step is lr sign(g) (bias-corrected moments) plus decoupled
  weight decay lr wd W on the weight matrices only;
* a constant gradient makes every AdamW step lr sign(g) after the decay, a
  closed form over several steps (checks both moment recursions);
* training on a separable toy problem lowers the loss.
"""
import numpy as np

from oracle import mlp as M


def _data(rng, b, f):
    x = rng.normal(size=(b, f))
    t = rng.dirichlet(np.ones(M.NBINS), size=b)
    return x, t


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    params = M.init(6, 7, seed=1)
    for k in params:
        if k.startswith("b"):
            params[k] = rng.normal(scale=0.3, size=params[k].shape)
    x, t = _data(rng, 5, 6)
    g = M.backward(params, M.forward(params, x), t)
    eps = 1e-6
    for k in params:
        num = np.zeros_like(params[k])
        it = np.nditer(params[k], flags=["multi_index"])
        for _ in it:
            i = it.multi_index
            old = params[k][i]
            params[k][i] = old + eps
            lp = M.loss(M.forward(params, x), t)
            params[k][i] = old - eps
            lm = M.loss(M.forward(params, x), t)
            params[k][i] = old
            num[i] = (lp - lm) / (2 * eps)
        np.testing.assert_allclose(g[k], num, rtol=1e-5, atol=1e-8, err_msg=k)


def test_cross_entropy_minimum_is_the_entropy():
    rng = np.random.default_rng(2)
    params = M.init(4, 8, seed=3)
    t = rng.dirichlet(np.ones(M.NBINS), size=1)
    params["W3"][:] = 0.0
    params["b3"][:] = np.log(t[0])
    x = rng.normal(size=(1, 4))
    cache = M.forward(params, x)
    np.testing.assert_allclose(cache["p"], t, rtol=1e-12)
    ent = float(-(t * np.log(t)).sum())
    assert M.loss(cache, t) == np.float64(ent) or abs(M.loss(cache, t) - ent) < 1e-12
    params["b3"][0] += 0.3          # any other distribution costs more
    assert M.loss(M.forward(params, x), t) > ent
    np.testing.assert_allclose(M.forward(params, rng.normal(size=(9, 4)))["p"].sum(axis=1), 1.0,
                               rtol=1e-14)


def test_first_adamw_step_closed_form():
    rng = np.random.default_rng(4)
    params = M.init(3, 5, seed=5)
    for k in ("b1", "b2", "b3"):    # nonzero biases, so decay on them would show
        params[k] = rng.normal(size=params[k].shape)
    before = {k: v.copy() for k, v in params.items()}
    grads = {k: rng.normal(size=v.shape) for k, v in params.items()}
    lr, wd = 1e-2, 0.1
    M.adamw_step(params, grads, {}, step=1, lr=lr, weight_decay=wd, eps=1e-12)
    for k in params:
        decay = lr * wd * before[k] if k.startswith("W") else 0.0
        expect = before[k] - decay - lr * np.sign(grads[k])
        np.testing.assert_allclose(params[k], expect, rtol=1e-9, atol=1e-12)


def test_constant_gradient_adamw_steps_in_closed_form():
    """With the same gradient g every step, the bias-corrected moments are g
    and g^2 exactly at every step, so each step subtracts lr sign(g) after the
    decoupled decay: W_n = a^n W_0 - lr sign(g) (1 - a^n)/(1 - a), a = 1 - lr wd
    (biases: a = 1, so b_n = b_0 - n lr sign(g))."""
    rng = np.random.default_rng(7)
    params = M.init(3, 5, seed=8)
    for k in ("b1", "b2", "b3"):
        params[k] = rng.normal(size=params[k].shape)
    before = {k: v.copy() for k, v in params.items()}
    grads = {k: rng.normal(size=v.shape) for k, v in params.items()}
    lr, wd, n = 1e-2, 0.1, 6
    state = {}
    for step in range(1, n + 1):
        M.adamw_step(params, grads, state, step=step, lr=lr, weight_decay=wd, eps=1e-12)
    a = 1.0 - lr * wd
    for k in params:
        if k.startswith("W"):
            expect = a ** n * before[k] - lr * np.sign(grads[k]) * (1 - a ** n) / (1 - a)
        else:
            expect = before[k] - n * lr * np.sign(grads[k])
        np.testing.assert_allclose(params[k], expect, rtol=1e-9, atol=1e-12, err_msg=k)


def test_training_lowers_the_loss():
    rng = np.random.default_rng(6)
    x = rng.normal(size=(256, 4))
    logits = np.stack([x[:, 0], -x[:, 0], x[:, 1], 0 * x[:, 1], -x[:, 1]], axis=1)
    t = np.exp(logits) / np.exp(logits).sum(axis=1, keepdims=True)
    params = M.init(4, 32, seed=7)
    state = {}
    l0 = M.loss(M.forward(params, x), t)
    for step in range(1, 301):
        cache = M.forward(params, x)
        M.adamw_step(params, M.backward(params, cache, t), state, step, lr=3e-3)
    l1 = M.loss(M.forward(params, x), t)
    ent = float(-(t * np.log(t)).sum(axis=1).mean())
    assert l1 < l0 and l1 - ent < 0.1 * (l0 - ent)
