"""Pins of O3 (the proposal MLP in FP64) against what mathematics fixes.

* GELU against the normal distribution function (scipy.stats.norm.cdf, an
  independent library routine): GELU(z) = z Phi(z); GELU(z) - GELU(-z) = z;
  its derivative against central differences.
* Softmax cross-entropy: equal logits give log G; the gradient rows sum to 0.
* The full gradient against central finite differences of the loss, every
  parameter tensor, on a tiny network.
* Adam's first step moves every weight by lr * g / (|g| + eps) exactly.
* Training separates a toy problem of well-apart clusters.
* Planted mistakes (a dropped term, a wrong sign, a transposed operand, the
  tanh GELU) must each break one of these pins.
"""
import copy

import numpy as np
import pytest
from scipy.stats import norm

from oracle import mlp


def _tiny(seed=0, d=5, h=7, g=4, n=6):
    rng = np.random.default_rng(seed)
    params = mlp.init_params(d, h, g, seed)
    for k in params:  # non-zero biases so their gradients are exercised
        if k.startswith("b"):
            params[k] = rng.normal(0, 0.3, params[k].shape)
    X = rng.normal(0, 1.0, (n, d))
    y = rng.integers(0, g, n)
    return params, X, y


def _fd_check(mod, params, X, y, h=1e-6):
    _, g = mod.loss_and_grad(params, X, y)
    worst = 0.0
    for k in params:
        it = np.nditer(params[k], flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            p1 = copy.deepcopy(params)
            p2 = copy.deepcopy(params)
            p1[k][idx] += h
            p2[k][idx] -= h
            fd = (mod.loss_and_grad(p1, X, y)[0] - mod.loss_and_grad(p2, X, y)[0]) / (2 * h)
            worst = max(worst, abs(fd - g[k][idx]) / max(1e-6, abs(fd) + abs(g[k][idx])))
    return worst


def test_gelu_is_z_times_normal_cdf():
    z = np.linspace(-6, 6, 241)
    assert np.allclose(mlp.gelu(z), z * norm.cdf(z), rtol=1e-13, atol=1e-15)
    assert np.allclose(mlp.gelu(z) - mlp.gelu(-z), z, rtol=1e-13, atol=1e-14)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15


def test_gelu_derivative_central_differences():
    z = np.linspace(-5, 5, 101)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, rtol=1e-7, atol=1e-9)


def test_softmax_xent_closed_forms():
    G = 410
    loss, d = mlp.softmax_xent(np.zeros((3, G)), np.array([0, 5, 409]))
    assert abs(loss - np.log(G)) < 1e-12
    assert np.allclose(d.sum(axis=1), 0.0, atol=1e-15)
    # a confident correct prediction costs almost nothing
    lg = np.zeros((1, 4))
    lg[0, 2] = 50.0
    assert mlp.softmax_xent(lg, np.array([2]))[0] < 1e-20


def test_gradient_matches_finite_differences():
    params, X, y = _tiny()
    assert _fd_check(mlp, params, X, y) < 1e-6


def test_adam_first_step_closed_form():
    params, X, y = _tiny(seed=3)
    _, g = mlp.loss_and_grad(params, X, y)
    before = copy.deepcopy(params)
    st = mlp.adam_init(params)
    mlp.adam_step(params, g, st, lr=1e-3, eps=1e-8)
    for k in params:
        want = before[k] - 1e-3 * g[k] / (np.abs(g[k]) + 1e-8)
        assert np.allclose(params[k], want, rtol=1e-12, atol=1e-15), k


def test_learns_separable_clusters():
    rng = np.random.default_rng(5)
    G, d, n = 6, 4, 3000
    centres = rng.uniform(-10, 10, (G, d))
    y = rng.integers(0, G, n)
    X = centres[y] + rng.normal(0, 0.3, (n, d))
    params = mlp.train(X, y, hidden=32, classes=G, seed=1, epochs=30, batch=256, lr=3e-3)
    assert (mlp.predict(params, X) == y).mean() > 0.98


def test_prediction_ties_take_the_lowest_index():
    params = mlp.init_params(3, 4, 5, 0)
    for k in ("W3", "b3"):
        params[k] = np.zeros_like(params[k])
    assert np.all(mlp.predict(params, np.ones((4, 3))) == 0)


# --- planted mistakes: each must break a pin above -------------------------
class _Planted:
    def __init__(self, **over):
        self.__dict__.update({k: getattr(mlp, k) for k in ("gelu", "gelu_grad", "softmax_xent", "forward")})
        self.__dict__.update(over)

    def loss_and_grad(self, params, X, y):
        logits, c = self.forward(params, X)
        loss, d3 = self.softmax_xent(logits, y)
        g = {"W3": d3.T @ c["a2"], "b3": d3.sum(axis=0)}
        d2 = (d3 @ params["W3"]) * self.gelu_grad(c["z2"])
        g["W2"] = d2.T @ c["a1"]
        g["b2"] = d2.sum(axis=0)
        d1 = (d2 @ params["W2"]) * self.gelu_grad(c["z1"])
        g["W1"] = d1.T @ c["X"]
        g["b1"] = d1.sum(axis=0)
        if getattr(self, "transpose_w2", False):
            g["W2"] = g["W2"].T
        return loss, g


@pytest.mark.parametrize("plant", ["grad_drops_z_phi", "grad_sign", "transpose_w2", "tanh_gelu"])
def test_planted_mistakes_are_caught(plant):
    params, X, y = _tiny(seed=11, d=5, h=5, g=4)
    if plant == "grad_drops_z_phi":
        mod = _Planted(gelu_grad=lambda z: 0.5 * (1.0 + __import__("scipy").special.erf(z / np.sqrt(2.0))))
        assert _fd_check(mod, params, X, y) > 1e-3
    elif plant == "grad_sign":
        def bad_xent(logits, yy):
            loss, d = mlp.softmax_xent(logits, yy)
            return loss, -d
        assert _fd_check(_Planted(softmax_xent=bad_xent), params, X, y) > 1e-3
    elif plant == "transpose_w2":
        assert _fd_check(_Planted(transpose_w2=True), params, X, y) > 1e-3
    else:
        z = np.linspace(-6, 6, 241)
        tanh_gelu = 0.5 * z * (1 + np.tanh(np.sqrt(2 / np.pi) * (z + 0.044715 * z ** 3)))
        assert not np.allclose(tanh_gelu, z * norm.cdf(z), rtol=1e-13, atol=1e-15)
