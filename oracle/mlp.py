"""O3: the learned group proposal's MLP in FP64 -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module; the product library never does.

The paper names no learned component; the proposal is the library's layered
form on top of the filtered method (its labels are the filtered method's,
exactly).  What it computes, written from the definitions:

* a multilayer perceptron D -> H -> H -> G with GELU activations,
  GELU(z) = z * Phi(z) = z/2 * (1 + erf(z / sqrt(2)))  (the exact form, not
  the tanh approximation);
* softmax cross-entropy over the G groups, averaged over the batch;
* gradients by the chain rule, layer by layer;
* Adam (Kingma & Ba, ICLR 2015): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
  step = lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps);
* Xavier-uniform initialisation: U(-a, a), a = sqrt(6 / (fan_in + fan_out)),
  biases zero;
* the prediction: the group with the largest logit (lowest index on ties).

Weights are row-major with the output index first: W1 is H x D, W2 H x H,
W3 G x H (a layer computes z = W a + b).
Pins: ``tests/test_oracle_mlp.py`` (finite-difference gradients, GELU values
of the normal distribution function, the uniform-logit loss log G, Adam's
first step, learning a separable toy problem, planted mistakes).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    # d/dz [z Phi(z)] = Phi(z) + z phi(z)
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def init_params(d_in: int, hidden: int, classes: int, seed: int) -> dict:
    rng = np.random.default_rng(seed)

    def xavier(fan_out, fan_in):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-a, a, size=(fan_out, fan_in))

    return {"W1": xavier(hidden, d_in), "b1": np.zeros(hidden),
            "W2": xavier(hidden, hidden), "b2": np.zeros(hidden),
            "W3": xavier(classes, hidden), "b3": np.zeros(classes)}


def forward(params: dict, X) -> tuple[np.ndarray, dict]:
    """Logits (n x G) and the intermediate values the gradient needs."""
    X = np.asarray(X, np.float64)
    z1 = X @ params["W1"].T + params["b1"]
    a1 = gelu(z1)
    z2 = a1 @ params["W2"].T + params["b2"]
    a2 = gelu(z2)
    z3 = a2 @ params["W3"].T + params["b3"]
    return z3, {"X": X, "z1": z1, "a1": a1, "z2": z2, "a2": a2}


def softmax_xent(logits, y) -> tuple[float, np.ndarray]:
    """Mean cross-entropy of the softmax and its gradient w.r.t. the logits."""
    y = np.asarray(y, np.int64)
    m = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - m)
    s = e.sum(axis=1, keepdims=True)
    logp = logits - m - np.log(s)
    n = logits.shape[0]
    loss = -logp[np.arange(n), y].mean()
    d = e / s
    d[np.arange(n), y] -= 1.0
    return float(loss), d / n


def loss_and_grad(params: dict, X, y) -> tuple[float, dict]:
    logits, c = forward(params, X)
    loss, d3 = softmax_xent(logits, y)
    g = {"W3": d3.T @ c["a2"], "b3": d3.sum(axis=0)}
    d2 = (d3 @ params["W3"]) * gelu_grad(c["z2"])
    g["W2"] = d2.T @ c["a1"]
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ params["W2"]) * gelu_grad(c["z1"])
    g["W1"] = d1.T @ c["X"]
    g["b1"] = d1.sum(axis=0)
    return loss, g


def adam_init(params: dict) -> dict:
    return {"t": 0, "m": {k: np.zeros_like(v) for k, v in params.items()},
            "v": {k: np.zeros_like(v) for k, v in params.items()}}


def adam_step(params: dict, grads: dict, state: dict, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8) -> None:
    state["t"] += 1
    t = state["t"]
    for k in params:
        state["m"][k] = b1 * state["m"][k] + (1.0 - b1) * grads[k]
        state["v"][k] = b2 * state["v"][k] + (1.0 - b2) * grads[k] * grads[k]
        mh = state["m"][k] / (1.0 - b1 ** t)
        vh = state["v"][k] / (1.0 - b2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)


def predict(params: dict, X) -> np.ndarray:
    logits, _ = forward(params, X)
    return np.argmax(logits, axis=1).astype(np.int32)  # first maximum: lowest index on ties


def train(X, y, hidden: int, classes: int, *, seed: int = 0, epochs: int = 5, batch: int = 8192,
          lr: float = 1e-3, shuffle_seed: int = 1) -> dict:
    """Adam on minibatches; returns the FP64 parameters."""
    X = np.asarray(X, np.float64)
    params = init_params(X.shape[1], hidden, classes, seed)
    state = adam_init(params)
    rng = np.random.default_rng(shuffle_seed)
    n = X.shape[0]
    for _ in range(epochs):
        order = rng.permutation(n)
        for s in range(0, n, batch):
            idx = order[s:s + batch]
            _, g = loss_and_grad(params, X[idx], y[idx])
            adam_step(params, g, state, lr=lr)
    return params
