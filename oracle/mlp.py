"""FP64 reference of the warm-start encoder network (numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). The paper has no
network; this is the plain definition of the encoder the library trains:

  x  = log(1 + y)                      (counts of one cell, n_in genes)
  z1 = W1 x + b1,  h1 = gelu(z1)       gelu(t) = t Phi(t), Phi the N(0,1) cdf
  z2 = W2 h1 + b2, h2 = gelu(z2)
  o  = W3 h2 + b3
  loss = mean over the batch and the n_out outputs of (o - target)^2

and its gradients by the chain rule, gelu'(t) = Phi(t) + t phi(t); the Adam
update of Kingma and Ba (bias-corrected first and second moments).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def gelu(t):
    return 0.5 * t * (1.0 + erf(t / np.sqrt(2.0)))


def gelu_prime(t):
    return 0.5 * (1.0 + erf(t / np.sqrt(2.0))) + t * np.exp(-0.5 * t * t) / np.sqrt(2.0 * np.pi)


def init_params(n_in, n_h1, n_h2, n_out, seed):
    """The seeded starting weights (drawn by the shared input module)."""
    import synth
    return synth.mlp_init(n_in, n_h1, n_h2, n_out, seed)


def forward(P, Y):
    return forward_x(P, np.log1p(np.asarray(Y, dtype=np.float64)))


def forward_x(P, X):
    """The forward pass from the inputs x = log(1 + y) themselves."""
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ P["W1"].T + P["b1"]
    H1 = gelu(Z1)
    Z2 = H1 @ P["W2"].T + P["b2"]
    H2 = gelu(Z2)
    O = H2 @ P["W3"].T + P["b3"]
    return O, (X, Z1, H1, Z2, H2)


def loss(P, Y, T):
    O, _ = forward(P, Y)
    return float(np.mean((O - T) ** 2))


def loss_grad(P, Y, T):
    O, (X, Z1, H1, Z2, H2) = forward(P, Y)
    B, n_out = O.shape
    dO = 2.0 * (O - T) / (B * n_out)
    g = {}
    g["W3"] = dO.T @ H2
    g["b3"] = dO.sum(0)
    dZ2 = (dO @ P["W3"]) * gelu_prime(Z2)
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(0)
    dZ1 = (dZ2 @ P["W2"]) * gelu_prime(Z1)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(0)
    return float(np.mean((O - T) ** 2)), g


def adam_step(P, g, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state holds m, v (dicts) and the step count k."""
    state["k"] = state.get("k", 0) + 1
    k = state["k"]
    for n in NAMES:
        m = state.setdefault("m", {}).setdefault(n, np.zeros_like(P[n]))
        v = state.setdefault("v", {}).setdefault(n, np.zeros_like(P[n]))
        m[:] = beta1 * m + (1 - beta1) * g[n]
        v[:] = beta2 * v + (1 - beta2) * g[n] ** 2
        mh = m / (1 - beta1 ** k)
        vh = v / (1 - beta2 ** k)
        P[n] = P[n] - lr * mh / (np.sqrt(vh) + eps)
