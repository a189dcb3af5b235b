"""FP64 reference of the learned opening-angle network.

TEST INFRASTRUCTURE (see the package docstring).  The network and its loss
are this project's reading of the learned-theta form: the paper has a single
global theta (Eq. mac) and no learned component.

Network (per group, 12 input features):
    z0 = (x - mu) / sigma                          (padded with 4 zeros to 16)
    h1 = gelu(W1 z0 + b1),  W1: 64 x 16
    h2 = gelu(W2 h1 + b2),  W2: 64 x 64
    h3 = gelu(W3 h2 + b3),  W3: 64 x 64
    z  = w4 . h3 + b4
    theta = 0.3 + 0.9 * sigmoid(z)
with gelu(x) = x * Phi(x) (Phi the standard normal CDF).  The GPU runs the
matrix products on tensor cores with BF16 operands (the layer inputs and the
weights rounded to BF16) and FP32 accumulation; `bf16=True` here rounds the
same operands the same way and accumulates in FP64.

Loss per sample, with label y (the largest theta meeting the error budget):
    L = (theta - y)^2 + lam * max(0, theta - y)^2      (lam = 4)
averaged over the batch: over-predicting theta (an error above budget) costs
five times more than under-predicting it.

Flat parameter layout (FP32 on the GPU), offsets in floats:
    W1 0 (64x16), b1 1024, W2 1088 (64x64), b2 5184, W3 5248, b3 9344,
    w4 9408 (8x64, row 0 used), b4 9920 (8, [0] used), mu 9928 (16),
    sigma 9944 (16); total 9960.
"""
from __future__ import annotations

import math

import numpy as np

H = 64
NIN = 12
KIN = 16
LAM = 4.0
OFF = dict(W1=0, b1=1024, W2=1088, b2=5184, W3=5248, b3=9344, w4=9408, b4=9920,
           mu=9928, sigma=9944)
NPARAM = 9960


def unpack(p):
    p = np.asarray(p, np.float64)
    return dict(
        W1=p[OFF["W1"]:OFF["W1"] + H * KIN].reshape(H, KIN),
        b1=p[OFF["b1"]:OFF["b1"] + H],
        W2=p[OFF["W2"]:OFF["W2"] + H * H].reshape(H, H),
        b2=p[OFF["b2"]:OFF["b2"] + H],
        W3=p[OFF["W3"]:OFF["W3"] + H * H].reshape(H, H),
        b3=p[OFF["b3"]:OFF["b3"] + H],
        w4=p[OFF["w4"]:OFF["w4"] + H],
        b4=p[OFF["b4"]],
        mu=p[OFF["mu"]:OFF["mu"] + KIN],
        sigma=p[OFF["sigma"]:OFF["sigma"] + KIN])


def pack_grads(g):
    out = np.zeros(NPARAM)
    out[OFF["W1"]:OFF["W1"] + H * KIN] = g["W1"].ravel()
    out[OFF["b1"]:OFF["b1"] + H] = g["b1"]
    out[OFF["W2"]:OFF["W2"] + H * H] = g["W2"].ravel()
    out[OFF["b2"]:OFF["b2"] + H] = g["b2"]
    out[OFF["W3"]:OFF["W3"] + H * H] = g["W3"].ravel()
    out[OFF["b3"]:OFF["b3"] + H] = g["b3"]
    out[OFF["w4"]:OFF["w4"] + H] = g["w4"]
    out[OFF["b4"]] = g["b4"]
    return out


def bf16(x):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    a = np.asarray(x, np.float32).copy()
    u = a.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    u = ((u + rounding) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(x):
    return x * 0.5 * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    Phi = 0.5 * (1.0 + _erf(x / math.sqrt(2.0)))
    phi = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return Phi + x * phi


def forward(p, x, bf=False):
    """Returns theta (B,) and the cache for backward.  x: (B, 12)."""
    P = unpack(p)
    q = (lambda a: bf16(a)) if bf else (lambda a: np.asarray(a, np.float64))
    x = np.asarray(x, np.float64)
    z0 = np.zeros((x.shape[0], KIN))
    z0[:, :NIN] = (x - P["mu"][:NIN]) / P["sigma"][:NIN]
    if bf:  # the GPU forms z0 in FP32
        z0 = np.asarray(z0, np.float32).astype(np.float64)
    a0 = q(z0)
    Z1 = a0 @ q(P["W1"]).T + P["b1"]
    h1 = gelu(Z1)
    a1 = q(h1)
    Z2 = a1 @ q(P["W2"]).T + P["b2"]
    h2 = gelu(Z2)
    a2 = q(h2)
    Z3 = a2 @ q(P["W3"]).T + P["b3"]
    h3 = gelu(Z3)
    z = h3 @ P["w4"] + P["b4"]
    s = 1.0 / (1.0 + np.exp(-z))
    theta = 0.3 + 0.9 * s
    return theta, dict(a0=a0, Z1=Z1, a1=a1, Z2=Z2, a2=a2, Z3=Z3, h3=h3, z=z, s=s, P=P, q=q)


def loss(theta, y):
    d = theta - np.asarray(y, np.float64)
    return float(np.mean(d * d + LAM * np.maximum(d, 0.0) ** 2))


def backward(p, x, y, bf=False):
    """Mean loss and its gradient (flat, NPARAM) by backpropagation."""
    theta, c = forward(p, x, bf)
    P, q = c["P"], c["q"]
    B = theta.shape[0]
    d = theta - np.asarray(y, np.float64)
    dtheta = (2.0 * d + 2.0 * LAM * np.maximum(d, 0.0)) / B
    dz = dtheta * 0.9 * c["s"] * (1.0 - c["s"])
    g = {}
    g["w4"] = dz @ c["h3"]
    g["b4"] = dz.sum()
    dh3 = np.outer(dz, P["w4"])
    dZ3 = dh3 * gelu_grad(c["Z3"])
    g["W3"] = q(dZ3).T @ c["a2"]
    g["b3"] = dZ3.sum(0)
    dh2 = q(dZ3) @ q(P["W3"])
    dZ2 = dh2 * gelu_grad(c["Z2"])
    g["W2"] = q(dZ2).T @ c["a1"]
    g["b2"] = dZ2.sum(0)
    dh1 = q(dZ2) @ q(P["W2"])
    dZ1 = dh1 * gelu_grad(c["Z1"])
    g["W1"] = q(dZ1).T @ c["a0"]
    g["b1"] = dZ1.sum(0)
    return loss(theta, y), pack_grads(g)


def adam(p, m, v, grad, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (p, m, v).  Entries whose
    gradient is always zero (padding, mu, sigma) never move."""
    p = np.asarray(p, np.float64)
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def pack_params(W1, b1, W2, b2, W3, b3, w4, b4, mu, sigma):
    """Flat FP32 parameter vector from its parts (W1 is 64 x 12)."""
    p = np.zeros(NPARAM)
    w1 = np.zeros((H, KIN))
    w1[:, :NIN] = W1
    p[OFF["W1"]:OFF["W1"] + H * KIN] = w1.ravel()
    p[OFF["b1"]:OFF["b1"] + H] = b1
    p[OFF["W2"]:OFF["W2"] + H * H] = np.ravel(W2)
    p[OFF["b2"]:OFF["b2"] + H] = b2
    p[OFF["W3"]:OFF["W3"] + H * H] = np.ravel(W3)
    p[OFF["b3"]:OFF["b3"] + H] = b3
    p[OFF["w4"]:OFF["w4"] + H] = w4
    p[OFF["b4"]] = b4
    p[OFF["mu"]:OFF["mu"] + NIN] = mu
    sg = np.ones(KIN)
    sg[:NIN] = sigma
    p[OFF["sigma"]:OFF["sigma"] + KIN] = sg
    return p.astype(np.float32)
