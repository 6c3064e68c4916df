"""FP64 CPU reference of the learned warm-start network (test infrastructure only).

A multilayer perceptron y = W_L' ... GELU(W_1' x + b_1) ... + b_L with the exact GELU
x/2 (1 + erf(x / sqrt 2)), trained on the mean squared error with AdamW.  With
``bf16=True`` the reference rounds to bfloat16 (round to nearest even) at the same points
as the GPU kernels — inputs, weights, pre-activations, activations and back-propagated
gradients — and computes everything else in double precision.  Only tests may import it.
"""
from __future__ import annotations

import math

import numpy as np

_erf = np.vectorize(math.erf)


def bf16(a):
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    x = np.asarray(a, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(Ws, bs, x, bf=True):
    """Returns (pred, cache) with cache = (inputs to every layer, pre-activations of hidden layers)."""
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    h = r(x)
    ins, pres = [], []
    for l, (W, b) in enumerate(zip(Ws, bs)):
        ins.append(h)
        z = h @ r(W) + np.asarray(b, dtype=np.float64)
        if l + 1 < len(Ws):
            pre = r(z)
            pres.append(pre)
            h = r(gelu(pre))
        else:
            return z, (ins, pres)


def loss_and_grads(Ws, bs, x, target, bf=True):
    """Mean squared error and its gradients with respect to every W and b."""
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    pred, (ins, pres) = forward(Ws, bs, x, bf)
    t = r(target)
    e = pred - t
    loss = float(np.mean(e * e))
    g = r(2.0 * e / e.size)
    dWs, dbs = [None] * len(Ws), [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        dWs[l] = ins[l].T @ g
        dbs[l] = g.sum(axis=0)
        if l > 0:
            g = r((g @ r(Ws[l]).T) * gelu_grad(pres[l - 1]))
    return loss, dWs, dbs


def adamw(w, m, v, g, step, lr, wd, b1=0.9, b2=0.999, eps=1e-8):
    """One AdamW step (bias-corrected moments, decoupled weight decay); returns (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    c1, c2 = 1 - b1 ** step, 1 - b2 ** step
    w = w - lr * ((m / c1) / (np.sqrt(v / c2) + eps) + wd * w)
    return w, m, v
