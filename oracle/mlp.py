"""FP64 MLP oracle for the learned surrogate.  TEST INFRASTRUCTURE ONLY.

The surrogate stands in for the random-interpolation model of the local
upscaled quantities S^m(xi_m), b^m(xi_m) (Sec. 3.1, Algs. 1-2): per patch
family a multilayer perceptron maps the cell's local random variables
xi_m (Eq. MsFEB2: the K_m parameters that the cell problem actually sees)
to the 10 packed entries of K_e / abar_cell and 3 load entries.

Network:  x -> GELU(x W1 + b1) -> GELU(. W2 + b2) -> GELU(. W3 + b3) -> . W4 + b4
GELU is the exact form 0.5 t (1 + erf(t / sqrt 2)).  Loss is the mean of the
squared error over batch rows and output columns.  Adam with bias
correction.  Plain numpy in float64; the backward pass is the chain rule
written out layer by layer.
"""
from __future__ import annotations

import math

import numpy as np

_erf = np.vectorize(math.erf)
_SQ2 = math.sqrt(2.0)
_ISQ2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(t):
    return 0.5 * t * (1.0 + _erf(t / _SQ2))


def gelu_grad(t):
    # d/dt [t Phi(t)] = Phi(t) + t phi(t)
    return 0.5 * (1.0 + _erf(t / _SQ2)) + t * _ISQ2PI * np.exp(-0.5 * t * t)


def forward(params, x):
    """params: list of (W, b) for the 4 layers.  Returns (y, cache)."""
    acts = [x]
    pre = []
    h = x
    for li, (W, b) in enumerate(params):
        z = h @ W + b
        pre.append(z)
        h = gelu(z) if li < len(params) - 1 else z
        acts.append(h)
    return h, (acts, pre)


def loss(y, t):
    d = y - t
    return float(np.mean(d * d))


def backward(params, cache, y, t):
    """Gradients of loss(y, t) = mean((y - t)^2) w.r.t. every (W, b)."""
    acts, pre = cache
    g = 2.0 * (y - t) / y.size
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        if li < len(params) - 1:
            g = g * gelu_grad(pre[li])
        gW = acts[li].T @ g
        gb = g.sum(axis=0)
        grads[li] = (gW, gb)
        g = g @ W.T
    return grads


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One bias-corrected Adam update in place; state = dict(t, m, v)."""
    state["t"] += 1
    t = state["t"]
    for li in range(len(params)):
        for j in range(2):
            g = grads[li][j]
            m = state["m"][li][j]
            v = state["v"][li][j]
            m *= beta1
            m += (1.0 - beta1) * g
            v *= beta2
            v += (1.0 - beta2) * g * g
            mhat = m / (1.0 - beta1 ** t)
            vhat = v / (1.0 - beta2 ** t)
            params[li][j][...] -= lr * mhat / (np.sqrt(vhat) + eps)


def adam_init(params):
    return {"t": 0,
            "m": [[np.zeros_like(W), np.zeros_like(b)] for W, b in params],
            "v": [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]}


def zero_row_sum_projector():
    """The 10x10 linear map onto packed symmetric 4x4 matrices with zero
    row sums, orthogonal in the packed coordinates: a zero-row-sum matrix
    is fixed by its 6 off-diagonal entries o (diagonal = -row sum), K = B o;
    the map is B (B^T B)^{-1} B^T."""
    pairs = [(l, lp) for l in range(4) for lp in range(l, 4)]
    off = [(l, lp) for (l, lp) in pairs if l != lp]
    B = np.zeros((10, 6))
    for q, (l, lp) in enumerate(pairs):
        for j, (i1, i2) in enumerate(off):
            if l != lp:
                B[q, j] = 1.0 if (l, lp) == (i1, i2) else 0.0
            else:
                B[q, j] = -1.0 if l in (i1, i2) else 0.0
    return B @ np.linalg.solve(B.T @ B, B.T)
