"""Oracle pieces of the learned surrogate.  TEST INFRASTRUCTURE ONLY.

* ``local_vars``  -- the cell's local parameters xi_m (Eq. MsFEB2): bump i is
  local to cell m when its Gaussian exceeds tau somewhere on the closed cell
  rectangle; sorted by the bump centre's offset from the cell's SW corner
  (y, then x); cells with the same offsets share a family (and a network).
* ``targets``     -- network inputs and scaled targets of a (sample, cell):
  x = xi_m zero padded to 16; y_0..9 = K_e / abar - K_ref, y_10..12 =
  b_l / (f H^2) - 1/4, abar the cell mean of a.
* ``predict``     -- the inverse map with the zero-row-sum projection.
* weight layout conversions between the flat [out][in] layout and the
  (W [in][out], b) pairs of ``oracle.mlp``.
"""
from __future__ import annotations

import math

import numpy as np

from . import mlp

K_IN, HID, K_OUT, OUT_USED = 16, 128, 16, 13
KREF_PACKED = np.array([4, -1, -2, -1, 4, -1, -2, 4, -1, 4], dtype=np.float64) / 6.0
SHAPES = [(HID, K_IN), (HID,), (HID, HID), (HID,), (HID, HID), (HID,), (K_OUT, HID), (K_OUT,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)


def local_vars(nf, nc, field, tau):
    H = 1.0 / nc
    nbx, nby, w = int(field["nbx"]), int(field["nby"]), float(field["width"])
    ncell = nc * nc
    k = np.zeros(ncell, dtype=np.int32)
    ids = -np.ones((ncell, K_IN), dtype=np.int32)
    fam = np.zeros(ncell, dtype=np.int32)
    keys = {}
    for cell in range(ncell):
        cx, cy = cell % nc, cell // nc
        x0, x1, y0, y1 = cx * H, (cx + 1) * H, cy * H, (cy + 1) * H
        loc = []
        for by in range(nby):
            for bx in range(nbx):
                px, py = (bx + 0.5) / nbx, (by + 0.5) / nby
                dx = max(x0 - px, 0.0, px - x1)
                dy = max(y0 - py, 0.0, py - y1)
                if math.exp(-(dx * dx + dy * dy) / (w * w)) >= tau:
                    loc.append(((round((py - y0) * nf * 1e6), round((px - x0) * nf * 1e6)), by * nbx + bx))
        loc.sort()
        if len(loc) > K_IN:
            raise ValueError("too many local variables")
        key = tuple(o for o, _ in loc)
        if key not in keys:
            keys[key] = len(keys)
        fam[cell] = keys[key]
        k[cell] = len(loc)
        for j, (_, i) in enumerate(loc):
            ids[cell, j] = i
    return k, ids, fam, len(keys)


def targets(xi_s, a_s, Ke_u, be_u, ids_cell, nf, nc, cell, f):
    """One unit: (x[16], y[16])."""
    rho = nf // nc
    cx, cy = cell % nc, cell // nc
    x = np.zeros(K_IN)
    for j, i in enumerate(ids_cell):
        if i >= 0:
            x[j] = xi_s[i]
    abar = a_s[cy * rho:(cy + 1) * rho, cx * rho:(cx + 1) * rho].mean()
    H = 1.0 / nc
    y = np.zeros(K_OUT)
    y[:10] = Ke_u / abar - KREF_PACKED
    y[10:13] = be_u[:3] / (f * H * H) - 0.25
    return x, y


def predict(y, abar, f, H):
    """K_e (10) and b_e (4) from a network output y (16)."""
    P = mlp.zero_row_sum_projector()
    K = abar * (KREF_PACKED + P @ y[:10])
    b = np.empty(4)
    b[:3] = f * H * H * (0.25 + y[10:13])
    b[3] = f * H * H - b[:3].sum()
    return K, b


def unflatten(wflat):
    """flat [out][in] layout -> list of (W [in][out], b) for oracle.mlp."""
    out, o = [], 0
    for li in range(4):
        ws, bs = SHAPES[2 * li], SHAPES[2 * li + 1]
        W = np.asarray(wflat[o:o + ws[0] * ws[1]], dtype=np.float64).reshape(ws).T.copy()
        o += ws[0] * ws[1]
        b = np.asarray(wflat[o:o + bs[0]], dtype=np.float64).copy()
        o += bs[0]
        out.append((W, b))
    return out


def flatten(params):
    parts = []
    for W, b in params:
        parts.append(W.T.reshape(-1))
        parts.append(b.reshape(-1))
    return np.concatenate(parts)


def forward(wflat, X):
    """FP64 forward of the flat-layout network on rows X [B][16]."""
    y, _ = mlp.forward(unflatten(wflat), np.asarray(X, dtype=np.float64))
    return y


def loss_and_grad(wflat, X, T):
    """Loss mean over rows and the 13 used outputs; gradient in the flat layout."""
    P = unflatten(wflat)
    X = np.asarray(X, dtype=np.float64)
    y, cache = mlp.forward(P, X)
    Tm = np.array(T, dtype=np.float64, copy=True)
    Tm[:, OUT_USED:] = y[:, OUT_USED:]       # unused outputs carry no loss
    d = (y - Tm)[:, :OUT_USED]
    loss = float(np.mean(d * d))
    # mlp.backward differentiates mean over all outputs; rescale to the 13 used
    grads = mlp.backward(P, cache, y, Tm)
    scale = K_OUT / OUT_USED
    grads = [(gW * scale, gb * scale) for gW, gb in grads]
    return loss, flatten(grads)
