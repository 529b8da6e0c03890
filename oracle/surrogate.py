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
* ``indicator``   -- the error indicator that sends a prediction back to the
  plain upscaler: an input outside the family's training box (widened by a
  margin, the out-of-range recompute of the remark closing Sec. 3.1.1), an
  energy of the x- or y-linear corner vector outside the cell's harmonic /
  arithmetic mean bounds, or a matrix that is not positive definite once
  the constants are factored out (the a-posteriori checks of Sec. 3.2);
  ``ensemble_disagrees`` the optional test of two networks' disagreement.
* ``minibatch_rows`` -- the training rows of one Adam step: SplitMix64
  (Steele, Lea and Flood, OOPSLA 2014, in Vigna's 64-bit form) of the seed,
  the family, the step and the row slot, reduced modulo the family's rows;
  every 10th row is held out (a drawn held-out row moves to its predecessor).
* ``train``       -- the Adam loop with bias correction and the cosine
  learning-rate decay from lr to lr_min over the steps of one call.
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


# ---------------------------------------------------------------- indicator

def _sym4(Kp):
    """Packed upper triangle (10) -> symmetric 4x4, corners SW, SE, NE, NW."""
    K = np.zeros((4, 4))
    q = 0
    for r in range(4):
        for c in range(r, 4):
            K[r, c] = K[c, r] = Kp[q]
            q += 1
    return K


# corner values of the two affine test functions on the cell (SW, SE, NE, NW)
V_XLIN = np.array([0.0, 1.0, 1.0, 0.0])
V_YLIN = np.array([0.0, 0.0, 1.0, 1.0])


def indicator(x, box, margin, Kp, abar, ahar, delta):
    """Reasons (a dict of booleans) why a surrogate prediction is rejected.

    x [16] network inputs; box [16][2] the family's training range per
    input; margin the widening as a fraction of each range; Kp the packed
    prediction; abar, ahar the arithmetic and harmonic means of a over the
    cell; delta the relative slack of the energy bounds.

    * range: some x_j lies below lo_j - margin (hi_j - lo_j) or above
      hi_j + margin (hi_j - lo_j).
    * energy: for v the x-linear and the y-linear corner vectors, v^T K v
      must lie in [ahar (1 - delta), abar (1 + delta)].  The cell problem
      with affine boundary data has the arithmetic mean as an upper bound
      (the affine function itself is admissible: Dirichlet principle) and
      the harmonic mean as a lower bound (Voigt-Reuss).
    * pd: K must be positive definite on vectors orthogonal to the
      constants (the kernel of an exact K_e is the constants): the
      smallest eigenvalue of Q^T K Q, Q an orthonormal basis of that
      complement, must be positive.
    """
    x = np.asarray(x, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    lo, hi = box[:, 0], box[:, 1]
    m = margin * (hi - lo)
    out_of_range = bool(np.any((x < lo - m) | (x > hi + m)))
    K = _sym4(np.asarray(Kp, dtype=np.float64))
    energy = False
    for v in (V_XLIN, V_YLIN):
        e = float(v @ K @ v)
        if not (ahar * (1.0 - delta) <= e <= abar * (1.0 + delta)):
            energy = True
    # orthonormal basis of the complement of the constants
    Q, _ = np.linalg.qr(np.array([[1.0, -1.0, 0.0, 0.0], [1.0, 0.0, -1.0, 0.0], [1.0, 0.0, 0.0, -1.0]]).T)
    lam = np.linalg.eigvalsh(Q.T @ K @ Q)
    not_pd = not bool(lam[0] > 0.0)
    return {"range": out_of_range, "energy": energy, "pd": not_pd}


def pack_upper_sym(M):
    """Symmetric 4x4 -> packed upper triangle (10)."""
    return np.array([M[r, c] for r in range(4) for c in range(r, 4)], dtype=np.float64)


def energy_values(Kp):
    """(v_x^T K v_x, v_y^T K v_y) of a packed matrix."""
    K = _sym4(np.asarray(Kp, dtype=np.float64))
    return float(V_XLIN @ K @ V_XLIN), float(V_YLIN @ K @ V_YLIN)


def flagged(x, box, margin, Kp, abar, ahar, delta):
    return any(indicator(x, box, margin, Kp, abar, ahar, delta).values())


def ensemble_disagrees(Kp1, Kp2, tol):
    """The ensemble test of two independently trained networks on the same
    unit: their packed predictions differ by more than tol relative to the
    first, ||Kp1 - Kp2|| > tol ||Kp1|| (Euclidean norm over the 10 packed
    entries)."""
    Kp1 = np.asarray(Kp1, dtype=np.float64)
    Kp2 = np.asarray(Kp2, dtype=np.float64)
    return bool(np.linalg.norm(Kp1 - Kp2) > tol * np.linalg.norm(Kp1))


# ---------------------------------------------------------------- training loop

_M64 = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 output for state increment applied once to x (Vigna's
    64-bit finaliser of the golden-gamma sequence)."""
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


BATCH = 64


def minibatch_rows(seed, fam, gstep, nrows):
    """Row indices (within the family) of training step gstep."""
    rows = []
    for slot in range(BATCH):
        key = (seed ^ (fam << 40) ^ (gstep << 16) ^ slot) & _M64
        r = splitmix64(key) % nrows
        if r % 10 == 9 and nrows > 1:
            r -= 1
        rows.append(r)
    return rows


def train(wflat, X, T, steps, step0=0, lr=1e-3, lr_min=1e-5, beta1=0.9, beta2=0.999, eps=1e-8,
          seed=0, fam=0, m=None, v=None):
    """FP64 Adam on one family's rows X [N][16], T [N][16] for `steps`
    minibatches starting at global step step0.  The learning rate of step
    gstep is lr_min + (lr - lr_min) (1 + cos(pi gstep / (step0 + steps))) / 2.
    Returns (weights, m, v, losses)."""
    w = np.asarray(wflat, dtype=np.float64).copy()
    m = np.zeros_like(w) if m is None else np.asarray(m, dtype=np.float64).copy()
    v = np.zeros_like(w) if v is None else np.asarray(v, dtype=np.float64).copy()
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    horizon = max(1.0, float(step0 + steps))
    losses = []
    for k in range(steps):
        gstep = step0 + k
        rows = minibatch_rows(seed, fam, gstep, X.shape[0])
        loss, g = loss_and_grad(w, X[rows], T[rows])
        losses.append(loss)
        rate = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * gstep / horizon))
        m = beta1 * m + (1.0 - beta1) * g
        v = beta2 * v + (1.0 - beta2) * g * g
        mhat = m / (1.0 - beta1 ** (gstep + 1))
        vhat = v / (1.0 - beta2 ** (gstep + 1))
        w = w - rate * mhat / (np.sqrt(vhat) + eps)
    return w, m, v, np.array(losses)
