"""Oracle of the random interpolation method.  TEST INFRASTRUCTURE ONLY.

The method (Sec. 3.1, Algorithms 1 and 2): per patch, the upscaled stiffness
S^m and load b^m are smooth functions of the patch's local parameters xi_m;
they are computed at the points of a tensor collocation grid (the 1-d node
sets may differ per direction) and every entry is replaced by its Lagrange
interpolant, which the online stage evaluates at the sample's xi_m.  A
sample whose xi_m leaves the collocation box is upscaled directly (Remark at
the end of Sec. 3.1.1).

Readings of the paper used here (the paper leaves these choices open):

* Nodes: Chebyshev points of the first kind, or the zeros of the Legendre
  polynomial (the paper's choice for uniform parameters), nu + 1 per
  direction on [-1, 1].
* Local parameters and their degrees: bump i acts on cell m with strength
  g = max over the cell of |d log a / d xi_i|, i.e. scale * exp(-d^2 / w^2)
  for a = exp(scale z) and (L gain / 4) exp(-d^2 / w^2) for the sigmoid
  transform, d the distance from the bump centre to the closed cell.  The
  degree nu is the smallest with 2 (g/2)^(nu+1) / (nu+1)! <= eps -- the
  bound on the Chebyshev coefficient of exp(g t) of that degree -- capped
  at nu_max; a bump with nu = 0 is frozen at xi_i = 0 (the node of the
  one-point rule).  The directions with nu >= 1 are the cell's local
  parameters xi_m.
* Families: cells whose local parameters sit at the same offsets from the
  cell's south-west corner with the same degrees have the same S^m(xi_m)
  (no oversampling: the coefficient on the cell is a translate), so one
  interpolant serves them all; it is built on the family's first cell.
* Order of the directions: by degree, then by offset (y, then x); the
  tensor grid's points are enumerated with the last direction fastest.
* Entries interpolated: the 10 packed entries of K_e and the 4 of b_e.

Functions: ``nodes``, ``lagrange`` (product form of the Lagrange basis),
``influence``, ``choose_nu``, ``cell_dims``, ``families``, ``build`` (the
offline stage on the FP64 oracle upscaler), ``evaluate`` (online stage,
plain nested sum over the tensor grid), ``upscale`` (all cells of samples,
direct upscale where a parameter leaves [-1, 1]).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

CHEBYSHEV, LEGENDRE = 0, 1
MAX_DIM = 16


def nodes(kind, nu):
    """nu + 1 collocation nodes on [-1, 1], ascending."""
    j = np.arange(nu + 1)
    if kind == CHEBYSHEV:
        return -np.cos((2 * j + 1) * math.pi / (2 * nu + 2))
    if kind == LEGENDRE:
        return np.polynomial.legendre.leggauss(nu + 1)[0]
    raise ValueError("unknown node kind")


def lagrange(x, t):
    """l_j(t) = prod_{k != j} (t - x_k) / (x_j - x_k), j = 0..len(x)-1."""
    n = len(x)
    out = np.ones(n)
    for j in range(n):
        for k in range(n):
            if k != j:
                out[j] *= (t - x[k]) / (x[j] - x[k])
    return out


def influence(field, d2):
    w = float(field["width"])
    psi = math.exp(-d2 / (w * w))
    if int(field["kind"]) == 0:
        return abs(float(field.get("scale", 1.0))) * psi
    if int(field["kind"]) == 1:
        return abs(float(field.get("contrast_log", 0.0)) * float(field.get("gain", 1.0))) / 4.0 * psi
    raise ValueError("the degree rule covers the exponential and sigmoid fields")


def choose_nu(g, eps, nu_max):
    nu = 0
    while nu < nu_max and 2.0 * (g / 2.0) ** (nu + 1) / math.factorial(nu + 1) > eps:
        nu += 1
    return nu


def cell_dims(nf, nc, field, cell, eps, nu_max):
    """[(oy, ox, nu, var)] of the cell's interpolated directions, in table order."""
    H = 1.0 / nc
    nbx, nby = int(field["nbx"]), int(field["nby"])
    cx, cy = cell % nc, cell // nc
    x0, x1, y0, y1 = cx * H, (cx + 1) * H, cy * H, (cy + 1) * H
    dims = []
    for by in range(nby):
        for bx in range(nbx):
            px, py = (bx + 0.5) / nbx, (by + 0.5) / nby
            dx = max(x0 - px, 0.0, px - x1)
            dy = max(y0 - py, 0.0, py - y1)
            nu = choose_nu(influence(field, dx * dx + dy * dy), eps, nu_max)
            if nu >= 1:
                oy = round((py - y0) * nf * 1e6)
                ox = round((px - x0) * nf * 1e6)
                dims.append((nu, oy, ox, by * nbx + bx))
    dims.sort()
    if len(dims) > MAX_DIM:
        raise ValueError("cell %d has %d interpolated directions > %d" % (cell, len(dims), MAX_DIM))
    return [(oy, ox, nu, var) for (nu, oy, ox, var) in dims]


def families(nf, nc, field, eps, nu_max):
    """fam[cell], keys (per family: ((oy, ox, nu), ...)), rep[fam] (first
    cell), dims[cell]."""
    ncell = nc * nc
    fam = np.zeros(ncell, dtype=np.int32)
    keys, rep, dims = [], [], []
    index = {}
    for cell in range(ncell):
        d = cell_dims(nf, nc, field, cell, eps, nu_max)
        key = tuple((oy, ox, nu) for (oy, ox, nu, _) in d)
        if key not in index:
            index[key] = len(keys)
            keys.append(key)
            rep.append(cell)
        fam[cell] = index[key]
        dims.append(d)
    return fam, keys, rep, dims


def build(nf, nc, f, field, eps, nu_max, kind=CHEBYSHEV):
    """Offline stage (Algorithm 1): per family, S and b of the family's
    first cell at every point of its tensor grid.  V[fam] is [N][14]
    (10 packed K_e entries, then 4 b_e entries)."""
    import oracle
    fam, keys, rep, dims = families(nf, nc, field, eps, nu_max)
    K = int(field["nbx"]) * int(field["nby"])
    rho = nf // nc
    V = []
    for fm, cell in enumerate(rep):
        d = dims[cell]
        xs = [nodes(kind, nu) for (_, _, nu, _) in d]
        cx, cy = cell % nc, cell // nc
        ex0, ey0 = cx * rho, cy * rho
        rows = []
        for idx in itertools.product(*[range(len(x)) for x in xs]):
            xi = np.zeros(K)
            for k, (_, _, _, var) in enumerate(d):
                xi[var] = xs[k][idx[k]]
            a = oracle.sample_coef_window(nf, field, xi, ex0, ex0 + rho, ey0, ey0 + rho)
            Ke, be, _, _ = oracle.cell(nf, nc, f, a, cx, cy, 0)
            rows.append(np.concatenate([Ke, be]))
        V.append(np.array(rows).reshape(-1, 14))
    return dict(nf=nf, nc=nc, f=f, field=dict(field), eps=eps, nu_max=nu_max, kind=kind,
                fam=fam, keys=keys, rep=rep, dims=dims, V=V)


def in_box(model, xi_row, cell):
    return all(abs(xi_row[var]) <= 1.0 for (_, _, _, var) in model["dims"][cell])


def evaluate(model, xi_row, cell):
    """Online stage (Algorithm 2) for one cell: the tensor Lagrange
    interpolant sum_p prod_k l_{i_k}(xi_k) V[p] -> (K_e[10], b_e[4])."""
    d = model["dims"][cell]
    V = model["V"][model["fam"][cell]]
    ls = [lagrange(nodes(model["kind"], nu), xi_row[var]) for (_, _, nu, var) in d]
    out = np.zeros(14)
    for p, idx in enumerate(itertools.product(*[range(len(l)) for l in ls])):
        w = 1.0
        for k, i in enumerate(idx):
            w *= ls[k][i]
        out += w * V[p]
    return out[:10], out[10:]


def upscale(model, xi, a=None):
    """K_e [S][ncell][10], b_e [S][ncell][4], fell_back [S][ncell]: the
    interpolant where every local parameter is in [-1, 1], else the direct
    FP64 upscale of the sample's coefficient ``a`` (required then)."""
    import oracle
    nf, nc, f = model["nf"], model["nc"], model["f"]
    S = xi.shape[0]
    ncell = nc * nc
    Ke = np.empty((S, ncell, 10))
    be = np.empty((S, ncell, 4))
    fb = np.zeros((S, ncell), dtype=np.uint8)
    for s in range(S):
        for cell in range(ncell):
            if in_box(model, xi[s], cell):
                Ke[s, cell], be[s, cell] = evaluate(model, xi[s], cell)
            else:
                if a is None:
                    raise ValueError("a sample leaves the collocation box and no coefficient was given")
                k, b, _, _ = oracle.cell(nf, nc, f, a[s], cell % nc, cell // nc, 0)
                Ke[s, cell], be[s, cell] = k, b
                fb[s, cell] = 1
    return Ke, be, fb
