"""Local KL expansion oracle (Sec. 2.1.1, Def. of the local KL expansion,
Eqs. localCov, localKL, local_KL_truncation), FP64 numpy.  TEST
INFRASTRUCTURE ONLY.

A random field kappa(x, omega) with mean kappa_bar and covariance Cov is
parametrized patch by patch: Cov restricted to the patch P_m, its
eigenpairs (lambda_k, f_k) with int_P f_k^2 = 1, the local parameters
xi_k = lambda_k^{-1/2} int_P (kappa - kappa_bar) f_k, and the truncated
expansion kappa_bar + sum_{k <= K_m} sqrt(lambda_k) xi_k f_k.

Discretisation: the piecewise-constant representation of the fine grid,
values at element centroids, midpoint quadrature with weight h^2 per
element, so the integral operator on P_m is the matrix h^2 C_m (C_m the
covariance between the patch's element centroids) and f_k are its
eigenvectors scaled to h^2 |f_k|^2 = 1.  Library routine used as a step:
numpy's eigh.

Covariances offered:
* ``cov_bumps``: the log-coefficient s * sum_i xi_i psi_i(x) of the bump
  fields of this repository (psi_i Gaussian bumps on the lattice, xi_i
  i.i.d. with variance 1/3 for U[-1, 1] or 1 for N(0, 1)), i.e.
  Cov(x, y) = s^2 var sum_i psi_i(x) psi_i(y), of rank at most the number
  of bumps;
* ``cov_gaussian``: the Gaussian covariance sigma^2 exp(-|x - y|^2 /
  beta^2) of the short-correlation example (Sec. 5.3).
"""
from __future__ import annotations

import numpy as np


def patch_centroids(nf, x0, x1, y0, y1):
    """Centroids [(y1-y0)*(x1-x0)][2] of the fine elements of the patch
    [x0, x1) x [y0, y1) (element indices), y-major."""
    h = 1.0 / nf
    ey, ex = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
    return np.stack([(ex.reshape(-1) + 0.5) * h, (ey.reshape(-1) + 0.5) * h], axis=1)


def bump_values(field, pts):
    """psi_i at the points: [len(pts)][nbx*nby], i = by*nbx + bx, centres at
    the lattice cell centres, psi_i(x) = exp(-|x - c_i|^2 / w^2)."""
    nbx, nby, w = int(field["nbx"]), int(field["nby"]), float(field["width"])
    cx = (np.arange(nbx) + 0.5) / nbx
    cy = (np.arange(nby) + 0.5) / nby
    Cx, Cy = np.meshgrid(cx, cy)                      # [nby][nbx]
    c = np.stack([Cx.reshape(-1), Cy.reshape(-1)], axis=1)
    d2 = ((pts[:, None, :] - c[None, :, :]) ** 2).sum(axis=2)
    return np.exp(-d2 / (w * w))


def cov_bumps(field, pts, dist="uniform"):
    """Covariance of s * z(x), z = sum_i xi_i psi_i, between the points."""
    var = 1.0 / 3.0 if dist == "uniform" else 1.0
    P = bump_values(field, pts)
    s = float(field.get("scale", 1.0))
    return (s * s * var) * (P @ P.T)


def cov_gaussian(pts, beta, sigma=1.0):
    d2 = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(axis=2)
    return sigma * sigma * np.exp(-d2 / (beta * beta))


def local_kl(C, h, energy=None, K=None):
    """Eigenpairs of the patch's integral operator h^2 C, descending, with
    f_k scaled to h^2 |f_k|^2 = 1.  Truncation: K modes, or the fewest
    modes whose eigenvalues reach the given share of the total (the
    paper's "99 % of the total spectrum"), or all modes with a positive
    eigenvalue.  Returns (lam [K], F [n][K], lam_all)."""
    w = h * h
    lam, U = np.linalg.eigh(w * C)
    order = np.argsort(lam)[::-1]
    lam, U = lam[order], U[:, order]
    if K is None:
        if energy is not None:
            cum = np.cumsum(np.maximum(lam, 0.0))
            K = int(np.searchsorted(cum, energy * cum[-1] * (1 - 1e-15)) + 1)
        else:
            K = int(np.sum(lam > 1e-12 * lam[0]))
    F = U[:, :K] / h                                  # h^2 |f|^2 = |U|^2 = 1
    return lam[:K], F, lam


def local_params(kappa, kappa_bar, lam, F, h):
    """xi_k = lambda_k^{-1/2} int_P (kappa - kappa_bar) f_k (Eq. localKL),
    kappa [..., n]."""
    return (h * h) * ((np.asarray(kappa) - kappa_bar) @ F) / np.sqrt(lam)


def reconstruct(xi, kappa_bar, lam, F):
    """kappa_bar + sum_k sqrt(lambda_k) xi_k f_k (Eq. local_KL_truncation)."""
    return kappa_bar + (np.asarray(xi) * np.sqrt(lam)) @ F.T
