"""Reduced-basis (POD) oracle, FP64 numpy.  TEST INFRASTRUCTURE ONLY.

Follows the reduced basis method of Sec. 3.2 for a cell without
oversampling (patch == cell):

* offline (Alg. 3): snapshots phi_l(x, omega_s) of the four multiscale
  basis functions over training samples; their mean phi_bar_l; the KL
  expansion of the centred snapshots in the energy inner product
  <u, v> = int a_bar grad u . grad v (Eq. KLphi and its footnote), with
  a_bar the training-mean coefficient; keep the leading modes while
  sqrt(lambda_q / lambda_1) >= tol (the truncation rule of Sec. 5.1).
  One basis V per cell serves all four l (the shared-basis reading used
  for the high-contrast example, Sec. 5.2); ``build_cell_per_l`` /
  ``online_cell_per_l`` give each of phi^1..phi^3 its own basis (the
  patch study, Sec. 5.1) with phi^4 from the partition of unity.
* online (Alg. 4): phi_rb,l = phi_bar_l + V c_l with the Galerkin system
  (V^T A(omega) V) c_l = -V^T A(omega) phi_bar_l (Eqs. localRB,
  localRBsystem); S_ll' and b_l from phi_rb by Eq. stiffness_local.

All matrices are formed explicitly from their definitions; the library
routines used as steps are numpy's Cholesky, eigh and solve.
"""
from __future__ import annotations

import numpy as np

_KREF = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]],
                 dtype=np.float64) / 6.0


def cell_stiffness(a_cell):
    """Full Q1 stiffness over the (rho+1)^2 nodes of one cell for the
    piecewise-constant coefficient a_cell[rho][rho] (y-major)."""
    rho = a_cell.shape[0]
    N = rho + 1
    A = np.zeros((N * N, N * N))
    for ey in range(rho):
        for ex in range(rho):
            idx = [ey * N + ex, ey * N + ex + 1, (ey + 1) * N + ex + 1, (ey + 1) * N + ex]
            for r in range(4):
                for c in range(4):
                    A[idx[r], idx[c]] += a_cell[ey, ex] * _KREF[r, c]
    return A


def interior_mask(rho):
    N = rho + 1
    m = np.zeros((N, N), dtype=bool)
    m[1:-1, 1:-1] = True
    return m.reshape(-1)


def load_weights(rho, f, h):
    """int f phi over the cell for a nodal vector phi: f h^2/4 times the
    number of cell elements touching each node."""
    N = rho + 1
    w = np.zeros((N, N))
    for ey in range(rho):
        for ex in range(rho):
            w[ey, ex] += 1
            w[ey, ex + 1] += 1
            w[ey + 1, ex + 1] += 1
            w[ey + 1, ex] += 1
    return (f * h * h / 4.0) * w.reshape(-1)


def cell_coef(a, nc, cx, cy):
    """a[..., nf, nf] -> the cell's block a[..., rho, rho]."""
    nf = a.shape[-1]
    rho = nf // nc
    return a[..., cy * rho:(cy + 1) * rho, cx * rho:(cx + 1) * rho]


def _kl_basis(X, R, n_nodes, inner, tol, max_rank, rank):
    """Eq. KLphi for centred snapshots X [n_interior][columns] in the energy
    inner product Abar = R R^T: eigenpairs of the covariance R^T X X^T R /
    columns, truncation, and the Abar-orthonormal modes R^{-T} w_q on the
    cell's nodes (zero on the boundary).  Returns (V, lam, rank)."""
    Y = R.T @ X
    C = (Y @ Y.T) / X.shape[1]                           # covariance in the energy metric
    lam, Wv = np.linalg.eigh(C)
    order = np.argsort(lam)[::-1]
    lam = lam[order]
    Wv = Wv[:, order]
    if rank is None:
        lam1 = lam[0] if lam[0] > 0 else 1.0
        keep = np.sqrt(np.maximum(lam, 0.0) / lam1) >= tol
        rank = int(np.sum(keep))
        if max_rank is not None:
            rank = min(rank, int(max_rank))
    rank = max(1, min(rank, X.shape[0]))
    Z = np.linalg.solve(R.T, Wv[:, :rank])               # zeta_q = R^{-T} w_q (Abar-orthonormal)
    V = np.zeros((n_nodes, rank))
    V[inner] = Z
    return V, lam, rank


def build_cell(phi_snap, a_train_cell, tol=1e-6, max_rank=None, rank=None):
    """phi_snap [Ns][4][(rho+1)^2] training basis functions of one cell;
    a_train_cell [Ns][rho][rho].  Returns dict(phibar[4][N2], V[N2][r]
    (zero on the boundary), lam (all eigenvalues, descending), rank)."""
    Ns = phi_snap.shape[0]
    rho = a_train_cell.shape[-1]
    inner = interior_mask(rho)
    phibar = phi_snap.mean(axis=0)                       # [4][N2]
    abar = a_train_cell.mean(axis=0)                     # [rho][rho]
    Abar = cell_stiffness(abar)[np.ix_(inner, inner)]    # energy inner product on H^1_0
    X = (phi_snap - phibar[None]).transpose(1, 0, 2).reshape(4 * Ns, -1)[:, inner].T  # n x 4Ns
    R = np.linalg.cholesky(Abar)                         # Abar = R R^T
    V, lam, rank = _kl_basis(X, R, phi_snap.shape[-1], inner, tol, max_rank, rank)
    return {"phibar": phibar, "V": V, "lam": lam, "rank": rank, "abar": abar}


def build_cell_per_l(phi_snap, a_train_cell, tol=1e-6, max_rank=None, ranks=None):
    """One reduced basis per basis function, the reading of the patch study
    (Sec. 5.1: the KL expansions of phi^1, phi^2, phi^3 separately, 15, 13
    and 15 modes there); phi^4 follows from the partition of unity.
    Returns dict(phibar[4][N2], V [three arrays N2 x r_l], lam [three
    spectra], rank [r_1, r_2, r_3], abar)."""
    Ns = phi_snap.shape[0]
    rho = a_train_cell.shape[-1]
    inner = interior_mask(rho)
    phibar = phi_snap.mean(axis=0)
    abar = a_train_cell.mean(axis=0)
    R = np.linalg.cholesky(cell_stiffness(abar)[np.ix_(inner, inner)])
    Vs, lams, rks = [], [], []
    for l in range(3):
        X = (phi_snap[:, l] - phibar[l][None])[:, inner].T   # n x Ns
        V, lam, r = _kl_basis(X, R, phi_snap.shape[-1], inner, tol, max_rank,
                              None if ranks is None else int(ranks[l]))
        Vs.append(V)
        lams.append(lam)
        rks.append(r)
    return {"phibar": phibar, "V": Vs, "lam": lams, "rank": rks, "abar": abar, "per_l": True}


def online_cell(model, a_cell, f, h):
    """Alg. 4 for one cell and one sample: returns (Ke[10], be[4])."""
    A = cell_stiffness(a_cell)
    V = model["V"]
    phibar = model["phibar"]
    M = V.T @ A @ V
    F = -(V.T @ A @ phibar.T)                            # r x 4
    c = np.linalg.solve(M, F)                            # r x 4
    phi_rb = phibar.T + V @ c                            # N2 x 4
    S = phi_rb.T @ A @ phi_rb
    rho = a_cell.shape[-1]
    b = load_weights(rho, f, h) @ phi_rb
    Ke = np.array([S[l, lp] for l in range(4) for lp in range(l, 4)])
    return Ke, b


def online_cell_per_l(model, a_cell, f, h):
    """Alg. 4 with one basis per basis function: for l = 1..3 the Galerkin
    system (V_l^T A V_l) c_l = -V_l^T A phi_bar_l, phi_rb,l = phi_bar_l +
    V_l c_l; phi_rb,4 = 1 - sum_l phi_rb,l; S and b by Eq.
    stiffness_local.  Returns (Ke[10], be[4])."""
    A = cell_stiffness(a_cell)
    phibar = model["phibar"]
    phi_rb = np.empty((phibar.shape[1], 4))
    for l in range(3):
        V = model["V"][l]
        c = np.linalg.solve(V.T @ A @ V, -(V.T @ A @ phibar[l]))
        phi_rb[:, l] = phibar[l] + V @ c
    phi_rb[:, 3] = 1.0 - phi_rb[:, :3].sum(axis=1)
    S = phi_rb.T @ A @ phi_rb
    b = load_weights(a_cell.shape[-1], f, h) @ phi_rb
    Ke = np.array([S[l, lp] for l in range(4) for lp in range(l, 4)])
    return Ke, b


def build_per_l(nf, nc, phi_train, a_train, tol=1e-6, max_rank=None):
    """Per-cell models with one basis per basis function (build_cell_per_l)."""
    return [build_cell_per_l(phi_train[:, cell], cell_coef(a_train, nc, cell % nc, cell // nc), tol=tol,
                             max_rank=max_rank) for cell in range(nc * nc)]


def upscale_per_l(models, nf, nc, f, a):
    """a [S][nf][nf] -> Ke [S][nc*nc][10], be [S][nc*nc][4] with per-l bases."""
    S = a.shape[0]
    Ke = np.empty((S, nc * nc, 10))
    be = np.empty((S, nc * nc, 4))
    h = 1.0 / nf
    for s in range(S):
        for cell in range(nc * nc):
            Ke[s, cell], be[s, cell] = online_cell_per_l(models[cell], cell_coef(a[s], nc, cell % nc, cell // nc),
                                                         f, h)
    return Ke, be


def build(nf, nc, phi_train, a_train, tol=1e-6, max_rank=None, ranks=None):
    """phi_train [Ns][nc*nc][4][(rho+1)^2], a_train [Ns][nf][nf] -> list of
    per-cell models (cell index cy*nc+cx)."""
    models = []
    for cell in range(nc * nc):
        cx, cy = cell % nc, cell // nc
        models.append(build_cell(phi_train[:, cell], cell_coef(a_train, nc, cx, cy), tol=tol,
                                 max_rank=max_rank,
                                 rank=None if ranks is None else int(ranks[cell])))
    return models


def upscale(models, nf, nc, f, a):
    """a [S][nf][nf] -> Ke [S][nc*nc][10], be [S][nc*nc][4]."""
    S = a.shape[0]
    Ke = np.empty((S, nc * nc, 10))
    be = np.empty((S, nc * nc, 4))
    h = 1.0 / nf
    for s in range(S):
        for cell in range(nc * nc):
            cx, cy = cell % nc, cell // nc
            Ke[s, cell], be[s, cell] = online_cell(models[cell], cell_coef(a[s], nc, cx, cy), f, h)
    return Ke, be


def affine_cell_coef(nf, nc, field, xi_row, cell, local_ids):
    """Eq. RBaffine restricted to the cell's local parameters: the affine
    field's coefficient on the cell with every non-local xi_i set to 0."""
    from . import sample_coef_window
    rho = nf // nc
    cx, cy = cell % nc, cell // nc
    x = np.zeros_like(np.asarray(xi_row, dtype=np.float64))
    ids = [int(i) for i in local_ids if i >= 0]
    x[ids] = np.asarray(xi_row)[ids]
    a = sample_coef_window(nf, field, x, cx * rho, (cx + 1) * rho, cy * rho, (cy + 1) * rho)
    return a[cy * rho:(cy + 1) * rho, cx * rho:(cx + 1) * rho]


def upscale_affine(models, nf, nc, f, field, xi, local_ids):
    """Alg. 4 on the local affine coefficient of every (sample, cell):
    K_e [S][nc*nc][10], b_e [S][nc*nc][4].  local_ids [nc*nc][16]."""
    S = xi.shape[0]
    Ke = np.empty((S, nc * nc, 10))
    be = np.empty((S, nc * nc, 4))
    h = 1.0 / nf
    for s in range(S):
        for cell in range(nc * nc):
            a_cell = affine_cell_coef(nf, nc, field, xi[s], cell, local_ids[cell])
            Ke[s, cell], be[s, cell] = online_cell(models[cell], a_cell, f, h)
    return Ke, be


def reduced_matrix(model, a_cell):
    """W^T A(a) W with W = [phibar_1..4, V] (the reduced quantities of Eq.
    localRBsystem and of the K_e assembly)."""
    Wf = np.concatenate([model["phibar"].T, model["V"]], axis=1)
    return Wf.T @ cell_stiffness(a_cell) @ Wf
