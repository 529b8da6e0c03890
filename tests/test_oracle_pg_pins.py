"""Pins of the Petrov-Galerkin oracle (Eq. stiffness_local_petrov: bilinear
test functions, deterministic load; non-symmetric coarse system), no GPU."""
import numpy as np
import pytest

from paper_1607_00693_gb300 import workloads as W

KREF = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
CDX, CDY = [0, 1, 1, 0], [0, 0, 1, 1]
FIELD = dict(kind=0, nbx=4, nby=4, width=0.1, scale=1.0)


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _coef(orc, nf, S, seed):
    return orc.sample_coef(nf, FIELD, W.draw_xi(FIELD, S, seed))


def test_pg_equals_galerkin_without_oversampling(orc):
    """o = 0: phi_l - q_l vanishes on the cell boundary and phi_l is
    discrete-harmonic, so a(phi_l, q_l') = a(phi_l, phi_l'); the load is
    f H^2 / 4 for every corner."""
    nf, nc, f = 32, 4, 1.3
    a = _coef(orc, nf, 1, 5)[0]
    for cell in range(nc * nc):
        cx, cy = cell % nc, cell // nc
        K, b = orc.cell_pg(nf, nc, f, a, cx, cy, 0)
        Kg, _, _, _ = orc.cell(nf, nc, f, a, cx, cy, 0)
        np.testing.assert_allclose(K, orc.unpack_upper(Kg), rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(b, np.full(4, f / nc ** 2 / 4), rtol=1e-15)


@pytest.mark.parametrize("o", [0, 1, 2, 3])
def test_pg_constant_coefficient_is_reference_stiffness(orc, o):
    """a = c: the oversampled basis is the cell's bilinear basis itself, so
    S_pg = c K_ref for every cell, boundary-clipped patches included."""
    nf, nc, c = 32, 4, 2.5
    a = np.full((nf, nf), c)
    for cell in range(nc * nc):
        K, _ = orc.cell_pg(nf, nc, 1.0, a, cell % nc, cell // nc, o)
        np.testing.assert_allclose(K, c * KREF, atol=1e-12)


@pytest.mark.parametrize("o", [1, 2, 3])
def test_pg_row_and_column_sums_vanish(orc, o):
    """Sum over test functions is 1 (zero row sums) and the recombined trial
    basis sums to 1 (zero column sums); with oversampling S_pg is not
    symmetric."""
    nf, nc = 32, 4
    a = _coef(orc, nf, 1, 9)[0]
    asym = 0.0
    for cell in (0, 5, 10, 15):
        K, _ = orc.cell_pg(nf, nc, 1.0, a, cell % nc, cell // nc, o)
        scale = np.abs(K).max()
        assert np.abs(K.sum(axis=1)).max() < 1e-12 * scale
        assert np.abs(K.sum(axis=0)).max() < 1e-12 * scale
        asym = max(asym, np.abs(K - K.T).max() / scale)
    assert asym > 1e-4


def _cell_stiffness(a, nf, cx, cy, rho):
    """Dense fine stiffness of the cell's elements on its (rho+1)^2 nodes."""
    N = rho + 1
    A = np.zeros((N * N, N * N))
    for ey in range(rho):
        for ex in range(rho):
            ae = a[cy * rho + ey, cx * rho + ex]
            idx = [(ey + CDY[c]) * N + ex + CDX[c] for c in range(4)]
            A[np.ix_(idx, idx)] += ae * KREF
    return A


@pytest.mark.parametrize("o", [0, 2])
def test_pg_brute_force_cell_assembly(orc, o):
    """S_pg[l][l'] = phi_l^T A_cell q_l' with A_cell assembled densely here,
    phi from the oracle's basis output and q_l' the cell's bilinears."""
    nf, nc = 32, 4
    rho = nf // nc
    a = _coef(orc, nf, 1, 13)[0]
    N = rho + 1
    X, Y = np.meshgrid(np.arange(N) / rho, np.arange(N) / rho)
    q = np.stack([(1 - X) * (1 - Y), X * (1 - Y), X * Y, (1 - X) * Y]).reshape(4, -1)
    for cell in (3, 6):
        cx, cy = cell % nc, cell // nc
        _, _, phi, _ = orc.cell(nf, nc, 1.0, a, cx, cy, o)
        A = _cell_stiffness(a, nf, cx, cy, rho)
        K, _ = orc.cell_pg(nf, nc, 1.0, a, cx, cy, o)
        np.testing.assert_allclose(K, phi.reshape(4, -1) @ A @ q.T, rtol=1e-11, atol=1e-13)


def _dense_pg_system(nc, Kpg, bpg):
    """sum_I U_I a(phi_I, q_J) = (f, q_J) written out per definition."""
    mi = nc - 1
    G = np.zeros((mi * mi, mi * mi))
    r = np.zeros(mi * mi)
    node = lambda i, j: (j - 1) * mi + (i - 1) if 0 < i < nc and 0 < j < nc else None
    for cy in range(nc):
        for cx in range(nc):
            S = Kpg[cy * nc + cx].reshape(4, 4)
            for J in range(4):           # test corner
                gJ = node(cx + CDX[J], cy + CDY[J])
                if gJ is None:
                    continue
                r[gJ] += bpg[cy * nc + cx, J]
                for I in range(4):       # trial corner
                    gI = node(cx + CDX[I], cy + CDY[I])
                    if gI is not None:
                        G[gJ, gI] += S[I, J]
    return G, r


@pytest.mark.parametrize("nc,o", [(4, 2), (8, 1)])
def test_pg_coarse_solve_matches_dense_library_solve(orc, nc, o):
    nf = 8 * nc
    a = _coef(orc, nf, 2, 21)
    ov = np.full(nc * nc, o, dtype=np.int8)
    Kpg, bpg = orc.upscale_pg(nf, nc, 1.0, a, ov)
    u = orc.coarse_solve_pg(nc, Kpg, bpg)
    for s in range(2):
        G, r = _dense_pg_system(nc, Kpg[s], bpg[s])
        assert np.abs(G - G.T).max() > 1e-6 * np.abs(G).max()
        x = np.linalg.solve(G, r)
        NN = nc + 1
        ui = u[s].reshape(NN, NN)[1:nc, 1:nc].reshape(-1)
        np.testing.assert_allclose(ui, x, rtol=1e-10, atol=1e-14)
        assert np.all(u[s].reshape(NN, NN)[[0, -1], :] == 0) and np.all(u[s].reshape(NN, NN)[:, [0, -1]] == 0)


def test_pg_coarse_constant_coefficient_equals_galerkin(orc):
    """a = 1 with oversampling: both forms are the coarse Q1 FEM."""
    nf, nc = 32, 4
    a = np.ones((1, nf, nf))
    ov = np.full(nc * nc, 2, dtype=np.int8)
    Kpg, bpg = orc.upscale_pg(nf, nc, 1.0, a, ov)
    Kg, bg = orc.upscale(nf, nc, 1.0, a, ov)
    np.testing.assert_allclose(orc.coarse_solve_pg(nc, Kpg, bpg), orc.coarse_solve(nc, Kg, bg),
                               rtol=1e-12, atol=1e-15)
