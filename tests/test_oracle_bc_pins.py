"""Pins of the oracle's coarse solve with mixed boundary data (prescribed
values on chosen node lines, zero flux on the rest of the boundary: the
anisotropy study of Sec. 5.2, Eqs. xsquarewave / ysquarewave), no GPU.
Closed forms that the Q1 discretisation reproduces exactly (linear and
harmonic-coordinate profiles, the 1D load solution with a zero-flux end),
a dense library solve, and the reduction to the plain zero-Dirichlet
solves, which are pinned on their own."""
import os
from fractions import Fraction

import numpy as np
import pytest

from tests import fem_ref
from paper_1607_00693_gb300 import workloads as W

KREF = fem_ref.KREF
KREF_PACKED = np.array([4, -1, -2, -1, 4, -1, -2, 4, -1, 4]) / 6.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "mixed_bc_layered_nc4.txt")


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _rho1(a_cells):
    """K_e (packed, and the 16-entry Petrov-Galerkin layout) and zero loads
    of H = h, where the cell problem is trivial: K_e = a_e K_ref."""
    nc = a_cells.shape[0]
    a = a_cells.reshape(-1)
    Kg = a[:, None] * KREF_PACKED[None]
    Kp = a[:, None] * KREF.reshape(1, 16)
    return Kg[None], Kp[None], np.zeros((1, nc * nc, 4))


def _lines(nc, iL, iR, gL, gR):
    NN = nc + 1
    m = np.zeros((NN, NN), dtype=np.uint8)
    g = np.zeros((NN, NN))
    m[:, iL] = m[:, iR] = 1
    g[:, iL], g[:, iR] = gL, gR
    return m.reshape(-1), g.reshape(-1)


def test_golden_layered_harmonic_coordinate(orc):
    """Hand-derived fractions of tests/golden/mixed_bc_layered_nc4.txt."""
    rows = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            rows[k] = v
    a_cols = np.array([float(x) for x in rows["a"]])
    T = np.array([float(Fraction(x)) for x in rows["T"]])
    nc = a_cols.size
    Kg, Kp, b = _rho1(np.tile(a_cols, (nc, 1)))
    m, g = _lines(nc, 0, nc, 0.0, 1.0)
    for pg, K in ((False, Kg), (True, Kp)):
        u = orc.coarse_solve_bc(nc, K, b, m, g, pg=pg)[0].reshape(nc + 1, nc + 1)
        np.testing.assert_allclose(u, np.tile(T, (nc + 1, 1)), rtol=0, atol=1e-15)


@pytest.mark.parametrize("pg", [False, True])
def test_constant_coefficient_between_interior_lines_is_linear(orc, pg):
    """a = c, u = 0 on x = iL H, 1 on x = iR H, zero flux elsewhere, no
    load: u is 0 left of the first line, linear between, 1 right of the
    second (bilinear functions are in the Q1 space and the constants solve
    the zero-flux parts)."""
    nc, iL, iR = 10, 2, 8
    Kg, Kp, b = _rho1(np.full((nc, nc), 2.5))
    m, g = _lines(nc, iL, iR, 0.0, 1.0)
    u = orc.coarse_solve_bc(nc, Kp if pg else Kg, b, m, g, pg=pg)[0].reshape(nc + 1, nc + 1)
    i = np.arange(nc + 1)
    ref = np.clip((i - iL) / (iR - iL), 0.0, 1.0)
    np.testing.assert_allclose(u, np.tile(ref, (nc + 1, 1)), rtol=0, atol=1e-13)


def test_layered_medium_gives_harmonic_coordinate(orc):
    """a = a(x) column-wise: between two lines the solution is the
    harmonic coordinate sum_{c<i} 1/a_c / sum 1/a_c, constant outside."""
    nc, iL, iR = 12, 1, 11
    rng = np.random.default_rng(7)
    a_cols = np.exp(rng.uniform(np.log(0.1), np.log(10.0), nc))
    Kg, Kp, b = _rho1(np.tile(a_cols, (nc, 1)))
    m, g = _lines(nc, iL, iR, 0.0, 1.0)
    inv = 1.0 / a_cols
    T = np.zeros(nc + 1)
    T[iL + 1:iR + 1] = np.cumsum(inv[iL:iR]) / inv[iL:iR].sum()
    T[iR:] = 1.0
    for pg, K in ((False, Kg), (True, Kp)):
        u = orc.coarse_solve_bc(nc, K, b, m, g, pg=pg)[0].reshape(nc + 1, nc + 1)
        np.testing.assert_allclose(u, np.tile(T, (nc + 1, 1)), rtol=0, atol=1e-13)


def test_load_with_zero_flux_ends_is_nodally_exact(orc):
    """a = 1, load f, u = 0 on x = xL and x = xR, zero flux on the rest:
    u depends on x alone and the 1D linear elements are nodally exact for
    -u'' = f, so u = f/2 (xL^2 - x^2) left of xL (u'(0) = 0), f/2 (x - xL)
    (xR - x) between, f/2 (x - xR)(2 - xR - x) right of xR (u'(1) = 0)."""
    nc, iL, iR, f = 10, 3, 7, 3.0
    H = 1.0 / nc
    Kg, Kp, _ = _rho1(np.ones((nc, nc)))
    b = np.full((1, nc * nc, 4), f * H * H / 4)
    m, g = _lines(nc, iL, iR, 0.0, 0.0)
    x = np.arange(nc + 1) * H
    xL, xR = iL * H, iR * H
    ref = np.where(x <= xL, 0.5 * f * (xL ** 2 - x ** 2),
                   np.where(x <= xR, 0.5 * f * (x - xL) * (xR - x), 0.5 * f * (x - xR) * (2 - xR - x)))
    for pg, K in ((False, Kg), (True, Kp)):
        u = orc.coarse_solve_bc(nc, K, b, m, g, pg=pg)[0].reshape(nc + 1, nc + 1)
        np.testing.assert_allclose(u, np.tile(ref, (nc + 1, 1)), rtol=1e-12, atol=1e-14)


def test_fine_grid_matches_dense_library_solve(orc):
    """H = h with a random coefficient, the square-wave lines of the
    workload along x and along y, and a load: the dense system of the test
    helper (all nodes, Dirichlet rows eliminated) solved by numpy."""
    nc, f = 9, 0.7
    rng = np.random.default_rng(3)
    a = np.exp(rng.uniform(np.log(0.2), np.log(5.0), (nc, nc)))
    Kg, Kp, _ = _rho1(a)
    H = 1.0 / nc
    b = np.full((1, nc * nc, 4), f * H * H / 4)
    A = fem_ref.stiffness(a)
    F = np.zeros((nc + 1) ** 2)
    for ey in range(nc):
        for ex in range(nc):
            for (j, i) in [(ey, ex), (ey, ex + 1), (ey + 1, ex + 1), (ey + 1, ex)]:
                F[j * (nc + 1) + i] += f * H * H / 4
    for axis in ("x", "y"):
        m, g = W.mixed_bc(nc, axis=axis, lines=(0.2, 0.7), period=0.4)
        d = m.astype(bool)
        ref = g.copy()
        ref[~d] = np.linalg.solve(A[np.ix_(~d, ~d)], F[~d] - A[np.ix_(~d, d)] @ g[d])
        for pg, K in ((False, Kg), (True, Kp)):
            u = orc.coarse_solve_bc(nc, K, b, m, g, pg=pg)[0]
            np.testing.assert_allclose(u, ref, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("o", [0, 2])
def test_zero_dirichlet_boundary_reduces_to_plain_solves(orc, o):
    """Dirichlet on the boundary ring with g = 0 is the problem of the plain
    coarse solves (Galerkin and the non-symmetric Petrov-Galerkin one with
    oversampling), so all agree."""
    nf, nc, f = 32, 4, 1.1
    field = dict(kind=0, nbx=4, nby=4, width=0.1, scale=1.0)
    a = orc.sample_coef(nf, field, W.draw_xi(field, 2, 12))
    over = np.full(nc * nc, o, dtype=np.int8)
    m = fem_ref.boundary_mask(nc, nc).astype(np.uint8)
    g = np.zeros((nc + 1) ** 2)
    Ke, be = orc.upscale(nf, nc, f, a, over)
    np.testing.assert_allclose(orc.coarse_solve_bc(nc, Ke, be, m, g), orc.coarse_solve(nc, Ke, be),
                               rtol=1e-12, atol=1e-15)
    Kp, bp = orc.upscale_pg(nf, nc, f, a, over)
    if o:
        assert np.abs(Kp - Kp.reshape(2, -1, 4, 4).transpose(0, 1, 3, 2).reshape(2, -1, 16)).max() > 1e-6
    np.testing.assert_allclose(orc.coarse_solve_bc(nc, Kp, bp, m, g, pg=True), orc.coarse_solve_pg(nc, Kp, bp),
                               rtol=1e-12, atol=1e-15)


def test_workload_lines_snap_to_nodes():
    """The boundary-data generator: lines x = 0.1 and 0.9 at nc = 20 (the
    high-contrast example's H = 0.05) are node columns 2 and 18, carrying
    the square wave; nothing else is prescribed."""
    m, g = W.mixed_bc(20, axis="x")
    m = m.reshape(21, 21)
    assert set(np.nonzero(m.any(axis=0))[0]) == {2, 18} and m[:, [2, 18]].all()
    gy = g.reshape(21, 21)[:, 2]
    assert set(np.unique(gy)) == {0.0, 1.0}
    m2, _ = W.mixed_bc(20, axis="y")
    assert (m2.reshape(21, 21).T == m).all()
