"""Pins of the oracle's oscillatory boundary data for the cell problems (the
MsFEM option of the short-correlation example, Sec. 5.3: on every patch edge
the nodal function interpolates its corner values linearly in the edge's
harmonic coordinate, the solution of the reduced 1D problem (a u')' = 0),
no GPU.  Closed forms (constant coefficient; layered media, where the cell
solution is a tensor product and K_e follows from 1D sums), symmetries of
the square (reflections and the transpose, which catch a wrong choice of
the elements along an edge), the reduced problem's constant flux, and the
invariants of the basis."""
import numpy as np
import pytest

from paper_1607_00693_gb300 import workloads as W

KREF_PACKED = np.array([4, -1, -2, -1, 4, -1, -2, 4, -1, 4]) / 6.0
KREF = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])          # 1D element stiffness (times h)
M1 = np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0      # 1D element mass (over h)
# corner l = (x index, y index) of the tensor factors: SW, SE, NE, NW
CORNER = [(0, 0), (1, 0), (1, 1), (0, 1)]


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _unpack(k):
    M = np.zeros((4, 4))
    q = 0
    for l in range(4):
        for lp in range(l, 4):
            M[l, lp] = M[lp, l] = k[q]
            q += 1
    return M


def _one_d(coef, U, V, Mat):
    """sum over the 1D elements c of coef_c * U[:, c:c+2] Mat V[:, c:c+2]^T."""
    out = np.zeros((2, 2))
    for c in range(len(coef)):
        out += coef[c] * U[:, c:c + 2] @ Mat @ V[:, c:c + 2].T
    return out


def _harmonic(coef):
    inv = 1.0 / np.asarray(coef)
    T = np.r_[0.0, np.cumsum(inv)] / inv.sum()
    return np.stack([1.0 - T, T])


def _linear(n):
    s = np.arange(n + 1) / n
    return np.stack([1.0 - s, s])


def _tensor_K(Ex, Mx, Ey, My):
    """K[(i,k),(j,l)] = Ex[i,j] My[k,l] + Mx[i,j] Ey[k,l] over the corners."""
    K = np.zeros((4, 4))
    for r, (i, k) in enumerate(CORNER):
        for c, (j, l) in enumerate(CORNER):
            K[r, c] = Ex[i, j] * My[k, l] + Mx[i, j] * Ey[k, l]
    return K


@pytest.mark.parametrize("o", [0, 1, 2, 3])
def test_constant_coefficient_is_reference_stiffness(orc, o):
    """a = c: the harmonic coordinate is arc length, so the data are the
    bilinear ones and K_e = c K_ref (clipped patches included); the
    Petrov-Galerkin matrix is c K_ref too."""
    nf, nc, c, f = 32, 4, 2.7, 1.3
    a = np.full((1, nf, nf), c)
    ov = np.full(nc * nc, o, dtype=np.int8)
    Ke, be = orc.upscale(nf, nc, f, a, ov, bc=orc.BC_OSCILLATORY)
    np.testing.assert_allclose(Ke[0], np.tile(c * KREF_PACKED, (nc * nc, 1)), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(be[0], f / nc ** 2 / 4, rtol=1e-12)
    Kp, _ = orc.upscale_pg(nf, nc, f, a, ov, bc=orc.BC_OSCILLATORY)
    np.testing.assert_allclose(Kp[0], np.tile(c * KREF.reshape(16), (nc * nc, 1)), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_layered_medium_tensor_closed_form(orc, axis):
    """a = a(x) column-wise (or a(y) row-wise), no oversampling: the edge data
    are the harmonic coordinate across the layers and linear along them, the
    product of the two is discrete-harmonic (the Q1 matrix is the tensor
    sum of 1D stiffness and mass), so the basis is that product and K_e is
    E_x (x) M_y + M_x (x) E_y of 1D sums; with bilinear test functions the
    Petrov-Galerkin matrix is the same sum with the linear 1D factors on
    the test side."""
    nf, nc = 32, 4
    rho = nf // nc
    rng = np.random.default_rng(17)
    prof = np.exp(rng.uniform(np.log(0.05), np.log(20.0), nf))
    a2 = np.tile(prof, (nf, 1)) if axis == "x" else np.tile(prof[:, None], (1, nf))
    ones = np.ones(rho)
    for cx, cy in [(0, 0), (2, 1), (3, 3)]:
        layers = prof[(cx if axis == "x" else cy) * rho:((cx if axis == "x" else cy) + 1) * rho]
        Hx, Lx = _harmonic(layers), _linear(rho)
        Ke, _, _, _ = orc.cell(nf, nc, 1.0, a2, cx, cy, 0, bc=orc.BC_OSCILLATORY)
        Kp, _ = orc.cell_pg(nf, nc, 1.0, a2, cx, cy, 0, bc=orc.BC_OSCILLATORY)
        if axis == "x":
            ref = _tensor_K(_one_d(layers, Hx, Hx, K1), _one_d(layers, Hx, Hx, M1),
                            _one_d(ones, Lx, Lx, K1), _one_d(ones, Lx, Lx, M1))
            ref_pg = _tensor_K(_one_d(layers, Hx, Lx, K1), _one_d(layers, Hx, Lx, M1),
                               _one_d(ones, Lx, Lx, K1), _one_d(ones, Lx, Lx, M1))
        else:
            ref = _tensor_K(_one_d(ones, Lx, Lx, K1), _one_d(ones, Lx, Lx, M1),
                            _one_d(layers, Hx, Hx, K1), _one_d(layers, Hx, Hx, M1))
            ref_pg = _tensor_K(_one_d(ones, Lx, Lx, K1), _one_d(ones, Lx, Lx, M1),
                               _one_d(layers, Hx, Lx, K1), _one_d(layers, Hx, Lx, M1))
        np.testing.assert_allclose(_unpack(Ke), ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())
        np.testing.assert_allclose(Kp, ref_pg, rtol=1e-11, atol=1e-12 * np.abs(ref_pg).max())
        # across the layers the energy is the harmonic mean, a_harm = rho / sum(1/a)
        # (the 1D E of the harmonic coordinate), not the bilinear data's value
        Eh = _one_d(layers, Hx, Hx, K1)
        np.testing.assert_allclose(Eh[0, 0], rho / np.sum(1.0 / layers) / rho, rtol=1e-12)


def _reflect(a, nf, kind):
    if kind == "x":
        return a[:, ::-1].copy()
    if kind == "y":
        return a[::-1, :].copy()
    return a.T.copy()


def _map_cell(cx, cy, nc, kind):
    if kind == "x":
        return nc - 1 - cx, cy
    if kind == "y":
        return cx, nc - 1 - cy
    return cy, cx


PERM = {"x": [1, 0, 3, 2], "y": [3, 2, 1, 0], "t": [0, 3, 2, 1]}


@pytest.mark.parametrize("kind", ["x", "y", "t"])
@pytest.mark.parametrize("o", [0, 2])
def test_symmetries_of_the_square(orc, kind, o):
    """Reflecting the medium in x or y, or transposing it, maps the unit of
    cell (cx, cy) onto the mirrored cell with the corners permuted, for
    both boundary data; an edge taking its coefficient from the wrong row
    or column of elements breaks this."""
    nf, nc = 32, 4
    field = dict(kind=0, nbx=4, nby=4, width=0.1, scale=1.0)
    a = orc.sample_coef(nf, field, W.draw_xi(field, 1, 23))[0]
    a = a * np.exp(np.random.default_rng(5).normal(0.0, 0.5, a.shape))  # no lattice symmetry left
    ar = _reflect(a, nf, kind)
    P = PERM[kind]
    for bc in (orc.BC_BILINEAR, orc.BC_OSCILLATORY):
        for cx, cy in [(0, 0), (1, 2), (3, 1)]:
            K, b, _, _ = orc.cell(nf, nc, 1.0, a, cx, cy, o, bc=bc)
            mx, my = _map_cell(cx, cy, nc, kind)
            Kr, br, _, _ = orc.cell(nf, nc, 1.0, ar, mx, my, o, bc=bc)
            np.testing.assert_allclose(_unpack(Kr)[np.ix_(P, P)], _unpack(K), rtol=1e-11,
                                       atol=1e-12 * np.abs(K).max())
            np.testing.assert_allclose(br[P], b, rtol=1e-11, atol=1e-15)


def test_edge_data_solve_the_reduced_problem(orc):
    """On each edge of the patch the data of every nodal function carry a
    constant 1D flux a_e (u_{e+1} - u_e) with a_e the element next to the
    segment, and run from its corner values (0 or 1)."""
    nf, nc, o = 32, 4, 2
    rng = np.random.default_rng(9)
    a = np.exp(rng.uniform(np.log(0.1), np.log(10.0), (nf, nf)))
    cx, cy = 1, 2
    x0, x1, y0, y1 = orc.patch_bounds(nf, nc, cx, cy, o)
    _, _, _, psi = orc.cell(nf, nc, 1.0, a, cx, cy, o, bc=orc.BC_OSCILLATORY)
    edges = {  # (values along the edge [l][k], coefficients of the adjacent elements)
        "bottom": (psi[:, 0, :], a[y0, x0:x1]),
        "top": (psi[:, -1, :], a[y1 - 1, x0:x1]),
        "left": (psi[:, :, 0], a[y0:y1, x0]),
        "right": (psi[:, :, -1], a[y0:y1, x1 - 1]),
    }
    for name, (vals, coef) in edges.items():
        for l in range(4):
            flux = coef * np.diff(vals[l])
            np.testing.assert_allclose(flux, flux.mean(), rtol=1e-12, atol=1e-15, err_msg=name)
            assert vals[l][0] in (0.0, 1.0) and vals[l][-1] in (0.0, 1.0)
        np.testing.assert_allclose(vals.sum(axis=0), 1.0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("o", [0, 1, 3])
def test_invariants(orc, o):
    """Symmetric positive semidefinite K_e with zero row sums, sum_l phi_l = 1
    on the cell, phi_l nodal at the cell corners, sum_l b_l = f H^2."""
    nf, nc, f = 32, 4, 0.8
    rho = nf // nc
    field = dict(kind=0, nbx=4, nby=4, width=0.1, scale=1.0)
    a = orc.sample_coef(nf, field, W.draw_xi(field, 2, 29))
    ov = np.full(nc * nc, o, dtype=np.int8)
    Ke, be, phi = orc.upscale(nf, nc, f, a, ov, want_phi=True, bc=orc.BC_OSCILLATORY)
    for k, b, ph in zip(Ke.reshape(-1, 10), be.reshape(-1, 4), phi.reshape(-1, 4, (rho + 1) ** 2)):
        M = _unpack(k)
        scale = np.abs(M).max()
        np.testing.assert_allclose(M.sum(axis=1), 0.0, atol=1e-12 * scale)
        assert np.linalg.eigvalsh(M).min() > -1e-12 * scale
        np.testing.assert_allclose(ph.sum(axis=0), 1.0, atol=1e-12)
        corners = [0, rho, (rho + 1) ** 2 - 1, rho * (rho + 1)]
        np.testing.assert_allclose(ph[:, corners], np.eye(4), atol=1e-12)
        np.testing.assert_allclose(b.sum(), f / nc ** 2, rtol=1e-12)


def test_golden_single_interior_node(orc):
    """Hand-derived centre values of tests/golden/cell_rho2_centre.txt for
    both boundary data (one interior node, H = 2h)."""
    import os
    from fractions import Fraction
    rows = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "cell_rho2_centre.txt")):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            rows[k] = v
    a = np.array([float(x) for x in rows["a"]]).reshape(2, 2)
    for bc, key in ((orc.BC_BILINEAR, "bilinear"), (orc.BC_OSCILLATORY, "oscillatory")):
        ref = np.array([float(Fraction(x)) for x in rows[key]])
        _, _, _, psi = orc.cell(2, 1, 1.0, a, 0, 0, 0, bc=bc)
        np.testing.assert_allclose(psi[:, 1, 1], ref, rtol=0, atol=1e-15)


def test_oscillatory_data_change_a_rough_medium(orc):
    """The option does something: in a rough medium the oscillatory and the
    bilinear data give different K_e (by far more than rounding), while both
    keep the invariants above."""
    nf, nc = 32, 4
    rng = np.random.default_rng(31)
    a = np.exp(rng.uniform(np.log(0.1), np.log(10.0), (1, nf, nf)))
    K0, _ = orc.upscale(nf, nc, 1.0, a)
    K1_, _ = orc.upscale(nf, nc, 1.0, a, bc=orc.BC_OSCILLATORY)
    assert np.abs(K1_ - K0).max() > 1e-3 * np.abs(K0).max()
