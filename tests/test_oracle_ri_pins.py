"""Pins of the random-interpolation oracle (Sec. 3.1, Algorithms 1-2), no GPU."""
import itertools
import math

import numpy as np
import pytest

from paper_1607_00693_gb300 import workloads as W


@pytest.fixture(scope="module")
def orc():
    import oracle
    from oracle import ri
    oracle.build()
    return oracle, ri


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("nu", [0, 1, 2, 4, 8])
def test_nodes_are_polynomial_zeros(orc, kind, nu):
    """Chebyshev nodes are the zeros of T_{nu+1}, Legendre nodes those of
    P_{nu+1}; ascending, inside (-1, 1), symmetric about 0."""
    _, ri = orc
    x = ri.nodes(kind, nu)
    assert len(x) == nu + 1 and np.all(np.diff(x) > 0) and np.all(np.abs(x) < 1)
    np.testing.assert_allclose(x, -x[::-1], atol=1e-15)
    c = np.zeros(nu + 2)
    c[-1] = 1.0
    val = np.polynomial.chebyshev.chebval(x, c) if kind == 0 else np.polynomial.legendre.legval(x, c)
    assert np.max(np.abs(val)) < 1e-13
    if nu == 1:  # closed forms
        np.testing.assert_allclose(x[1], 1 / math.sqrt(2) if kind == 0 else 1 / math.sqrt(3), rtol=1e-15)


@pytest.mark.parametrize("nu", [1, 2, 3, 5, 8])
def test_lagrange_basis(orc, nu):
    """l_j(x_i) = delta_ij; sum_j l_j = 1; degree <= nu is reproduced and the
    error at degree nu + 1 is the nodal polynomial prod_k (t - x_k)."""
    _, ri = orc
    x = ri.nodes(0, nu)
    for i in range(nu + 1):
        np.testing.assert_allclose(ri.lagrange(x, x[i]), np.eye(nu + 1)[i], atol=1e-14)
    for t in np.linspace(-1, 1, 17):
        l = ri.lagrange(x, t)
        assert abs(l.sum() - 1) < 1e-13
        for p in range(nu + 1):
            assert abs(l @ x ** p - t ** p) < 1e-12
        assert abs((t ** (nu + 1) - l @ x ** (nu + 1)) - np.prod(t - x)) < 1e-12


@pytest.mark.parametrize("g", [1.0, 0.21, 0.044, 2e-3])
@pytest.mark.parametrize("eps", [1e-2, 1e-3, 1e-4])
def test_degree_rule_bounds_exp_interpolation(orc, g, eps):
    """The chosen degree interpolates exp(g t) on [-1, 1] within 2 eps (the
    rule bounds the first neglected Chebyshev coefficient), and one degree
    less does not meet the rule."""
    _, ri = orc
    nu = ri.choose_nu(g, eps, 12)
    t = np.linspace(-1, 1, 401)
    x = ri.nodes(0, nu)
    err = max(abs(ri.lagrange(x, s) @ np.exp(g * x) - math.exp(g * s)) for s in t)
    assert err <= 2 * eps
    if nu > 0:
        assert 2 * (g / 2) ** nu / math.factorial(nu) > eps


def _poly_model(ri, radices, coef, kind=0):
    """A fake one-family model whose data are a polynomial of per-direction
    degree < radix, so its interpolant must reproduce it exactly."""
    dims = [(0, k, r - 1, k) for k, r in enumerate(radices)]
    xs = [ri.nodes(kind, r - 1) for r in radices]
    rows = []
    for idx in itertools.product(*[range(r) for r in radices]):
        pt = np.array([xs[k][i] for k, i in enumerate(idx)])
        rows.append(coef(pt))
    return dict(kind=kind, dims=[dims], fam=np.array([0]), V=[np.array(rows)])


def test_tensor_interpolant_reproduces_anisotropic_polynomials(orc):
    """Direction k of degree nu_k: t0^2 t1 t2^3 (radices 3, 2, 4) and mixed
    terms are exact; a transposed grid enumeration would not be."""
    _, ri = orc
    radices = [3, 2, 4]

    def f(p):
        base = p[0] ** 2 * p[1] * p[2] ** 3 + 0.5 * p[0] - 2 * p[2] ** 2 + 0.25 * p[1] * p[2]
        return np.array([base * (q + 1) for q in range(14)])

    m = _poly_model(ri, radices, f)
    rng = np.random.default_rng(7)
    for _ in range(20):
        t = rng.uniform(-1, 1, 3)
        K, b = ri.evaluate(m, t, 0)
        np.testing.assert_allclose(np.concatenate([K, b]), f(t), rtol=1e-12, atol=1e-12)
    # a degree above a direction's radix is not reproduced
    m2 = _poly_model(ri, [2, 2, 2], lambda p: np.full(14, p[1] ** 2))
    K, _ = ri.evaluate(m2, np.array([0.3, 0.2, -0.4]), 0)
    assert abs(K[0] - 0.04) > 1e-3


@pytest.fixture(scope="module")
def model64(orc):
    _, ri = orc
    w = W.workload("msfem_64")
    return w, ri.build(w["nf"], w["nc"], w["f"], w["field"], 1e-3, 8, ri.LEGENDRE)


def test_collocation_data_are_direct_upscales_for_every_cell_of_a_family(orc, model64):
    """At a grid point the interpolant returns the data, and the data built on
    the family's first cell equal the direct FP64 upscale of ANOTHER cell of
    the family at the same local parameters (the translation reading)."""
    oracle, ri = orc
    w, m = model64
    nf, nc, fld = w["nf"], w["nc"], w["field"]
    rho = nf // nc
    K = W.n_vars(fld)
    rng = np.random.default_rng(3)
    checked = 0
    for fm in range(len(m["keys"])):
        cells = np.flatnonzero(m["fam"] == fm)
        if len(cells) < 2:
            continue
        cell = int(cells[-1])
        d = m["dims"][cell]
        xs = [ri.nodes(m["kind"], nu) for (_, _, nu, _) in d]
        grid = list(itertools.product(*[range(len(x)) for x in xs]))
        for p in rng.choice(len(grid), size=min(3, len(grid)), replace=False):
            xi = np.zeros(K)
            for k, (_, _, _, var) in enumerate(d):
                xi[var] = xs[k][grid[p][k]]
            cx, cy = cell % nc, cell // nc
            a = oracle.sample_coef_window(nf, fld, xi, cx * rho, (cx + 1) * rho, cy * rho, (cy + 1) * rho)
            Kd, bd, _, _ = oracle.cell(nf, nc, w["f"], a, cx, cy, 0)
            np.testing.assert_allclose(m["V"][fm][p], np.concatenate([Kd, bd]), rtol=1e-11, atol=1e-13)
            Ki, bi = ri.evaluate(m, xi, cell)
            np.testing.assert_allclose(np.concatenate([Ki, bi]), m["V"][fm][p], rtol=1e-11, atol=1e-13)
            checked += 1
    assert checked >= 10


def test_interpolation_converges_and_meets_target(orc):
    """Thm. approx_S: the error against the direct upscale of the full
    coefficient falls as eps (hence every nu) tightens, and at eps = 1e-3
    the coarse solution is within 1e-4 of the direct one."""
    oracle, ri = orc
    w = W.workload("msfem_64")
    nf, nc, f, fld = w["nf"], w["nc"], w["f"], w["field"]
    xi = W.draw_xi(fld, 6, 123)
    a = oracle.sample_coef(nf, fld, xi)
    K0, b0 = oracle.upscale(nf, nc, f, a)
    u0 = oracle.coarse_solve(nc, K0, b0)
    errs = []
    for eps in (3e-2, 3e-3, 1e-3):
        m = ri.build(nf, nc, f, fld, eps, 8, ri.CHEBYSHEV)
        K1, b1, fb = ri.upscale(m, xi, a)
        assert not fb.any()
        errs.append(np.abs(K1 - K0).max() / np.abs(K0).max())
        u1 = oracle.coarse_solve(nc, K1, b1)
    assert errs[0] > errs[1] > errs[2]
    assert np.linalg.norm(u1 - u0) / np.linalg.norm(u0) < 1e-4


def test_box_exit_falls_back_to_direct(orc, model64):
    """A local parameter outside [-1, 1] sends the unit to the direct upscale
    (remark closing Sec. 3.1.1); frozen directions do not."""
    oracle, ri = orc
    w, m = model64
    nf, nc, f, fld = w["nf"], w["nc"], w["f"], w["field"]
    xi = W.draw_xi(fld, 2, 5)
    cell = 9
    var = m["dims"][cell][-1][3]
    xi[0, var] = 1.5
    local = {v for (_, _, _, v) in m["dims"][cell]}
    frozen = min(set(range(W.n_vars(fld))) - local)
    xi[1, frozen] = 5.0
    a = oracle.sample_coef(nf, fld, xi)
    K, b, fb = ri.upscale(m, xi, a)
    assert fb[0, cell] == 1 and fb[1, cell] == 0
    assert all(fb[1, c] == (frozen in {v for (_, _, _, v) in m["dims"][c]}) for c in range(nc * nc))
    Kd, bd, _, _ = oracle.cell(nf, nc, f, a[0], cell % nc, cell // nc, 0)
    np.testing.assert_array_equal(K[0, cell], Kd)
    with pytest.raises(ValueError):
        ri.upscale(m, xi, None)


def test_all_frozen_is_the_mean_field_upscale(orc):
    """eps above every strength freezes every bump: one grid point per cell,
    the upscale of a = exp(0) = 1, i.e. the Q1 reference stiffness with
    zero row sums and b = f H^2 / 4."""
    oracle, ri = orc
    nf, nc = 32, 4
    fld = dict(kind=0, nbx=4, nby=4, width=0.1, scale=1.0)
    m = ri.build(nf, nc, 1.0, fld, 10.0, 8)
    assert len(m["keys"]) == 1 and len(m["V"][0]) == 1
    K, b = ri.evaluate(m, np.zeros(16), 5)
    np.testing.assert_allclose(K, np.array([4, -1, -2, -1, 4, -1, -2, 4, -1, 4]) / 6.0, atol=1e-12)
    np.testing.assert_allclose(b, np.full(4, 1.0 / 16 / 4), rtol=1e-12)
