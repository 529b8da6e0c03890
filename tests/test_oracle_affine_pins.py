"""Pins of the affine field (Eq. RBaffine) and of the affine split of the
reduced quantities (Eq. localAF) in the oracle, no GPU."""
import numpy as np
import pytest

from paper_1607_00693_gb300 import workloads as W


@pytest.fixture(scope="module")
def orc():
    import oracle
    from oracle import pod, surrogate
    oracle.build()
    return oracle, pod, surrogate


def test_affine_field_is_the_exponent_of_the_exponential_field(orc):
    """a_affine - gain = scale z = log(a_exp) for the same xi (the two kinds
    share z), and a_affine - gain is linear in xi."""
    oracle, _, _ = orc
    nf = 32
    fa = dict(kind=2, nbx=4, nby=4, width=0.1, scale=0.7, gain=2.0)
    fe = dict(kind=0, nbx=4, nby=4, width=0.1, scale=0.7)
    x1, x2 = W.draw_xi(fa, 2, 3), W.draw_xi(fa, 2, 4)
    a1 = oracle.sample_coef(nf, fa, x1)
    np.testing.assert_allclose(a1 - 2.0, np.log(oracle.sample_coef(nf, fe, x1)), atol=1e-14)
    a2 = oracle.sample_coef(nf, fa, x2)
    a12 = oracle.sample_coef(nf, fa, x1 + x2)
    np.testing.assert_allclose(a12 - 2.0, (a1 - 2.0) + (a2 - 2.0), atol=1e-14)
    w = oracle.sample_coef_window(nf, fa, x1[0], 4, 12, 8, 16)
    np.testing.assert_array_equal(w[8:16, 4:12], a1[0, 8:16, 4:12])


@pytest.fixture(scope="module")
def trained(orc):
    oracle, pod, surrogate = orc
    w = W.workload("pod_affine_64")
    nf, nc = 32, 4
    fld = w["field"]
    xi = W.draw_xi(fld, 30, 6)
    a = oracle.sample_coef(nf, fld, xi)
    _, _, phi = oracle.upscale(nf, nc, 1.0, a, want_phi=True)
    models = pod.build(nf, nc, phi, a, tol=1e-6, max_rank=12)
    k, ids, _, _ = surrogate.local_vars(nf, nc, fld, w["tau"])
    return nf, nc, fld, models, k, ids


def test_reduced_quantities_split_by_the_affine_parts(orc, trained):
    """Eq. localAF: W^T A(xi) W = gain G_0 + scale sum_k xi_k G_k with
    G_0 = W^T A(1) W and G_k = W^T A(psi_k) W, psi_k read off the field as
    the coefficient of a one-hot xi with gain 0 and scale 1."""
    oracle, pod, _ = orc
    nf, nc, fld, models, k, ids = trained
    rho = nf // nc
    unit = dict(fld, gain=0.0, scale=1.0)
    xi = W.draw_xi(fld, 1, 17)[0]
    for cell in (0, 5, 10):
        m = models[cell]
        cx, cy = cell % nc, cell // nc
        G = pod.reduced_matrix(m, pod.affine_cell_coef(nf, nc, fld, xi, cell, ids[cell]))
        acc = fld["gain"] * pod.reduced_matrix(m, np.ones((rho, rho)))
        for j in range(k[cell]):
            e = np.zeros(W.n_vars(fld))
            e[ids[cell, j]] = 1.0
            psi = oracle.sample_coef(nf, unit, e[None])[0, cy * rho:(cy + 1) * rho, cx * rho:(cx + 1) * rho]
            acc += fld["scale"] * xi[ids[cell, j]] * pod.reduced_matrix(m, psi)
        np.testing.assert_allclose(G, acc, rtol=1e-12, atol=1e-12 * np.abs(G).max())


def test_local_truncation_bound(orc, trained):
    """Dropping the non-local bumps changes a by at most |scale| sum |xi_i|
    tau on the cell (each dropped bump is below tau there)."""
    oracle, pod, _ = orc
    nf, nc, fld, models, k, ids = trained
    rho = nf // nc
    tau = W.workload("pod_affine_64")["tau"]
    xi = W.draw_xi(fld, 3, 8)
    a = oracle.sample_coef(nf, fld, xi)
    for s in range(3):
        for cell in range(nc * nc):
            cx, cy = cell % nc, cell // nc
            at = pod.affine_cell_coef(nf, nc, fld, xi[s], cell, ids[cell])
            full = a[s, cy * rho:(cy + 1) * rho, cx * rho:(cx + 1) * rho]
            dropped = [i for i in range(W.n_vars(fld)) if i not in set(ids[cell, :k[cell]])]
            bound = abs(fld["scale"]) * tau * np.abs(xi[s, dropped]).sum()
            assert np.abs(full - at).max() <= bound + 1e-15
