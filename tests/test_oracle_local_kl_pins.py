"""Pins of the local KL oracle (Sec. 2.1.1: Eqs. localCov, localKL,
local_KL_truncation), no GPU.  The bump covariance against the C sampler's
own field; the eigenpairs against the definition (orthonormality, eigen
relation, trace); exact reconstruction with every mode; whitened local
parameters on samples of the field; the KL tail identity for the truncation
error; the tensor structure of the separable Gaussian covariance; and the
locality the paper reports (fewer local than global modes)."""
import numpy as np
import pytest

from paper_1607_00693_gb300 import workloads as W

NF, NC = 32, 4
FIELD = dict(kind=0, nbx=4, nby=4, width=0.1, scale=0.7, contrast_log=0.0, gain=1.0)


@pytest.fixture(scope="module")
def setup():
    import oracle
    from oracle import local_kl
    oracle.build()
    return oracle, local_kl


def _patch(orc, cx, cy, o):
    x0, x1, y0, y1 = orc.patch_bounds(NF, NC, cx, cy, o)
    return x0, x1, y0, y1


def test_bump_values_reproduce_the_sampled_log_coefficient(setup):
    """log a from the C sampler equals s * sum_i xi_i psi_i at the element
    centroids, with the bump values of the local KL module."""
    orc, lk = setup
    xi = W.draw_xi(FIELD, 4, 11)
    a = orc.sample_coef(NF, FIELD, xi)
    pts = lk.patch_centroids(NF, 0, NF, 0, NF)
    P = lk.bump_values(FIELD, pts)
    np.testing.assert_allclose(np.log(a.reshape(4, -1)), FIELD["scale"] * xi @ P.T, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("o", [0, 2])
def test_eigenpairs_and_exact_reconstruction(setup, o):
    orc, lk = setup
    h = 1.0 / NF
    x0, x1, y0, y1 = _patch(orc, 1, 2, o)
    pts = lk.patch_centroids(NF, x0, x1, y0, y1)
    C = lk.cov_bumps(FIELD, pts)
    lam, F, lam_all = lk.local_kl(C, h)
    np.testing.assert_allclose(h * h * F.T @ F, np.eye(len(lam)), atol=1e-10)
    np.testing.assert_allclose(h * h * C @ F, F * lam, rtol=1e-9, atol=1e-12 * lam[0] / h)
    assert lam_all.sum() == pytest.approx(h * h * np.trace(C), rel=1e-12)
    assert len(lam) <= FIELD["nbx"] * FIELD["nby"]          # rank of sum_i psi_i psi_i^T
    # every sample of the field lies in the span of the modes, up to the
    # modes below the cutoff (bumps far from the patch, variance ~1e-17):
    # their share of a sample is at most sqrt(3 K sum of their eigenvalues
    # / h^2) per element for |xi_i| <= 1
    xi = W.draw_xi(FIELD, 3, 12)
    a = orc.sample_coef(NF, FIELD, xi)
    kap = np.log(a[:, y0:y1, x0:x1].reshape(3, -1))
    z = lk.local_params(kap, 0.0, lam, F, h)
    dropped = np.maximum(lam_all[len(lam):], 0.0).sum()
    bound = np.sqrt(3.0 * 16 * dropped) / h + 1e-12 * np.abs(kap).max()
    assert np.abs(lk.reconstruct(z, 0.0, lam, F) - kap).max() <= bound


def test_local_parameters_are_whitened_and_tail_is_the_truncation_error(setup):
    """On samples of the field the local parameters have mean 0 and identity
    covariance (within sampling error), and the mean squared L2 error of the
    K-term truncation is the sum of the dropped eigenvalues."""
    orc, lk = setup
    h = 1.0 / NF
    x0, x1, y0, y1 = _patch(orc, 2, 1, 1)
    pts = lk.patch_centroids(NF, x0, x1, y0, y1)
    lam, F, lam_all = lk.local_kl(lk.cov_bumps(FIELD, pts), h)
    N = 20000
    xi = W.draw_xi(FIELD, N, 13)
    kap = FIELD["scale"] * xi @ lk.bump_values(FIELD, pts).T      # the field at the centroids
    z = lk.local_params(kap, 0.0, lam, F, h)
    tol = 6.0 / np.sqrt(N)
    assert np.abs(z.mean(axis=0)).max() < tol
    np.testing.assert_allclose(np.cov(z.T, bias=True), np.eye(len(lam)), atol=tol * 1.5)
    K = 3
    lamK, FK, _ = lk.local_kl(lk.cov_bumps(FIELD, pts), h, K=K)
    err = h * h * ((kap - lk.reconstruct(lk.local_params(kap, 0.0, lamK, FK, h), 0.0, lamK, FK)) ** 2).sum(axis=1)
    assert err.mean() == pytest.approx(lam_all[K:].sum(), rel=0.05)


def test_gaussian_covariance_is_a_tensor_product(setup):
    """exp(-|x-y|^2/beta^2) factorises in x and y and the patch's centroids
    form a tensor grid, so the 2D eigenvalues are the products of the 1D
    ones (1D operator h C_1)."""
    orc, lk = setup
    h = 1.0 / NF
    pts = lk.patch_centroids(NF, 8, 16, 4, 12)                    # 8 x 8 elements
    lam2 = np.sort(lk.local_kl(lk.cov_gaussian(pts, 0.15), h, K=64)[0])[::-1]
    x = (np.arange(8) + 0.5) * h
    C1 = np.exp(-((x[:, None] - x[None, :]) ** 2) / 0.15 ** 2)
    l1 = np.linalg.eigvalsh(h * C1)
    ref = np.sort(np.outer(l1, l1).reshape(-1))[::-1]
    np.testing.assert_allclose(lam2, ref, rtol=1e-9, atol=1e-14 * ref[0])


def test_local_expansion_needs_fewer_modes_than_global(setup):
    """The paper's observation (Sec. 5.3): for a short correlation length
    the local KL keeps 99 % of the spectrum with far fewer modes than the
    global one."""
    orc, lk = setup
    h = 1.0 / NF
    beta = 0.1
    _, _, lam_g = lk.local_kl(lk.cov_gaussian(lk.patch_centroids(NF, 0, NF, 0, NF), beta), h)
    Kg = lk.local_kl(lk.cov_gaussian(lk.patch_centroids(NF, 0, NF, 0, NF), beta), h, energy=0.99)[0].size
    x0, x1, y0, y1 = _patch(orc, 1, 1, 2)
    Kl = lk.local_kl(lk.cov_gaussian(lk.patch_centroids(NF, x0, x1, y0, y1), beta), h, energy=0.99)[0].size
    assert Kl * 4 < Kg
    assert np.cumsum(lam_g)[Kg - 1] >= 0.99 * lam_g.sum() > np.cumsum(lam_g)[Kg - 2]
