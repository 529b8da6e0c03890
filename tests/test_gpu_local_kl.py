"""Local KL parametrization on the GPU (Sec. 2.1.1) against the FP64 oracle
(oracle/local_kl.py).  Eigenvalues of every patch within 1e-10 (those above
1e-8 of the largest, plus 1e-13 of the largest for the library's absolute
eigensolver accuracy); the local parameters are compared through quantities
that do not depend on the sign (or, in a degenerate eigenspace, the basis)
of the modes: the reconstruction sum_k sqrt(lambda_k) xi_k f_k on the patch
and sum_k xi_k^2, over the modes whose span is well determined (eigenvalues
above 1e-6 of the largest: both eigensolvers resolve the rest only to
their absolute accuracy).  With the bump covariance (rank at most the
number of bumps) all kept modes reconstruct the field on the patch up to
those ill-determined directions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1607_00693_gb300 import api
from paper_1607_00693_gb300 import workloads as W

DEV = "cuda:0"
NF, NC = 32, 4
FIELD = dict(kind=0, nbx=4, nby=4, width=0.1, scale=0.7, contrast_log=0.0, gain=1.0)


@pytest.fixture(scope="module")
def orc():
    import oracle
    from paper_1607_00693_gb300.build import build_library
    oracle.build()
    build_library()
    return oracle


def _patch_points(orc, lk, cell, o):
    x0, x1, y0, y1 = orc.patch_bounds(NF, NC, cell % NC, cell // NC, o)
    return lk.patch_centroids(NF, x0, x1, y0, y1), (x0, x1, y0, y1)


def _gpu_recon(lam, w, xi, n, h):
    # f_k = w_k sqrt(lambda_k) / h^2 ; sum_k sqrt(lambda_k) xi_k f_k = sum_k lambda_k xi_k w_k / h^2
    K = int(np.sum(lam > 0))
    return (lam[:K] * xi[:K]) @ w[:K, :n] / (h * h)


@pytest.mark.parametrize("o", [0, 1])
def test_local_kl_bumps(orc, o):
    from oracle import local_kl as lk
    g = api.grid(NF, NC, 1.0)
    fld = api.field_from_dict(FIELD)
    kmax = 16
    h, ks = api.stomsfem_local_kl_build(g, o, api.KL_BUMPS, fld, var=1.0 / 3.0, kmax=kmax)
    try:
        lam_g, w_g = api.stomsfem_local_kl_modes(h, g, kmax)
        S = 6
        xi_field = W.draw_xi(FIELD, S, 21)
        a = orc.sample_coef(NF, FIELD, xi_field)
        kappa = np.log(a)
        xi = torch.empty((S, NC * NC, kmax), dtype=torch.float64, device=DEV)
        api.stomsfem_local_kl_project(h, torch.from_numpy(kappa).to(DEV), xi)
        torch.cuda.synchronize()
        xi = xi.cpu().numpy()
    finally:
        api.stomsfem_local_kl_destroy(h)
    hh = 1.0 / NF
    for cell in range(NC * NC):
        pts, (x0, x1, y0, y1) = _patch_points(orc, lk, cell, o)
        C = lk.cov_bumps(FIELD, pts, "uniform")
        lam_o, F_o, lam_all = lk.local_kl(C, hh)
        big = lam_all[:kmax] > 1e-8 * lam_all[0]
        np.testing.assert_allclose(lam_g[cell, :kmax][big], lam_all[:kmax][big], rtol=1e-10,
                                   atol=1e-13 * lam_all[0])
        assert ks[cell] == min(kmax, len(lam_o))
        n = pts.shape[0]
        # modes well separated from the numerically zero part of the
        # spectrum (rank <= 16): their span is determined to ~1e-16 / 1e-6
        good = int(np.sum(lam_all[:ks[cell]] > 1e-6 * lam_all[0]))
        for s in range(S):
            kp = kappa[s, y0:y1, x0:x1].reshape(-1)
            xo = lk.local_params(kp, 0.0, lam_o, F_o, hh)
            rg = (lam_g[cell, :good] * xi[s, cell, :good]) @ w_g[cell, :good, :n] / (hh * hh)
            ro = lk.reconstruct(xo[:good], 0.0, lam_o[:good], F_o[:, :good])
            scale = np.abs(kp).max()
            np.testing.assert_allclose(rg, ro, rtol=0, atol=1e-9 * scale)
            assert np.sum(xi[s, cell, :good] ** 2) == pytest.approx(np.sum(xo[:good] ** 2), rel=1e-9)
            # every kept mode: the field on the patch, up to the modes whose
            # eigenvalues sit at the rounding level of the largest
            rall = _gpu_recon(lam_g[cell], w_g[cell], xi[s, cell], n, hh)
            np.testing.assert_allclose(rall, kp, rtol=0, atol=1e-5 * scale)
            assert np.all(xi[s, cell, ks[cell]:] == 0.0)


def test_local_kl_gaussian_energy_truncation(orc):
    """Gaussian covariance (beta = 0.1) on 10 x 10-element patches, modes for
    99 % of the spectrum: the same count as the oracle, eigenvalues, and the
    truncated reconstruction of a field sample (the eigenspaces cut at the
    count are whole when the count falls in a spectral gap, which is checked)."""
    from oracle import local_kl as lk
    g = api.grid(NF, NC, 1.0)
    o, kmax = 1, 32
    h, ks = api.stomsfem_local_kl_build(g, o, api.KL_GAUSSIAN, None, beta=0.1, sigma=1.0, kmax=kmax,
                                        energy=0.99)
    r = np.random.default_rng(5)
    hh = 1.0 / NF
    try:
        lam_g, w_g = api.stomsfem_local_kl_modes(h, g, kmax)
        kappa = r.standard_normal((2, NF, NF))
        xi = torch.empty((2, NC * NC, kmax), dtype=torch.float64, device=DEV)
        api.stomsfem_local_kl_project(h, torch.from_numpy(kappa).to(DEV), xi)
        torch.cuda.synchronize()
        xi = xi.cpu().numpy()
    finally:
        api.stomsfem_local_kl_destroy(h)
    checked = 0
    for cell in (0, 5, 10, 15):
        pts, (x0, x1, y0, y1) = _patch_points(orc, lk, cell, o)
        C = lk.cov_gaussian(pts, 0.1)
        lam_o, F_o, lam_all = lk.local_kl(C, hh, energy=0.99)
        K = len(lam_o)
        assert ks[cell] == K
        np.testing.assert_allclose(lam_g[cell, :K], lam_o, rtol=1e-9, atol=1e-13 * lam_o[0])
        if lam_all[K - 1] > (1 + 1e-6) * lam_all[K]:      # a gap: the kept space is unique
            n = pts.shape[0]
            for s in range(2):
                kp = kappa[s, y0:y1, x0:x1].reshape(-1)
                ro = lk.reconstruct(lk.local_params(kp, 0.0, lam_o, F_o, hh), 0.0, lam_o, F_o)
                rg = _gpu_recon(lam_g[cell], w_g[cell], xi[s, cell], n, hh)
                np.testing.assert_allclose(rg, ro, rtol=1e-8, atol=1e-8 * np.abs(ro).max())
            checked += 1
    assert checked >= 1
