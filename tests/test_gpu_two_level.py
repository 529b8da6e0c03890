"""Two-level Monte Carlo pieces on the GPU (Remark in Sec. 4.1.1, Eq.
MCmean2level) against the FP64 oracle: the fine-grid Q1 FEM solver
(nf = 64 down to the one-unknown grid), the restriction to the coarse
nodes, the moments, and the composed estimator on the 64^2 / 8^2 grid."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1607_00693_gb300 import api
from paper_1607_00693_gb300 import workloads as W

DEV = "cuda:0"


@pytest.fixture(scope="module")
def orc():
    from paper_1607_00693_gb300.build import build_library
    import oracle
    build_library()
    oracle.build()
    return oracle


def _fine(g, a_np):
    a = torch.from_numpy(a_np).to(DEV)
    u = torch.empty((a.shape[0], (g.nf + 1) ** 2), dtype=torch.float64, device=DEV)
    api.stomsfem_fine_fem(g, a, u)
    torch.cuda.synchronize()
    return u.cpu().numpy()


@pytest.mark.parametrize("nf", [2, 3, 17, 64])
def test_fine_fem_matches_oracle(orc, nf):
    r = np.random.default_rng(nf)
    a = np.exp(r.uniform(-2, 2, size=(3, nf, nf)))
    g = api.grid(nf, 1, 1.7)
    u = _fine(g, a)
    uo = np.stack([orc.fine_fem(nf, 1.7, a[s]) for s in range(3)])
    assert (np.linalg.norm(u - uo, axis=1) / np.linalg.norm(uo, axis=1)).max() <= 1e-10


def test_two_level_estimator_matches_oracle(orc):
    """N_0 = 24 coarse samples and N_1 = 8 independent samples on both
    levels: the estimate and its sampling variance through the C ABI."""
    w = W.workload("msfem_64")
    nf, nc, fld = w["nf"], w["nc"], w["field"]
    g = api.grid(nf, nc, w["f"])
    nn = (nc + 1) ** 2
    x0 = W.draw_xi(fld, 24, 101)
    x1 = W.draw_xi(fld, 8, 102)
    a0, a1 = orc.sample_coef(nf, fld, x0), orc.sample_coef(nf, fld, x1)

    def coarse(a_np, mom):
        a = torch.from_numpy(a_np).to(DEV)
        S = a.shape[0]
        Ke = torch.empty((S, nc * nc, 10), dtype=torch.float64, device=DEV)
        be = torch.empty((S, nc * nc, 4), dtype=torch.float64, device=DEV)
        u = torch.empty((S, nn), dtype=torch.float64, device=DEV)
        api.stomsfem_upscale(g, a, Ke, be)
        api.stomsfem_coarse_solve(g, Ke, be, u, *mom)
        return u

    m0 = [torch.zeros(nn, dtype=torch.float64, device=DEV) for _ in range(2)] + \
         [torch.zeros(1, dtype=torch.float64, device=DEV)]
    m1 = [torch.zeros(nn, dtype=torch.float64, device=DEV) for _ in range(2)] + \
         [torch.zeros(1, dtype=torch.float64, device=DEV)]
    coarse(a0, m0)
    uH1 = coarse(a1, (None, None, None))
    uh1 = torch.empty((8, (nf + 1) ** 2), dtype=torch.float64, device=DEV)
    api.stomsfem_fine_fem(g, torch.from_numpy(a1).to(DEV), uh1)
    d = torch.empty((8, nn), dtype=torch.float64, device=DEV)
    api.stomsfem_restrict_to_coarse(g, uh1, d, u_coarse=uH1)
    api.stomsfem_mc_moments(d, *m1)
    torch.cuda.synchronize()
    est = (m0[0] + m1[0]).cpu().numpy()
    var = (m0[1] / m0[2] / m0[2] + m1[1] / m1[2] / m1[2]).cpu().numpy()

    uH0o = orc.coarse_solve(nc, *orc.upscale(nf, nc, w["f"], a0))
    uH1o = orc.coarse_solve(nc, *orc.upscale(nf, nc, w["f"], a1))
    uh1o = orc.restrict_to_coarse(np.stack([orc.fine_fem(nf, w["f"], a1[s]) for s in range(8)]), nf, nc)
    esto, varo = orc.two_level_mean(uH0o, uh1o, uH1o)
    np.testing.assert_allclose(est, esto, rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(var, varo, rtol=1e-7, atol=1e-20)
