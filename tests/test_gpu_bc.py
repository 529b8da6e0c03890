"""Coarse solves with mixed boundary data on the GPU (the anisotropy study of
Sec. 5.2, Eqs. xsquarewave / ysquarewave: prescribed values on node lines,
zero flux on the rest of the boundary) against the FP64 oracle, Galerkin
(blocked Cholesky) and Petrov-Galerkin (banded LU), with moments, several
warps' worth of samples, the widest grid (nc = 62), and the reduction to the
plain zero-Dirichlet solves.  Both sides are FP64 with different
elimination orders; the coarse systems' condition numbers reach about 4e5
(nc = 62, contrast 100), so the FP64 forward error bound is about 1e-10 of
the solution's scale: the tolerance is 1e-9 of it, as for the other coarse
solves."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1607_00693_gb300 import api
from paper_1607_00693_gb300 import workloads as W

DEV = "cuda:0"
KREF = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
KREF_PACKED = np.array([4, -1, -2, -1, 4, -1, -2, 4, -1, 4]) / 6.0
FIELD = dict(kind=0, nbx=4, nby=4, width=0.1, scale=1.0)


@pytest.fixture(scope="module")
def orc():
    from paper_1607_00693_gb300.build import build_library
    import oracle
    build_library()
    oracle.build()
    return oracle


def _t(x, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(x) if dtype is None else np.ascontiguousarray(x, dtype=dtype)).to(DEV)


def gpu_bc(nc, pg, K, b, dm, gv, moments=False):
    g = api.grid(nc, nc, 1.0)  # nf is not used by the coarse solve
    S = K.shape[0]
    nn = (nc + 1) ** 2
    u = torch.full((S, nn), 7.0, dtype=torch.float64, device=DEV)
    mean = m2 = cnt = None
    if moments:
        mean = torch.zeros(nn, dtype=torch.float64, device=DEV)
        m2 = torch.zeros(nn, dtype=torch.float64, device=DEV)
        cnt = torch.zeros(1, dtype=torch.float64, device=DEV)
    api.stomsfem_coarse_solve_bc(g, pg, _t(K), _t(b), _t(dm, np.uint8), _t(gv, np.float64), u, mean, m2, cnt)
    torch.cuda.synchronize()
    out = u.cpu().numpy()
    if moments:
        return out, mean.cpu().numpy(), m2.cpu().numpy(), cnt.cpu().numpy()
    return out


def close(ug, uo, tol=1e-9):
    scale = max(1.0, float(np.abs(uo).max()))
    assert np.isfinite(ug).all()
    assert float(np.abs(ug - uo).max()) <= tol * scale


@pytest.mark.parametrize("axis", ["x", "y"])
def test_msfem_grid_both_forms_with_moments(orc, axis):
    """nf = 64, nc = 8 with oversampling 0..2 per cell, 9 samples (more
    than one block of warps), the square-wave lines of the workload."""
    nf, nc, S = 64, 8, 9
    a = orc.sample_coef(nf, FIELD, W.draw_xi(FIELD, S, 31))
    ov = np.random.default_rng(2).integers(0, 3, nc * nc).astype(np.int8)
    dm, gv = W.mixed_bc(nc, axis=axis, lines=(0.25, 0.75), period=0.5)
    Ke, be = orc.upscale(nf, nc, 1.0, a, ov)
    Kp, bp = orc.upscale_pg(nf, nc, 1.0, a, ov)
    for pg, K, b in ((0, Ke, be), (1, Kp, bp)):
        uo = orc.coarse_solve_bc(nc, K, b, dm, gv, pg=bool(pg))
        ug, mean, m2, cnt = gpu_bc(nc, pg, K, b, dm, gv, moments=True)
        close(ug, uo)
        mo, vo = orc.mc_moments(uo)
        assert cnt[0] == S
        np.testing.assert_allclose(mean, mo, rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(m2 / S, vo, rtol=1e-8, atol=1e-14)
        # the prescribed values are reproduced exactly
        d = dm.astype(bool)
        np.testing.assert_array_equal(ug[:, d], np.tile(gv[d], (S, 1)))


@pytest.mark.parametrize("nc", [1, 2, 5, 33, 62])
def test_cell_sizes_up_to_the_band_limit(orc, nc):
    """H = h systems (K_e = a_e K_ref; for the Petrov-Galerkin form plus an
    antisymmetric zero-row-sum part, which keeps the symmetric part SPD and
    so the system as well conditioned as the Galerkin one) from one cell to
    nc = 62, the widest band (nc + 2 = 64), with a load and interior lines."""
    rng = np.random.default_rng(nc)
    S = 3
    a = np.exp(rng.uniform(np.log(0.1), np.log(10.0), (S, nc * nc)))
    Kg = a[..., None] * KREF_PACKED
    T = np.array([[0, 1, 0, -1], [-1, 0, 1, 0], [0, -1, 0, 1], [1, 0, -1, 0]], dtype=np.float64)
    d = rng.uniform(-0.1, 0.1, (S, nc * nc, 1))
    Kp = a[..., None] * (KREF.reshape(16) + d * T.reshape(16))
    b = np.full((S, nc * nc, 4), 0.25 / nc ** 2)
    dm, gv = W.mixed_bc(nc, axis="x", lines=(0.1, 0.9), period=0.5)
    for pg, K in ((0, Kg), (1, Kp)):
        uo = orc.coarse_solve_bc(nc, K, b, dm, gv, pg=bool(pg))
        close(gpu_bc(nc, pg, K, b, dm, gv), uo)


def test_zero_boundary_ring_is_the_plain_solves(orc):
    """Prescribed zeros on the boundary ring: the GPU results equal the
    plain zero-Dirichlet coarse solves (Galerkin and Petrov-Galerkin)."""
    nf, nc, S = 64, 8, 4
    a = orc.sample_coef(nf, FIELD, W.draw_xi(FIELD, S, 32))
    ov = np.full(nc * nc, 2, dtype=np.int8)
    ring = np.zeros((nc + 1, nc + 1), dtype=np.uint8)
    ring[0, :] = ring[-1, :] = ring[:, 0] = ring[:, -1] = 1
    dm, gv = ring.reshape(-1), np.zeros((nc + 1) ** 2)
    g = api.grid(nf, nc, 1.0)
    Ke, be = orc.upscale(nf, nc, 1.0, a, ov)
    Kp, bp = orc.upscale_pg(nf, nc, 1.0, a, ov)
    u0 = torch.empty((S, (nc + 1) ** 2), dtype=torch.float64, device=DEV)
    api.stomsfem_coarse_solve(g, _t(Ke), _t(be), u0)
    u1 = torch.empty_like(u0)
    api.stomsfem_coarse_solve_pg(g, _t(Kp), _t(bp), u1)
    torch.cuda.synchronize()
    close(gpu_bc(nc, 0, Ke, be, dm, gv), u0.cpu().numpy(), 1e-11)
    close(gpu_bc(nc, 1, Kp, bp, dm, gv), u1.cpu().numpy(), 1e-11)


def test_full_size_coarse_grid_sampled(orc):
    """The upscale_1024 coarse grid (nc = 32) with the benchmark's batch
    shape: 512 samples of synthetic H = h element matrices; every sample
    is solved, 8 of them (first, last, spread) checked against the oracle,
    all checked for finiteness and the prescribed values."""
    nc, S = 32, 512
    rng = np.random.default_rng(1024)
    a = np.exp(rng.uniform(np.log(0.1), np.log(10.0), (S, nc * nc)))
    K = a[..., None] * KREF_PACKED
    b = np.full((S, nc * nc, 4), 0.25 / nc ** 2)
    dm, gv = W.mixed_bc(nc, axis="y")
    ug = gpu_bc(nc, 0, K, b, dm, gv)
    d = dm.astype(bool)
    assert np.isfinite(ug).all()
    np.testing.assert_array_equal(ug[:, d], np.tile(gv[d], (S, 1)))
    pick = np.unique(np.r_[0, S - 1, np.linspace(1, S - 2, 6).astype(int)])
    uo = orc.coarse_solve_bc(nc, K[pick], b[pick], dm, gv)
    close(ug[pick], uo)


def test_empty_and_argument_checks():
    g = api.grid(64, 8, 1.0)
    nn = 81
    K = torch.zeros((0, 64, 10), dtype=torch.float64, device=DEV)
    b = torch.zeros((0, 64, 4), dtype=torch.float64, device=DEV)
    dm = torch.zeros(nn, dtype=torch.uint8, device=DEV)
    gv = torch.zeros(nn, dtype=torch.float64, device=DEV)
    u = torch.zeros((0, nn), dtype=torch.float64, device=DEV)
    api.stomsfem_coarse_solve_bc(g, 0, K, b, dm, gv, u)   # S = 0: nothing to do
    with pytest.raises(Exception):
        api.stomsfem_coarse_solve_bc(api.grid(63, 63, 1.0), 0, K, b, dm, gv, u)
