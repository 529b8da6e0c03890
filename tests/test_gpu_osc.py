"""Oscillatory boundary data of the cell problems on the GPU (the MsFEM option
of the short-correlation example, Sec. 5.3: harmonic coordinate along each
patch edge) against the FP64 oracle: Galerkin and Petrov-Galerkin, every
precision, per-cell oversampling with clipped patches, the basis output,
a constant coefficient, and the bilinear choice of the same call.

Tolerances as in test_gpu_parity / test_gpu_pg: relative Frobenius per unit
1e-11 (FP64), 1e-10 (FP32 factor + FP64 refinement), 1e-5 (FP32)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1607_00693_gb300 import api
from paper_1607_00693_gb300 import workloads as W

TOL = {api.FP64: 1e-11, api.FP32_REFINED: 1e-10, api.FP32: 1e-5}
DEV = "cuda:0"
FIELD = dict(kind=0, nbx=4, nby=4, width=0.1, scale=1.0)


@pytest.fixture(scope="module")
def orc():
    from paper_1607_00693_gb300.build import build_library
    import oracle
    build_library()
    oracle.build()
    return oracle


def rel_unit(Kg, Ko):
    num = np.linalg.norm((Kg - Ko).reshape(-1, Ko.shape[-1]), axis=1)
    den = np.linalg.norm(Ko.reshape(-1, Ko.shape[-1]), axis=1)
    return float(np.max(num / den))


def gpu(nf, nc, a_np, pg, bc, ov=None, precision=api.FP64, want_phi=False):
    g = api.grid(nf, nc, 1.0)
    a = torch.from_numpy(a_np).to(DEV)
    S = a.shape[0]
    KN = 16 if pg else 10
    Ke = torch.full((S, nc * nc, KN), 7.0, dtype=torch.float64, device=DEV)
    be = torch.full((S, nc * nc, 4), 7.0, dtype=torch.float64, device=DEV)
    st = torch.full((S, nc * nc), 99, dtype=torch.int32, device=DEV)
    phi = (torch.empty((S, nc * nc, 4, (nf // nc + 1) ** 2), dtype=torch.float64, device=DEV)
           if want_phi else None)
    o_t, mo = None, 0
    if ov is not None:
        o_t = torch.from_numpy(np.ascontiguousarray(ov, dtype=np.int8)).to(DEV)
        mo = int(np.max(ov))
    api.stomsfem_upscale_bc(g, pg, bc, a, Ke, be, oversample=o_t, max_oversample=mo, precision=precision,
                            phi=phi, unit_status=st)
    torch.cuda.synchronize()
    out = [Ke.cpu().numpy(), be.cpu().numpy(), st.cpu().numpy()]
    if want_phi:
        out.append(phi.cpu().numpy())
    return out


@pytest.mark.parametrize("pg", [False, True])
@pytest.mark.parametrize("precision", [api.FP64, api.FP32_REFINED, api.FP32])
def test_oversampled_rho32(orc, pg, precision):
    """H/h = 32, oversampling 0..4 per cell (clipped at the domain boundary),
    an odd sample count (the idle half of the last warp mirrors)."""
    nf, nc = 128, 4
    fld = dict(W.workload("upscale_1024")["field"], nbx=4, nby=4, width=0.125)
    a = orc.sample_coef(nf, fld, W.draw_xi(fld, 3, 71))
    ov = np.random.default_rng(21).integers(0, 5, size=nc * nc).astype(np.int8)
    assert (ov == 0).any() and (ov > 0).any()
    if pg:
        Ko, bo = orc.upscale_pg(nf, nc, 1.0, a, ov, bc=orc.BC_OSCILLATORY)
        Ko = Ko.reshape(3, nc * nc, 16)
    else:
        Ko, bo = orc.upscale(nf, nc, 1.0, a, ov, bc=orc.BC_OSCILLATORY)
    Kg, bg, st = gpu(nf, nc, a, pg, api.BC_OSCILLATORY, ov, precision)
    assert (st == 0).all()
    assert rel_unit(Kg, Ko) <= TOL[precision]
    if pg:
        np.testing.assert_array_equal(bg, bo)
    else:
        assert rel_unit(bg, bo) <= TOL[precision]
    # the option changes the result: the bilinear data give other matrices
    Kb, _, _ = gpu(nf, nc, a, pg, api.BC_BILINEAR, ov, precision)
    assert rel_unit(Kb, Ko) > 100 * TOL[precision]


@pytest.mark.parametrize("pg", [False, True])
def test_rough_medium_without_oversampling_and_basis(orc, pg):
    """The msfem_64 grid (H/h = 8) with a rough lognormal medium, no
    oversampling (every edge of every patch carries oscillatory data), the
    basis output in FP64."""
    nf, nc, S = 64, 8, 5
    rng = np.random.default_rng(64)
    a = np.exp(rng.uniform(np.log(0.1), np.log(10.0), (S, nf, nf)))
    if pg:
        Ko, bo = orc.upscale_pg(nf, nc, 1.0, a, bc=orc.BC_OSCILLATORY)
        Kg, bg, st = gpu(nf, nc, a, True, api.BC_OSCILLATORY)
        np.testing.assert_array_equal(bg, bo)
        # without oversampling the Petrov-Galerkin matrix no longer equals
        # the Galerkin one: the oscillatory phi differs from q on the edges
        Kgal, _ = orc.upscale(nf, nc, 1.0, a, bc=orc.BC_OSCILLATORY)
        assert np.abs(Ko.reshape(S, -1, 16)[..., 1] - Kgal[..., 1]).max() > 1e-4
    else:
        Ko, bo, phio = orc.upscale(nf, nc, 1.0, a, want_phi=True, bc=orc.BC_OSCILLATORY)
        Kg, bg, st, phig = gpu(nf, nc, a, False, api.BC_OSCILLATORY, want_phi=True)
        assert float(np.abs(phig - phio).max()) <= 1e-11
        assert rel_unit(bg, bo) <= 1e-11
    assert (st == 0).all()
    assert rel_unit(Kg, Ko.reshape(Kg.shape)) <= 1e-11
    for precision in (api.FP32, api.FP32_REFINED):
        Kp, _, st = gpu(nf, nc, a, pg, api.BC_OSCILLATORY, precision=precision)
        assert (st == 0).all()
        assert rel_unit(Kp, Ko.reshape(Kp.shape)) <= TOL[precision]


def test_constant_coefficient_and_bilinear_choice(orc):
    """a = c gives c K_ref with either data; bc = BC_BILINEAR through the
    same call is bitwise the plain upscaling call."""
    nf, nc, c = 64, 8, 3.25
    a = np.full((2, nf, nf), c)
    ov = np.random.default_rng(4).integers(0, 3, size=nc * nc).astype(np.int8)
    kref = np.array([4, -1, -2, -1, 4, -1, -2, 4, -1, 4]) / 6.0
    for precision in (api.FP64, api.FP32):
        Kg, _, st = gpu(nf, nc, a, False, api.BC_OSCILLATORY, ov, precision)
        assert (st == 0).all()
        np.testing.assert_allclose(Kg, np.broadcast_to(c * kref, Kg.shape), rtol=TOL[precision],
                                   atol=TOL[precision] * c)
    a = orc.sample_coef(nf, FIELD, W.draw_xi(FIELD, 3, 77))
    g = api.grid(nf, nc, 1.0)
    at = torch.from_numpy(a).to(DEV)
    K0 = torch.empty((3, nc * nc, 10), dtype=torch.float64, device=DEV)
    b0 = torch.empty((3, nc * nc, 4), dtype=torch.float64, device=DEV)
    api.stomsfem_upscale(g, at, K0, b0, precision=api.FP64)
    K1, b1, _ = gpu(nf, nc, a, False, api.BC_BILINEAR)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(K1, K0.cpu().numpy())
    np.testing.assert_array_equal(b1, b0.cpu().numpy())


def test_argument_checks():
    g = api.grid(64, 8, 1.0)
    a = torch.ones((1, 64, 64), dtype=torch.float64, device=DEV)
    Ke = torch.empty((1, 64, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((1, 64, 4), dtype=torch.float64, device=DEV)
    with pytest.raises(Exception):
        api.stomsfem_upscale_bc(g, False, 2, a, Ke, be)
