"""Petrov-Galerkin form on the GPU (Eq. stiffness_local_petrov) against the
FP64 oracle: the 16-entry local matrices with per-cell oversampling (both
FP32 launches, FP32 + refinement, FP64), the non-symmetric coarse solve with
moments, the widest coarse band, and end to end.

Tolerances as in test_gpu_parity: relative Frobenius per unit 1e-11 (FP64),
1e-10 (FP32 factor + FP64 refinement), 1e-5 (FP32); coarse solution 1e-9."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1607_00693_gb300 import api
from paper_1607_00693_gb300 import workloads as W

TOL = {api.FP64: 1e-11, api.FP32_REFINED: 1e-10, api.FP32: 1e-5}
DEV = "cuda:0"


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


def gpu_pg(nf, nc, a_np, ov=None, precision=api.FP64, want_phi=False):
    g = api.grid(nf, nc, 1.0)
    a = torch.from_numpy(a_np).to(DEV)
    S = a.shape[0]
    Ke = torch.full((S, nc * nc, 16), 7.0, dtype=torch.float64, device=DEV)
    be = torch.full((S, nc * nc, 4), 7.0, dtype=torch.float64, device=DEV)
    st = torch.full((S, nc * nc), 99, dtype=torch.int32, device=DEV)
    phi = (torch.empty((S, nc * nc, 4, (nf // nc + 1) ** 2), dtype=torch.float64, device=DEV)
           if want_phi else None)
    o_t, mo = None, 0
    if ov is not None:
        o_t = torch.from_numpy(np.ascontiguousarray(ov, dtype=np.int8)).to(DEV)
        mo = int(np.max(ov))
    api.stomsfem_upscale_pg(g, a, Ke, be, oversample=o_t, max_oversample=mo, precision=precision,
                            phi=phi, unit_status=st)
    torch.cuda.synchronize()
    out = [Ke.cpu().numpy(), be.cpu().numpy(), st.cpu().numpy()]
    if want_phi:
        out.append(phi.cpu().numpy())
    return out


@pytest.mark.parametrize("precision", [api.FP64, api.FP32_REFINED, api.FP32])
def test_pg_oversampled_rho32(orc, precision):
    """H/h = 32, oversampling 0..4 per cell (clipped at the domain boundary),
    an odd sample count (the idle half of the last warp mirrors)."""
    nf, nc = 128, 4
    fld = dict(W.workload("upscale_1024")["field"], nbx=4, nby=4, width=0.125)
    a = orc.sample_coef(nf, fld, W.draw_xi(fld, 3, 7))
    ov = np.random.default_rng(20).integers(0, 5, size=nc * nc).astype(np.int8)
    assert (ov == 0).any() and (ov > 0).any()
    Ko, bo = orc.upscale_pg(nf, nc, 1.0, a, ov)
    Kg, bg, st = gpu_pg(nf, nc, a, ov, precision)
    assert (st == 0).all()
    assert rel_unit(Kg, Ko) <= TOL[precision]
    np.testing.assert_array_equal(bg, bo)
    # the oversampled cells are not symmetric
    K4 = Kg.reshape(-1, 16, 4, 4)[:, ov > 0]
    assert np.abs(K4 - np.swapaxes(K4, -1, -2)).max() > 1e-6 * np.abs(K4).max()


def test_pg_without_oversampling_is_galerkin(orc):
    """No oversampling: the Petrov-Galerkin matrices are the Galerkin ones
    (FP32 forward-only route and FP64), the load f H^2 / 4."""
    w = W.workload("msfem_64")
    a = orc.sample_coef(w["nf"], w["field"], W.draw_xi(w["field"], 6, 3))
    Kgal, _ = orc.upscale(w["nf"], w["nc"], 1.0, a)
    full = np.stack([orc.unpack_upper(k).reshape(16) for k in Kgal.reshape(-1, 10)]).reshape(6, 64, 16)
    for prec in (api.FP64, api.FP32):
        Kg, bg, _ = gpu_pg(w["nf"], w["nc"], a, None, prec)
        assert rel_unit(Kg, full) <= TOL[prec]
        np.testing.assert_allclose(bg, 1.0 / 64 / 4, rtol=1e-15)


def test_pg_phi_output(orc):
    """The basis written next to the Petrov-Galerkin matrices is the trial
    basis of the Galerkin form (same cell problems)."""
    nf, nc = 24, 4
    a = np.exp(np.random.default_rng(2).uniform(-1.5, 1.5, size=(2, nf, nf)))
    ov = np.full(nc * nc, 1, dtype=np.int8)
    _, _, po = orc.upscale(nf, nc, 1.0, a, ov, want_phi=True)
    Ko, bo = orc.upscale_pg(nf, nc, 1.0, a, ov)
    Kg, bg, _, pg = gpu_pg(nf, nc, a, ov, want_phi=True)
    assert rel_unit(Kg, Ko) <= 1e-11
    assert np.max(np.abs(pg - po)) <= 1e-11


def _coarse_pg(g, K, b, mom=None):
    S = K.shape[0]
    nn = (g.nc + 1) ** 2
    u = torch.empty((S, nn), dtype=torch.float64, device=DEV)
    args = mom if mom is not None else (None, None, None)
    api.stomsfem_coarse_solve_pg(g, torch.from_numpy(K).to(DEV), torch.from_numpy(b).to(DEV), u, *args)
    torch.cuda.synchronize()
    return u.cpu().numpy()


def test_pg_coarse_solve_and_moments(orc):
    """Non-symmetric coarse systems of 24 samples in two uneven batches
    through the running moment accumulators."""
    w = W.workload("msfem_64")
    a = orc.sample_coef(w["nf"], w["field"], W.draw_xi(w["field"], 24, 5))
    ov = np.full(64, 2, dtype=np.int8)
    Ko, bo = orc.upscale_pg(w["nf"], w["nc"], 1.0, a, ov)
    uo = orc.coarse_solve_pg(w["nc"], Ko, bo)
    g = api.grid(w["nf"], w["nc"], 1.0)
    nn = 81
    mean = torch.zeros(nn, dtype=torch.float64, device=DEV)
    m2 = torch.zeros(nn, dtype=torch.float64, device=DEV)
    cnt = torch.zeros(1, dtype=torch.float64, device=DEV)
    u1 = _coarse_pg(g, Ko[:17].copy(), bo[:17].copy(), (mean, m2, cnt))
    u2 = _coarse_pg(g, Ko[17:].copy(), bo[17:].copy(), (mean, m2, cnt))
    ug = np.concatenate([u1, u2])
    assert (np.linalg.norm(ug - uo, axis=1) / np.linalg.norm(uo, axis=1)).max() <= 1e-9
    mo, vo = orc.mc_moments(uo)
    np.testing.assert_allclose(mean.cpu().numpy(), mo, rtol=1e-11, atol=1e-18)
    inner = vo > 0
    np.testing.assert_allclose((m2.cpu().numpy() / 24)[inner], vo[inner], rtol=1e-8)


@pytest.mark.parametrize("nc", [2, 3, 64])
def test_pg_coarse_band_extremes(orc, nc):
    """nc = 64 (half bandwidth 64: two window rows per lane) down to the
    one- and four-unknown systems; H/h = 4 with two oversampling layers
    keeps the local matrices non-symmetric."""
    r = np.random.default_rng(nc)
    nf = 4 * nc
    a = np.exp(r.uniform(-1, 1, size=(2, nf, nf)))
    ov = np.full(nc * nc, 2, dtype=np.int8)
    Ko, bo = orc.upscale_pg(nf, nc, 1.0, a, ov)
    K4 = Ko.reshape(2, -1, 4, 4)
    assert np.abs(K4 - np.swapaxes(K4, -1, -2)).max() > 1e-2 * np.abs(K4).max()
    uo = orc.coarse_solve_pg(nc, Ko, bo)
    ug = _coarse_pg(api.grid(nf, nc, 1.0), Ko, bo)
    assert (np.linalg.norm(ug - uo, axis=1) / np.linalg.norm(uo, axis=1)).max() <= 1e-9


def test_pg_end_to_end_fp32_against_fp64(orc):
    """rho = 32 with oversampling 0..4: the FP32 form's coarse solution stays
    within 1e-6 of the FP64 form's, which matches the oracle's."""
    nf, nc = 256, 8
    w = W.workload("upscale_1024")
    fld = dict(w["field"], nbx=8, nby=8)
    xi = W.draw_xi(fld, 4, 31)
    ov = np.random.default_rng(33).integers(0, 5, size=nc * nc).astype(np.int8)
    g = api.grid(nf, nc, 1.0)
    a = torch.empty((4, nf, nf), dtype=torch.float64, device=DEV)
    api.stomsfem_sample_coef(g, api.field_from_dict(fld), torch.from_numpy(xi).to(DEV), a)
    torch.cuda.synchronize()
    an = a.cpu().numpy()
    out = {}
    for prec in (api.FP64, api.FP32):
        Kg, bg, st = gpu_pg(nf, nc, an, ov, prec)
        assert (st == 0).all()
        out[prec] = _coarse_pg(g, Kg, bg)
    Ko, bo = orc.upscale_pg(nf, nc, 1.0, an, ov)
    uo = orc.coarse_solve_pg(nc, Ko, bo)
    rel = lambda x, y: (np.linalg.norm(x - y, axis=1) / np.linalg.norm(y, axis=1)).max()
    assert rel(out[api.FP64], uo) <= 1e-9
    assert rel(out[api.FP32], out[api.FP64]) <= 1e-6
