"""The FP32 forms' factorisation engines through stomsfem_upscale_engine
against the oracle, at patch sizes that reach every compiled panel height
of the one-unit-per-warp FMA engine (WIDE: column blocks of 16, one, two
and three panel rows per lane) and of the two-units-per-warp engine, in
both unit orders; K_e and b_e per unit within the form's tolerance (FP32
1e-5 up to H/h = 32 and 1e-5 (rho/32)^2 above, the FP32 factor's error
growing with the condition number of the cell matrix, which grows like
rho^2; FP32 + two FP64 refinement sweeps 1e-10; relative Frobenius)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1607_00693_gb300 import api

DEV = "cuda:0"
TOL = {api.FP32: 1e-5, api.FP32_REFINED: 1e-10}

# (nf, nc, oversampling range): half bandwidths 16 (H/h = 8, o <= 4), 41
# (H/h = 32, o <= 4) and 64 (H/h = 64, o = 0)
CASES = [(64, 8, 5), (128, 4, 5), (128, 2, 1)]


@pytest.fixture(scope="module")
def lib():
    from paper_1607_00693_gb300.build import build_library
    build_library()


def _rel(x, y):
    return float(np.max(np.linalg.norm(x - y, axis=-1) / np.linalg.norm(y, axis=-1)))


@pytest.mark.parametrize("nf,nc,orange", CASES)
@pytest.mark.parametrize("precision", [api.FP32, api.FP32_REFINED])
@pytest.mark.parametrize("engine,order", [(api.ENGINE_WIDE, api.ORDER_CELL), (api.ENGINE_WIDE, api.ORDER_PATCH),
                                          (api.ENGINE_BLOCKED, api.ORDER_PATCH)])
def test_engine_matches_oracle(lib, orc, nf, nc, orange, precision, engine, order):
    r = np.random.default_rng(nf * 7 + nc)
    S = 3
    a = np.exp(r.uniform(-1.5, 1.5, size=(S, nf, nf)))
    ov = r.integers(0, orange, size=nc * nc).astype(np.int8)
    Ko, bo = orc.upscale(nf, nc, 1.0, a, ov)
    g = api.grid(nf, nc, 1.0)
    at = torch.from_numpy(a).to(DEV)
    Ke = torch.empty((S, nc * nc, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((S, nc * nc, 4), dtype=torch.float64, device=DEV)
    st = torch.full((S, nc * nc), 7, dtype=torch.int32, device=DEV)
    api.stomsfem_upscale(g, at, Ke, be, oversample=torch.from_numpy(ov).to(DEV), max_oversample=int(ov.max()),
                         precision=precision, refine_iters=2, unit_status=st, engine=engine, order=order)
    torch.cuda.synchronize()
    assert np.all(st.cpu().numpy() == 0)
    tol = TOL[precision] * (max(1.0, (nf / nc / 32) ** 2) if precision == api.FP32 else 1.0)
    assert _rel(Ke.cpu().numpy(), Ko) <= tol
    assert _rel(be.cpu().numpy(), bo) <= tol


def test_wide_engine_refused_in_fp64(lib):
    g = api.grid(64, 8, 1.0)
    a = torch.ones((1, 64, 64), dtype=torch.float64, device=DEV)
    Ke = torch.empty((1, 64, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((1, 64, 4), dtype=torch.float64, device=DEV)
    with pytest.raises(Exception):
        api.stomsfem_upscale(g, a, Ke, be, precision=api.FP64, engine=api.ENGINE_WIDE)
    with pytest.raises(Exception):
        api.stomsfem_upscale(g, a, Ke, be, precision=api.FP32, engine=5)
    with pytest.raises(Exception):
        api.stomsfem_upscale(g, a, Ke, be, precision=api.FP32, order=2)
