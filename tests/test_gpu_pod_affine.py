"""Affine reduced basis on the GPU (Sec. 3.2.2, Eqs. RBaffine and localAF)
against the FP64 oracle: the reduced quantities assembled from xi and the
per-cell affine parts, solved in FP32 (and refined in FP64); the sampler's
affine field; argument errors.

Tolerances: the FP32 reduced quantities and Cholesky give K_e within 1e-4
(relative per unit) of the oracle's reduced-basis K_e on the local affine
coefficient; after FP64 refinement 1e-10."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1607_00693_gb300 import api, _lib
from paper_1607_00693_gb300 import workloads as W

DEV = "cuda:0"


@pytest.fixture(scope="module")
def setup():
    import oracle
    from oracle import pod, surrogate
    from paper_1607_00693_gb300.build import build_library
    oracle.build()
    build_library()
    w = W.workload("pod_affine_64")
    nf, nc, fld = w["nf"], w["nc"], w["field"]
    Ns = 40
    xi = W.draw_xi(fld, Ns, w["train_seed"])
    a_tr = oracle.sample_coef(nf, fld, xi)
    _, _, phi_o = oracle.upscale(nf, nc, w["f"], a_tr, want_phi=True)
    models = pod.build(nf, nc, phi_o, a_tr, tol=1e-6, max_rank=27)
    ranks = [m["rank"] for m in models]
    _, ids, _, _ = surrogate.local_vars(nf, nc, fld, w["tau"])
    g = api.grid(nf, nc, w["f"])
    F = api.field_from_dict(fld)
    a_t = torch.from_numpy(a_tr).to(DEV)
    rho = nf // nc
    Ke = torch.empty((Ns, nc * nc, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((Ns, nc * nc, 4), dtype=torch.float64, device=DEV)
    phi = torch.empty((Ns, nc * nc, 4, (rho + 1) ** 2), dtype=torch.float64, device=DEV)
    api.stomsfem_upscale(g, a_t, Ke, be, phi=phi)
    h, _ = api.stomsfem_pod_build(g, phi, a_t, ranks=ranks)
    api.stomsfem_pod_set_affine(h, g, F, w["tau"])
    xt = W.draw_xi(fld, 37, w["seed"])
    yield dict(oracle=oracle, pod=pod, w=w, g=g, F=F, models=models, ids=ids, h=h, xt=xt, nf=nf, nc=nc)
    api.stomsfem_pod_destroy(h)


def _rel(x, y):
    return float(np.max(np.linalg.norm(x - y, axis=-1) / np.linalg.norm(y, axis=-1)))


def _gpu(setup, refine):
    g, nc, nf = setup["g"], setup["nc"], setup["nf"]
    xt = torch.from_numpy(setup["xt"]).to(DEV)
    S = xt.shape[0]
    a = None
    if refine:
        a = torch.empty((S, nf, nf), dtype=torch.float64, device=DEV)
        api.stomsfem_sample_coef(g, setup["F"], xt, a)
    Ke = torch.empty((S, nc * nc, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((S, nc * nc, 4), dtype=torch.float64, device=DEV)
    st = torch.full((S, nc * nc), 9, dtype=torch.int32, device=DEV)
    api.stomsfem_pod_upscale_affine(setup["h"], g, xt, Ke, be, a=a, refine_iters=refine, unit_status=st)
    torch.cuda.synchronize()
    return Ke.cpu().numpy(), be.cpu().numpy(), st.cpu().numpy()


def test_affine_sampler_matches_oracle(setup):
    oracle, w, g = setup["oracle"], setup["w"], setup["g"]
    xt = setup["xt"][:5]
    a = torch.empty((5, w["nf"], w["nf"]), dtype=torch.float64, device=DEV)
    api.stomsfem_sample_coef(g, setup["F"], torch.from_numpy(xt).to(DEV), a)
    torch.cuda.synchronize()
    np.testing.assert_allclose(a.cpu().numpy(), oracle.sample_coef(w["nf"], w["field"], xt), rtol=1e-14)


def test_affine_online_matches_oracle(setup):
    """37 samples x 64 cells: K_e, b_e of the FP32 affine online stage
    against the oracle's Alg. 4 on the local affine coefficient."""
    pod, w = setup["pod"], setup["w"]
    Ko, bo = pod.upscale_affine(setup["models"], setup["nf"], setup["nc"], w["f"], w["field"], setup["xt"],
                                setup["ids"])
    Kg, bg, st = _gpu(setup, 0)
    assert (st == 0).all()
    assert _rel(Kg, Ko) <= 1e-4
    assert _rel(bg, bo) <= 1e-4


def test_affine_online_refined(setup):
    """FP64 refinement through the stencil of a: the reduced-basis solution
    itself (1e-10), on the sample's full coefficient, which the affine field
    and tau = 1e-6 make equal to the local one up to 1e-6."""
    pod, w = setup["pod"], setup["w"]
    oracle = setup["oracle"]
    a = oracle.sample_coef(setup["nf"], w["field"], setup["xt"])
    Ko, bo = pod.upscale(setup["models"], setup["nf"], setup["nc"], w["f"], a)
    Kg, bg, st = _gpu(setup, 4)
    assert (st == 0).all()
    assert _rel(Kg, Ko) <= 1e-10
    assert _rel(bg, bo) <= 1e-10


def test_affine_argument_errors(setup):
    g = setup["g"]
    with pytest.raises(_lib.StomsfemError):
        api.stomsfem_pod_set_affine(setup["h"], g, api.field_from_dict(W.workload("pod_64")["field"]), 1e-6)
    xt = torch.from_numpy(setup["xt"]).to(DEV)
    Ke = torch.empty((37, 64, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((37, 64, 4), dtype=torch.float64, device=DEV)
    with pytest.raises(_lib.StomsfemError):   # refinement without a
        api.stomsfem_pod_upscale_affine(setup["h"], g, xt, Ke, be, a=None, refine_iters=2)
