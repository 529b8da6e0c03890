"""Every entry point that takes a caller's workspace gives the same results
whatever the workspace held before the call: each is run once on a zeroed
workspace and once on one whose every byte is 0xFF (a NaN in FP32 and FP64),
and the outputs must be finite and agree (bit for bit where the kernels
have a fixed summation order, else to 1e-12).  A kernel that read scratch
before writing it, even multiplied by zero, would carry the NaN into its
results."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1607_00693_gb300 import api
from paper_1607_00693_gb300 import workloads as W

DEV = "cuda:0"

@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1607_00693_gb300.build import build_library
    build_library()

def _ws(nbytes, fill):
    return torch.full((max(int(nbytes), 1),), fill, dtype=torch.uint8, device=DEV)

def _twice(run, nbytes):
    """run(workspace) -> list of output tensors, on a zeroed and on a NaN-filled workspace."""
    outs = []
    for fill in (0, 0xFF):
        res = run(_ws(nbytes, fill))
        torch.cuda.synchronize()
        outs.append([t.detach().cpu().numpy().copy() for t in res])
    return outs

def _same(outs, exact, what):
    for x0, x1 in zip(*outs):
        assert np.all(np.isfinite(x0)) and np.all(np.isfinite(x1)), what
        if exact:
            np.testing.assert_array_equal(x0, x1, err_msg=what)
        else:
            np.testing.assert_allclose(x1, x0, rtol=1e-12, atol=1e-14 * float(np.abs(x0).max()), err_msg=what)

def _coef(name, S, seed, nf=None, nc=None):
    w = W.workload(name)
    nf = nf or w["nf"]
    nc = nc or w["nc"]
    g = api.grid(nf, nc, w["f"])
    fld = api.field_from_dict(w["field"])
    xi = torch.from_numpy(W.draw_xi(w["field"], S, seed, w["dist"])).to(DEV)
    a = torch.empty((S, nf, nf), dtype=torch.float64, device=DEV)
    api.stomsfem_sample_coef(g, fld, xi, a)
    return w, g, fld, xi, a

@pytest.mark.parametrize("nf,S,channels", [(64, 3, False), (128, 2, False), (128, 2, True)])
def test_fine_fem(nf, S, channels):
    """The direct path (nf <= 64) and the multigrid CG (above) with bilinear
    transfers (a lognormal medium) and with operator-dependent ones (a
    channel medium of contrast 10^4)."""
    if channels:
        fd = dict(W.workload("contrast_2048")["field"], nbx=16, nby=16, width=1.5 / 16)
        g = api.grid(nf, 4, 1.0)
        xi = torch.from_numpy(W.draw_xi(fd, S, 3, "normal")).to(DEV)
        a = torch.empty((S, nf, nf), dtype=torch.float64, device=DEV)
        api.stomsfem_sample_coef(g, api.field_from_dict(fd), xi, a)
        assert float(a.max() / a.min()) > 1e3
    else:
        _, g, _, _, a = _coef("upscale_1024", S, 3, nf=nf, nc=4)
    u = torch.empty((S, (nf + 1) ** 2), dtype=torch.float64, device=DEV)

    def run(ws):
        api.stomsfem_fine_fem(g, a, u, workspace=ws)
        return [u]

    # the CG's dot products are block sums with atomics: agreement to rounding
    _same(_twice(run, api.stomsfem_fine_fem_workspace_size(g, S)), exact=nf <= 64, what="fine FEM")

@pytest.mark.parametrize("prec", [api.FP64, api.FP32_REFINED, api.FP32])
def test_upscale_with_oversampling(prec):
    S, nf, nc = 3, 128, 4
    _, g, _, _, a = _coef("upscale_1024", S, 5, nf=nf, nc=nc)
    ov = torch.from_numpy(np.array([0, 1, 2, 3] * 4, dtype=np.int8)).to(DEV)
    Ke = torch.empty((S, nc * nc, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((S, nc * nc, 4), dtype=torch.float64, device=DEV)
    _, rb = api.stomsfem_upscale_workspace_size(g, 3, prec)

    def run(ws):
        api.stomsfem_upscale(g, a, Ke, be, oversample=ov, max_oversample=3, precision=prec, refine_iters=1,
                             workspace=ws)
        return [Ke, be]

    _same(_twice(run, rb), exact=True, what="upscale precision %d" % prec)

def test_coarse_solves():
    S, nf, nc = 4, 64, 8
    _, g, _, _, a = _coef("msfem_64", S, 7, nf=nf, nc=nc)
    Ke = torch.empty((S, nc * nc, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((S, nc * nc, 4), dtype=torch.float64, device=DEV)
    api.stomsfem_upscale(g, a, Ke, be)
    u = torch.empty((S, (nc + 1) ** 2), dtype=torch.float64, device=DEV)

    def run(ws):
        api.stomsfem_coarse_solve(g, Ke, be, u, workspace=ws)
        return [u]

    _same(_twice(run, api.stomsfem_coarse_workspace_size(g, S)), exact=True, what="coarse solve")
    Kpg = torch.empty((S, nc * nc, 16), dtype=torch.float64, device=DEV)
    api.stomsfem_upscale_pg(g, a, Kpg, be)

    def run_pg(ws):
        api.stomsfem_coarse_solve_pg(g, Kpg, be, u, workspace=ws)
        return [u]

    _same(_twice(run_pg, api.stomsfem_coarse_pg_workspace_size(g, S)), exact=True, what="Petrov-Galerkin solve")

def test_pod_surrogate_interpolation():
    """The reduced forms on the 64^2 / 8^2 grid: POD (FP64 refinement and the
    tensor-core path), the surrogate with an ensemble partner (untrained
    networks: most units fall back, so the fallback upscaling runs too) and
    random interpolation."""
    S = 5
    w, g, fld, xi, a = _coef("pod_64", 12, 11)
    nc = w["nc"]
    rho = w["nf"] // nc
    Ke0 = torch.empty((12, nc * nc, 10), dtype=torch.float64, device=DEV)
    be0 = torch.empty((12, nc * nc, 4), dtype=torch.float64, device=DEV)
    phi = torch.empty((12, nc * nc, 4, (rho + 1) ** 2), dtype=torch.float64, device=DEV)
    api.stomsfem_upscale(g, a, Ke0, be0, phi=phi)
    hp, _ = api.stomsfem_pod_build(g, phi, a, tol=1e-6, max_rank=12)
    a5, xi5 = a[:S].contiguous(), xi[:S].contiguous()
    Ke = torch.empty((S, nc * nc, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((S, nc * nc, 4), dtype=torch.float64, device=DEV)
    fb = torch.empty((S, nc * nc), dtype=torch.uint8, device=DEV)
    try:
        for refine in (0, 2):
            def run_pod(ws):
                api.stomsfem_pod_upscale(hp, g, a5, Ke, be, refine_iters=refine, workspace=ws)
                return [Ke, be]

            _same(_twice(run_pod, api.stomsfem_pod_workspace_size(hp, S)), exact=True, what="POD refine %d" % refine)
    finally:
        api.stomsfem_pod_destroy(hp)
    _, _, _, nfam = api.stomsfem_local_vars(g, fld, 1e-6)
    h1, _ = api.stomsfem_surrogate_create(g, fld, 1e-6, api.xavier_weights(nfam, 0))
    h2, _ = api.stomsfem_surrogate_create(g, fld, 1e-6, api.xavier_weights(nfam, 1))
    try:
        api.stomsfem_surrogate_set_partner(h1, h2, 0.02)

        def run_sur(ws):
            api.stomsfem_surrogate_infer(h1, g, xi5, a5, Ke, be, fb, workspace=ws)
            return [Ke, be, fb]

        _same(_twice(run_sur, api.stomsfem_surrogate_workspace_size(h1, S)), exact=True, what="surrogate")
    finally:
        api.stomsfem_surrogate_destroy(h1)
        api.stomsfem_surrogate_destroy(h2)
    wr = W.workload("ri_64")
    gr = api.grid(wr["nf"], wr["nc"], wr["f"])
    fr = api.field_from_dict(wr["field"])
    hr, _ = api.stomsfem_ri_build(gr, fr, wr["eps"], wr["nu_max"], wr["nodes"])
    xr = torch.from_numpy(W.draw_xi(wr["field"], S, 13)).to(DEV)
    ar = torch.empty((S, wr["nf"], wr["nf"]), dtype=torch.float64, device=DEV)
    api.stomsfem_sample_coef(gr, fr, xr, ar)
    try:
        def run_ri(ws):
            api.stomsfem_ri_upscale(hr, gr, xr, ar, Ke, be, fb, workspace=ws)
            return [Ke, be, fb]

        _same(_twice(run_ri, api.stomsfem_ri_workspace_size(hr, S)), exact=True, what="random interpolation")
    finally:
        api.stomsfem_ri_destroy(hr)
