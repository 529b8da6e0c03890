"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (relative Frobenius per unit for K_e, relative L2 for the
coarse solution): FP64 path 1e-11 / 1e-9; FP32 factor + FP64 refinement
1e-10; FP32 throughout 1e-5.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1607_00693_gb300 import api
from paper_1607_00693_gb300 import workloads as W

TOL = {api.FP64: 1e-11, api.FP32_REFINED: 1e-10, api.FP32: 1e-5}
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1607_00693_gb300.build import build_library
    build_library()


def rel_unit(Kg, Ko):
    num = np.linalg.norm((Kg - Ko).reshape(-1, Ko.shape[-1]), axis=1)
    den = np.linalg.norm(Ko.reshape(-1, Ko.shape[-1]), axis=1)
    return float(np.max(num / den))


def gpu_upscale(nf, nc, f, a_np, ov=None, precision=api.FP64, refine=2, want_phi=False, status=False):
    g = api.grid(nf, nc, f)
    a = torch.from_numpy(a_np).to(DEV)
    S = a.shape[0]
    Ke = torch.empty((S, nc * nc, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((S, nc * nc, 4), dtype=torch.float64, device=DEV)
    phi = (torch.empty((S, nc * nc, 4, (nf // nc + 1) ** 2), dtype=torch.float64, device=DEV)
           if want_phi else None)
    st = torch.full((S, nc * nc), 99, dtype=torch.int32, device=DEV)
    o_t = None
    mo = 0
    if ov is not None:
        o_t = torch.from_numpy(np.ascontiguousarray(ov, dtype=np.int8)).to(DEV)
        mo = int(np.max(ov))
    api.stomsfem_upscale(g, a, Ke, be, oversample=o_t, max_oversample=mo, precision=precision,
                         refine_iters=refine, phi=phi, unit_status=st)
    torch.cuda.synchronize()
    out = [Ke.cpu().numpy(), be.cpu().numpy()]
    if want_phi:
        out.append(phi.cpu().numpy())
    if status:
        out.append(st.cpu().numpy())
    return out


def test_sample_coef_matches_oracle(orc):
    for name in ("msfem_64", "upscale_1024", "contrast_2048"):
        w = W.workload(name)
        nf = w["nf"] if name == "msfem_64" else 256
        xi = W.draw_xi(w["field"], 3, w["seed"], w["dist"])
        ref = orc.sample_coef(nf, w["field"], xi)
        a = torch.empty((3, nf, nf), dtype=torch.float64, device=DEV)
        api.stomsfem_sample_coef(api.grid(nf, w["nc"]), api.field_from_dict(w["field"]),
                                 torch.from_numpy(xi).to(DEV), a)
        got = a.cpu().numpy()
        assert np.max(np.abs(got / ref - 1)) < 1e-13, name


def test_sample_coef_fp32_arithmetic(orc):
    """The FP32-arithmetic sampler (for the FP32 upscaling form) against the
    FP64 oracle: z is a sum of nbx*nby FP32 products, so its absolute error is
    a few eps32 times the sum of |terms|; a = exp(scale z) turns that into a
    relative error of |scale| times it (EXP), and exp(c sigma(g z)) into
    c g / 4 times it (EXP_SIGMOID).  The bounds below are those estimates
    with the fields' largest sums of |terms|, times 4."""
    eps = 2.0 ** -24
    for name in ("msfem_64", "upscale_1024", "contrast_2048"):
        w = W.workload(name)
        fld = w["field"]
        nf = w["nf"] if name == "msfem_64" else 256
        xi = W.draw_xi(fld, 3, w["seed"], w["dist"])
        ref = orc.sample_coef(nf, fld, xi)
        a = torch.empty((3, nf, nf), dtype=torch.float64, device=DEV)
        api.stomsfem_sample_coef_precision(api.grid(nf, w["nc"]), api.field_from_dict(fld),
                                           torch.from_numpy(xi).to(DEV), a, precision=api.FP32)
        got = a.cpu().numpy()
        # sum of |xi_i psi_i(x)| over the bumps, bounded by max|xi| times the
        # largest bump sum (<= (1 + 2 sqrt(pi) w n)^2 for a lattice of spacing 1/n)
        nb = max(fld["nbx"], fld["nby"])
        tsum = np.abs(xi).max() * (1.0 + 2.0 * np.sqrt(np.pi) * fld["width"] * nb) ** 2
        if fld["kind"] == api.FIELD_EXP:
            gain = abs(fld.get("scale", 1.0))
        else:
            gain = fld["contrast_log"] * fld["gain"] / 4.0
        bound = 4 * (gain * tsum * 8 * eps + 4 * eps)
        err = np.max(np.abs(got / ref - 1))
        assert err <= bound, (name, err, bound)


@pytest.mark.parametrize("precision", [api.FP64, api.FP32_REFINED, api.FP32])
def test_upscale_msfem_64(orc, precision):
    w = W.workload("msfem_64")
    xi = W.draw_xi(w["field"], 16, w["seed"])
    a = orc.sample_coef(w["nf"], w["field"], xi)
    Ko, bo = orc.upscale(w["nf"], w["nc"], w["f"], a)
    Kg, bg = gpu_upscale(w["nf"], w["nc"], w["f"], a, precision=precision)
    assert rel_unit(Kg, Ko) <= TOL[precision]
    assert rel_unit(bg, bo) <= TOL[precision]


@pytest.mark.parametrize("precision", [api.FP64, api.FP32_REFINED, api.FP32])
def test_upscale_oversampled_rho32(orc, precision):
    """H/h = 32 with per-cell oversampling 0..4 (clipped at the domain
    boundary), several tiles of warps and a ragged tail of units."""
    nf, nc = 128, 4
    w = W.workload("upscale_1024")
    fld = dict(w["field"], nbx=4, nby=4, width=0.125)
    xi = W.draw_xi(fld, 3, 7)
    a = orc.sample_coef(nf, fld, xi)
    ov = np.random.default_rng(20).integers(0, 5, size=nc * nc).astype(np.int8)
    Ko, bo = orc.upscale(nf, nc, 1.0, a, ov)
    Kg, bg = gpu_upscale(nf, nc, 1.0, a, ov, precision=precision)
    assert rel_unit(Kg, Ko) <= TOL[precision]
    assert rel_unit(bg, bo) <= TOL[precision]


def test_phi_output_and_small_rho(orc):
    for (nf, nc, o) in [(16, 8, 0), (24, 4, 1), (12, 12, 0), (30, 3, 2)]:
        r = np.random.default_rng(nf)
        a = np.exp(r.uniform(-1.5, 1.5, size=(2, nf, nf)))
        ov = np.full(nc * nc, o, dtype=np.int8)
        Ko, bo, po = orc.upscale(nf, nc, 1.0, a, ov, want_phi=True)
        Kg, bg, pg = gpu_upscale(nf, nc, 1.0, a, ov, want_phi=True)
        assert rel_unit(Kg, Ko) <= 1e-11, (nf, nc, o)
        assert rel_unit(bg, bo) <= 1e-11
        assert np.max(np.abs(pg - po)) <= 1e-11


def test_coarse_solve_and_moments(orc):
    w = W.workload("msfem_64")
    xi = W.draw_xi(w["field"], 32, w["seed"])
    a = orc.sample_coef(w["nf"], w["field"], xi)
    Ko, bo = orc.upscale(w["nf"], w["nc"], w["f"], a)
    uo = orc.coarse_solve(w["nc"], Ko, bo)
    g = api.grid(w["nf"], w["nc"], w["f"])
    nn = (w["nc"] + 1) ** 2
    u = torch.empty((32, nn), dtype=torch.float64, device=DEV)
    mean = torch.zeros(nn, dtype=torch.float64, device=DEV)
    m2 = torch.zeros(nn, dtype=torch.float64, device=DEV)
    cnt = torch.zeros(1, dtype=torch.float64, device=DEV)
    Kt, bt = torch.from_numpy(Ko).to(DEV), torch.from_numpy(bo).to(DEV)
    # two uneven batches through the running accumulators
    api.stomsfem_coarse_solve(g, Kt[:20].contiguous(), bt[:20].contiguous(), u[:20], mean, m2, cnt)
    api.stomsfem_coarse_solve(g, Kt[20:].contiguous(), bt[20:].contiguous(), u[20:], mean, m2, cnt)
    torch.cuda.synchronize()
    ug = u.cpu().numpy()
    rel = np.linalg.norm(ug - uo, axis=1) / np.linalg.norm(uo, axis=1)
    assert rel.max() <= 1e-9
    mo, vo = orc.mc_moments(uo)
    assert cnt.item() == 32
    np.testing.assert_allclose(mean.cpu().numpy(), mo, rtol=1e-12, atol=1e-18)
    inner = vo > 0
    np.testing.assert_allclose((m2.cpu().numpy() / 32)[inner], vo[inner], rtol=1e-9)


def test_coarse_nc64_bandwidth(orc):
    """The widest coarse system (nc = 64, bandwidth 64: two window rows per lane)."""
    nc = 64
    r = np.random.default_rng(3)
    a = np.exp(r.uniform(-1, 1, size=(1, nc, nc)))
    Ko, bo = orc.upscale(nc, nc, 1.0, a)   # rho = 1: K_e = a_e K_ref
    uo = orc.coarse_solve(nc, Ko, bo)
    g = api.grid(nc, nc, 1.0)
    u = torch.empty((1, (nc + 1) ** 2), dtype=torch.float64, device=DEV)
    api.stomsfem_coarse_solve(g, torch.from_numpy(Ko).to(DEV), torch.from_numpy(bo).to(DEV), u)
    torch.cuda.synchronize()
    ug = u.cpu().numpy()
    assert np.linalg.norm(ug - uo) / np.linalg.norm(uo) <= 1e-9


def test_end_to_end_msfem_64(orc):
    """xi -> a -> K_e -> u on the GPU (all kernels), vs the oracle chain."""
    w = W.workload("msfem_64")
    S = w["samples"]
    xi = W.draw_xi(w["field"], S, w["seed"])
    a_o = orc.sample_coef(w["nf"], w["field"], xi)
    Ko, bo = orc.upscale(w["nf"], w["nc"], w["f"], a_o)
    uo = orc.coarse_solve(w["nc"], Ko, bo)
    g = api.grid(w["nf"], w["nc"], w["f"])
    a = torch.empty((S, w["nf"], w["nf"]), dtype=torch.float64, device=DEV)
    api.stomsfem_sample_coef(g, api.field_from_dict(w["field"]), torch.from_numpy(xi).to(DEV), a)
    Ke = torch.empty((S, w["nc"] ** 2, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((S, w["nc"] ** 2, 4), dtype=torch.float64, device=DEV)
    api.stomsfem_upscale(g, a, Ke, be)
    u = torch.empty((S, (w["nc"] + 1) ** 2), dtype=torch.float64, device=DEV)
    api.stomsfem_coarse_solve(g, Ke, be, u)
    torch.cuda.synchronize()
    ug = u.cpu().numpy()
    rel = np.linalg.norm(ug - uo, axis=1) / np.linalg.norm(uo, axis=1)
    assert rel.max() <= 1e-9


def test_full_size_upscale_1024_sampled(orc):
    """The H/h = 32 workload at full grid size (1024^2, oversampling 0..4)
    in the bench's launch configuration; sampled units against the oracle
    one by one."""
    w = W.workload("upscale_1024")
    S = 2
    xi = W.draw_xi(w["field"], S, w["seed"])
    ov = W.draw_oversample(w["nc"], w["oversample"])
    a = orc.sample_coef(w["nf"], w["field"], xi, nthreads=0)
    res = {}
    for prec in (api.FP64, api.FP32_REFINED, api.FP32):
        res[prec] = gpu_upscale(w["nf"], w["nc"], w["f"], a, ov, precision=prec)
    r = np.random.default_rng(0)
    for u in list(r.choice(S * w["nc"] ** 2, size=12, replace=False)) + [0, S * w["nc"] ** 2 - 1]:
        s, cell = divmod(int(u), w["nc"] ** 2)
        cx, cy = cell % w["nc"], cell // w["nc"]
        Ko, bo, _, _ = orc.cell(w["nf"], w["nc"], w["f"], a[s], cx, cy, int(ov[cell]))
        for prec, (Kg, bg) in res.items():
            k = Kg[s, cell]
            assert np.linalg.norm(k - Ko) / np.linalg.norm(Ko) <= TOL[prec], (prec, u)
            assert np.linalg.norm(bg[s, cell] - bo) / np.linalg.norm(bo) <= TOL[prec], (prec, u)
    # properties at every unit: zero row sums and loads summing to f H^2
    H = 1.0 / w["nc"]
    for prec, (Kg, bg) in res.items():
        tol = max(TOL[prec], 1e-12)
        assert np.max(np.abs(bg.sum(axis=2) - H * H)) <= tol * H * H
        K = Kg.reshape(-1, 10)
        rows = np.stack([K[:, 0] + K[:, 1] + K[:, 2] + K[:, 3], K[:, 1] + K[:, 4] + K[:, 5] + K[:, 6],
                         K[:, 2] + K[:, 5] + K[:, 7] + K[:, 8], K[:, 3] + K[:, 6] + K[:, 8] + K[:, 9]])
        assert np.max(np.abs(rows)) <= max(tol, 1e-9) * np.max(np.abs(K))


def test_status_on_indefinite_unit(orc):
    """A negative coefficient in one cell makes that unit's matrix
    indefinite: its status reports the pivot, its outputs are NaN, every
    other unit is unaffected."""
    nf, nc = 32, 4
    r = np.random.default_rng(1)
    a = np.exp(r.uniform(-1, 1, size=(1, nf, nf)))
    a[0, 12:20, 12:20] = -5.0   # inside cell (1..2, 1..2)
    Ko, bo = orc.upscale(nf, nc, 1.0, np.abs(a))
    Kg, bg, st = gpu_upscale(nf, nc, 1.0, a, status=True)
    bad = st[0] != 0
    assert bad.any() and np.all(st[0][bad] > 0)
    assert np.all(np.isnan(Kg[0][bad]))
    good = ~bad
    assert np.all(np.isfinite(Kg[0][good]))


@pytest.mark.parametrize("precision", [api.FP32, api.FP32_REFINED])
def test_paired_units_one_indefinite(orc, precision):
    """The FP32 forms factorise one cell of two consecutive samples per warp
    in lockstep.  Sample 1 has an indefinite cell: that unit alone reports
    its pivot and NaN outputs; its warp partner (sample 0, same cell), the
    other cells of sample 1 and the unpaired last sample (S odd) match the
    oracle."""
    nf, nc = 64, 2
    r = np.random.default_rng(5)
    a = np.exp(r.uniform(-1, 1, size=(3, nf, nf)))
    a[1, 40:50, 40:50] = -5.0   # inside cell (1, 1) of sample 1
    ov = np.array([0, 1, 2, 3], dtype=np.int8)
    Kg, bg, st = gpu_upscale(nf, nc, 1.0, a, ov, precision=precision, status=True)
    assert st[1, 3] > 0 and np.all(np.isnan(Kg[1, 3])) and np.all(np.isnan(bg[1, 3]))
    ok = np.ones((3, nc * nc), dtype=bool)
    ok[1, 3] = False
    assert np.all(st[ok] == 0)
    Ko, bo = orc.upscale(nf, nc, 1.0, np.abs(a), ov)
    num = np.linalg.norm(Kg - Ko, axis=-1)[ok]
    assert np.max(num / np.linalg.norm(Ko, axis=-1)[ok]) <= TOL[precision]
    assert np.max(np.linalg.norm(bg - bo, axis=-1)[ok] / np.linalg.norm(bo, axis=-1)[ok]) <= TOL[precision]


def test_fp32_forward_only_route(orc):
    """In the FP32 form, cells without oversampling (and no phi output) get
    K_e = p^T A p - y^T y and the load from z . y (forward substitution
    only); asking for phi forces the back-substitution route.  Both agree
    with the FP64 oracle within the FP32 tolerance, and with each other."""
    nf, nc = 128, 4
    r = np.random.default_rng(3)
    a = np.exp(r.uniform(-4.6, 4.6, size=(3, nf, nf)))     # contrast up to 1e4
    Ko, bo = orc.upscale(nf, nc, 1.0, a)
    K1, b1 = gpu_upscale(nf, nc, 1.0, a, precision=api.FP32)
    K2, b2, _ = gpu_upscale(nf, nc, 1.0, a, precision=api.FP32, want_phi=True)
    for K, b in ((K1, b1), (K2, b2)):
        assert rel_unit(K, Ko) <= TOL[api.FP32]
        assert rel_unit(b, bo) <= TOL[api.FP32]
    assert rel_unit(K1, K2) <= TOL[api.FP32]


@pytest.mark.parametrize("layout", ["all_zero", "none_zero", "mixed"])
def test_fp32_split_launch_cell_lists(orc, layout):
    """The FP32 form with an oversample array runs the cells without
    oversampling and the others as two launches from device cell lists;
    either list may be empty.  A workspace without room for the lists after
    the slots falls back to one launch.  All agree with the oracle."""
    nf, nc = 64, 4
    r = np.random.default_rng(11)
    a = np.exp(r.uniform(-1.5, 1.5, size=(3, nf, nf)))
    ov = {"all_zero": np.zeros(nc * nc), "none_zero": r.integers(1, 4, size=nc * nc),
          "mixed": r.integers(0, 3, size=nc * nc)}[layout].astype(np.int8)
    Ko, bo = orc.upscale(nf, nc, 1.0, a, ov)
    Kg, bg = gpu_upscale(nf, nc, 1.0, a, ov, precision=api.FP32)
    assert rel_unit(Kg, Ko) <= TOL[api.FP32]
    assert rel_unit(bg, bo) <= TOL[api.FP32]
    # one block of slots exactly: no room for the cell lists, single launch
    g = api.grid(nf, nc)
    slot, _ = api.stomsfem_upscale_workspace_size(g, 3, api.FP32)
    ws = torch.empty(8 * slot, dtype=torch.uint8, device=DEV)
    at = torch.from_numpy(a).to(DEV)
    Ke = torch.empty((3, nc * nc, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((3, nc * nc, 4), dtype=torch.float64, device=DEV)
    api.stomsfem_upscale(g, at, Ke, be, oversample=torch.from_numpy(ov).to(DEV), max_oversample=3,
                         precision=api.FP32, workspace=ws)
    torch.cuda.synchronize()
    assert rel_unit(Ke.cpu().numpy(), Ko) <= TOL[api.FP32]
    assert rel_unit(be.cpu().numpy(), bo) <= TOL[api.FP32]


def _assemble_residual(Ke, be, u, nc):
    """|| S u - b || / ||b|| for the coarse system assembled from K_e, b_e
    (written out here independently of both the library and the oracle)."""
    NN = nc + 1
    r = np.zeros(NN * NN)
    b = np.zeros(NN * NN)
    loc = [(0, 0), (1, 0), (1, 1), (0, 1)]
    for cell in range(nc * nc):
        cx, cy = cell % nc, cell // nc
        K = np.zeros((4, 4))
        q = 0
        for l in range(4):
            for lp in range(l, 4):
                K[l, lp] = K[lp, l] = Ke[cell, q]
                q += 1
        idx = [(cy + dy) * NN + cx + dx for (dx, dy) in loc]
        r[idx] += K @ u[idx]
        b[idx] += be[cell]
    inner = np.zeros((NN, NN), dtype=bool)
    inner[1:-1, 1:-1] = True
    inner = inner.reshape(-1)
    return np.linalg.norm((r - b)[inner]) / np.linalg.norm(b[inner])


def test_full_size_contrast_2048_sampled(orc):
    """High-contrast workload at full size (2048^2 fine, 64^2 coarse, contrast
    1e4, 32x32 bumps, xi ~ N(0,1)): sampled units against the oracle (which
    evaluates the coefficient on each sampled patch itself), and the coarse
    solve checked through the residual of the assembled coarse system."""
    w = W.workload("contrast_2048")
    S, nf, nc = 2, w["nf"], w["nc"]
    xi = W.draw_xi(w["field"], S, w["seed"], w["dist"])
    g = api.grid(nf, nc, w["f"])
    a = torch.empty((S, nf, nf), dtype=torch.float64, device=DEV)
    api.stomsfem_sample_coef(g, api.field_from_dict(w["field"]), torch.from_numpy(xi).to(DEV), a)
    res = {}
    for prec in (api.FP64, api.FP32_REFINED, api.FP32):
        Ke = torch.empty((S, nc * nc, 10), dtype=torch.float64, device=DEV)
        be = torch.empty((S, nc * nc, 4), dtype=torch.float64, device=DEV)
        api.stomsfem_upscale(g, a, Ke, be, precision=prec)
        res[prec] = (Ke, be)
    u = torch.empty((S, (nc + 1) ** 2), dtype=torch.float64, device=DEV)
    api.stomsfem_coarse_solve(g, res[api.FP64][0], res[api.FP64][1], u)
    torch.cuda.synchronize()
    rho = nf // nc
    r = np.random.default_rng(5)
    for u_ in list(r.choice(S * nc * nc, size=6, replace=False)) + [S * nc * nc - 1]:
        s, cell = divmod(int(u_), nc * nc)
        cx, cy = cell % nc, cell // nc
        ao = orc.sample_coef_window(nf, w["field"], xi[s], cx * rho, (cx + 1) * rho, cy * rho,
                                    (cy + 1) * rho)
        Ko, bo, _, _ = orc.cell(nf, nc, w["f"], ao, cx, cy, 0)
        for prec, (Ke, be) in res.items():
            k = Ke[s, cell].cpu().numpy()
            assert np.linalg.norm(k - Ko) / np.linalg.norm(Ko) <= TOL[prec], (prec, u_)
            assert np.linalg.norm(be[s, cell].cpu().numpy() - bo) / np.linalg.norm(bo) <= TOL[prec]
    Kn, bn, un = res[api.FP64][0].cpu().numpy(), res[api.FP64][1].cpu().numpy(), u.cpu().numpy()
    for s in range(S):
        assert _assemble_residual(Kn[s], bn[s], un[s], nc) <= 1e-10
