"""Random interpolation on the GPU (Sec. 3.1, Algorithms 1-2) against the
oracle: the offline collocation data, the online interpolant (second
barycentric form, FP32 sum) on ragged family tiles, exact nodes, the direct
fallback outside the collocation box, and the degenerate all-frozen case."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1607_00693_gb300 import api
from paper_1607_00693_gb300 import workloads as W

DEV = "cuda:0"
# FP32 sum over <= 360 grid points with Lagrange weights of Lebesgue
# constant <= 3 per direction: 2e-5 of the unit's largest entry
RTOL_UNIT = 2e-5


@pytest.fixture(scope="module")
def setup():
    from paper_1607_00693_gb300.build import build_library
    import oracle
    from oracle import ri
    build_library()
    oracle.build()
    w = W.workload("msfem_64")
    g = api.grid(w["nf"], w["nc"], w["f"])
    fld = api.field_from_dict(w["field"])
    models = {}
    for kind in (api.RI_CHEBYSHEV, api.RI_LEGENDRE):
        h, nfam = api.stomsfem_ri_build(g, fld, 1e-3, 8, kind)
        m = ri.build(w["nf"], w["nc"], w["f"], w["field"], 1e-3, 8, kind)
        assert nfam == len(m["keys"])
        models[kind] = (h, m)
    yield oracle, ri, w, g, fld, models
    for h, _ in models.values():
        api.stomsfem_ri_destroy(h)


def _unit_close(K, Ko, rtol=RTOL_UNIT):
    scale = np.abs(Ko).max(axis=-1, keepdims=True)
    return np.abs(K - Ko) <= rtol * scale


@pytest.mark.parametrize("kind", [0, 1])
def test_collocation_data_match_oracle(setup, kind):
    """Offline stage: the FP64 upscaler on the GPU at every grid point of every
    family equals the oracle's direct upscale (both FP64)."""
    _, _, _, _, _, models = setup
    h, m = models[kind]
    Vo = np.concatenate(m["V"])
    V = api.stomsfem_ri_values(h, len(Vo))
    np.testing.assert_allclose(V, Vo, rtol=1e-10, atol=1e-13)


def _run(g, h, xi, a=None):
    S = xi.shape[0]
    ncell = g.nc * g.nc
    Ke = torch.full((S, ncell, 10), 7.0, dtype=torch.float64, device=DEV)
    be = torch.full((S, ncell, 4), 7.0, dtype=torch.float64, device=DEV)
    fb = torch.full((S, ncell), 9, dtype=torch.uint8, device=DEV)
    api.stomsfem_ri_upscale(h, g, xi, a, Ke, be, fb)
    torch.cuda.synchronize()
    return Ke.cpu().numpy(), be.cpu().numpy(), fb.cpu().numpy()


@pytest.mark.parametrize("kind", [0, 1])
def test_online_matches_oracle_ragged_tiles(setup, kind):
    """S = 37 samples: every family's unit count (37 x its cells) leaves a
    ragged last tile of 256; every unit against the oracle's interpolant."""
    oracle, ri, w, g, _, models = setup
    h, m = models[kind]
    xi = W.draw_xi(w["field"], 37, 1234 + kind)
    Ke, be, fb = _run(g, h, torch.tensor(xi, device=DEV))
    assert (fb == 0).all()
    for s in range(xi.shape[0]):
        for c in range(g.nc * g.nc):
            Ko, bo = ri.evaluate(m, xi[s], c)
            assert _unit_close(Ke[s, c], Ko).all(), (s, c)
            assert _unit_close(be[s, c], bo).all(), (s, c)


def test_exact_nodes_and_box_corners(setup):
    """Local parameters exactly at grid nodes return the collocation data
    (the barycentric form's exact-node branch); +-1 is inside the box."""
    _, ri, w, g, _, models = setup
    h, m = models[api.RI_CHEBYSHEV]
    K = W.n_vars(w["field"])
    rng = np.random.default_rng(5)
    S = 64
    xi = np.zeros((S, K))
    cell = 27
    d = m["dims"][cell]
    xs = [ri.nodes(m["kind"], nu) for (_, _, nu, _) in d]
    idx = [rng.integers(0, len(x), S) for x in xs]
    for k, (_, _, _, var) in enumerate(d):
        xi[:, var] = xs[k][idx[k]]
    xi[0, [v for (_, _, _, v) in d]] = 1.0
    xi[1, [v for (_, _, _, v) in d]] = -1.0
    Ke, be, fb = _run(g, h, torch.tensor(xi, device=DEV))
    assert (fb == 0).all()
    V = m["V"][m["fam"][cell]]
    radix = [len(x) for x in xs]
    for s in range(2, S):
        p = 0
        for k in range(len(d)):
            p = p * radix[k] + int(idx[k][s])
        # FP32 nodes: the node test is exact in FP32, the data rounded to FP32
        np.testing.assert_allclose(Ke[s, cell], V[p, :10], rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(be[s, cell], V[p, 10:], rtol=1e-6, atol=1e-9)
    for s in (0, 1):
        Ko, bo = ri.evaluate(m, xi[s], cell)
        assert _unit_close(Ke[s, cell], Ko).all()


def test_box_exit_falls_back_to_fp64(setup):
    """Normal xi (some |xi_i| > 1): units with a local parameter outside the
    box are upscaled directly in FP64 (fell_back = 1, equal to the oracle's
    direct cell solve); the rest interpolated; without a coefficient they get
    NaN and fell_back = 2."""
    oracle, ri, w, g, fld, models = setup
    h, m = models[api.RI_LEGENDRE]
    xi = W.draw_xi(w["field"], 9, 77, dist="normal")
    xt = torch.tensor(xi, device=DEV)
    a = torch.empty((9, w["nf"], w["nf"]), dtype=torch.float64, device=DEV)
    api.stomsfem_sample_coef(g, fld, xt, a)
    Ke, be, fb = _run(g, h, xt, a)
    ao = oracle.sample_coef(w["nf"], w["field"], xi)
    Ko, bo, fbo = ri.upscale(m, xi, ao)
    np.testing.assert_array_equal(fb, fbo)
    assert 0 < fb.sum() < fb.size
    out = fb == 1
    np.testing.assert_allclose(Ke[out], Ko[out], rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(be[out], bo[out], rtol=1e-10, atol=1e-15)
    assert _unit_close(Ke[~out], Ko[~out]).all() and _unit_close(be[~out], bo[~out]).all()
    Ke2, be2, fb2 = _run(g, h, xt, None)
    np.testing.assert_array_equal(fb2, np.where(out, 2, 0))
    assert np.isnan(Ke2[out]).all() and np.isnan(be2[out]).all()
    np.testing.assert_array_equal(Ke2[~out], Ke[~out])


def test_all_frozen_and_empty(setup):
    """eps above every strength: one grid point, every unit gets the a = 1
    upscale (K_ref, f H^2 / 4); S = 0 is a no-op."""
    _, _, w, g, fld, _ = setup
    h, nfam = api.stomsfem_ri_build(g, fld, 10.0, 8)
    try:
        assert nfam == 1
        xi = W.draw_xi(w["field"], 5, 3)
        Ke, be, fb = _run(g, h, torch.tensor(xi, device=DEV))
        kref = np.array([4, -1, -2, -1, 4, -1, -2, 4, -1, 4]) / 6.0
        np.testing.assert_allclose(Ke, np.broadcast_to(kref, Ke.shape), rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(be, 1.0 / 64 / 4, rtol=1e-6)
        assert (fb == 0).all()
        e = torch.empty((0, 64, 10), dtype=torch.float64, device=DEV)
        api.stomsfem_ri_upscale(h, g, torch.empty((0, 16), dtype=torch.float64, device=DEV), None, e,
                                torch.empty((0, 64, 4), dtype=torch.float64, device=DEV),
                                torch.empty((0, 64), dtype=torch.uint8, device=DEV))
    finally:
        api.stomsfem_ri_destroy(h)


def test_full_size_sampled_and_coarse_error(setup):
    """10^5 samples (the bench's launch): 300 sampled units against the oracle,
    and the coarse solutions of 64 samples within 1e-4 of plain FP64 MsFEM."""
    oracle, ri, w, g, fld, models = setup
    h, m = models[api.RI_LEGENDRE]
    S = 100000
    xi = W.draw_xi(w["field"], S, W.workload("ri_64")["seed"])
    xt = torch.tensor(xi, device=DEV)
    Ke = torch.empty((S, 64, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((S, 64, 4), dtype=torch.float64, device=DEV)
    fb = torch.empty((S, 64), dtype=torch.uint8, device=DEV)
    api.stomsfem_ri_upscale(h, g, xt, None, Ke, be, fb)
    torch.cuda.synchronize()
    assert int(fb.sum().item()) == 0
    rng = np.random.default_rng(11)
    for s, c in zip(rng.integers(0, S, 300), rng.integers(0, 64, 300)):
        Ko, bo = ri.evaluate(m, xi[s], int(c))
        assert _unit_close(Ke[s, c].cpu().numpy(), Ko).all()
        assert _unit_close(be[s, c].cpu().numpy(), bo).all()
    n = 64
    a = torch.empty((n, 64, 64), dtype=torch.float64, device=DEV)
    api.stomsfem_sample_coef(g, fld, xt[:n].contiguous(), a)
    K0 = torch.empty((n, 64, 10), dtype=torch.float64, device=DEV)
    b0 = torch.empty((n, 64, 4), dtype=torch.float64, device=DEV)
    api.stomsfem_upscale(g, a, K0, b0)
    u0 = oracle.coarse_solve(8, K0.cpu().numpy(), b0.cpu().numpy())
    u1 = oracle.coarse_solve(8, Ke[:n].cpu().numpy(), be[:n].cpu().numpy())
    assert np.linalg.norm(u1 - u0) / np.linalg.norm(u0) < 1e-4


def test_many_directions_low_degree(setup):
    """eps = 1e-4 with degrees capped at 2: up to 8 directions and 1296 grid
    points per family, so several outer directions around the inner block."""
    oracle, ri, w, g, fld, _ = setup
    h, nfam = api.stomsfem_ri_build(g, fld, 1e-4, 2, api.RI_CHEBYSHEV)
    try:
        m = ri.build(w["nf"], w["nc"], w["f"], w["field"], 1e-4, 2, ri.CHEBYSHEV)
        assert nfam == len(m["keys"]) and max(len(d) for d in m["dims"]) == 8
        Vo = np.concatenate(m["V"])
        np.testing.assert_allclose(api.stomsfem_ri_values(h, len(Vo)), Vo, rtol=1e-10, atol=1e-13)
        xi = W.draw_xi(w["field"], 3, 99)
        Ke, be, fb = _run(g, h, torch.tensor(xi, device=DEV))
        assert (fb == 0).all()
        for s in range(3):
            for c in range(64):
                Ko, bo = ri.evaluate(m, xi[s], c)
                assert _unit_close(Ke[s, c], Ko).all(), (s, c)
                assert _unit_close(be[s, c], bo).all(), (s, c)
    finally:
        api.stomsfem_ri_destroy(h)


def test_checkpoint_roundtrip(setup):
    """save -> load gives the same data and the same online results, with no
    offline solves; the stored plan is checked against the re-derived one."""
    _, _, w, g, _, models = setup
    h, m = models[api.RI_LEGENDRE]
    blob = api.stomsfem_ri_save(h)
    assert blob[:8] == b"STMFRIT1"
    h2, nfam = api.stomsfem_ri_load(blob)
    try:
        assert nfam == len(m["keys"])
        n = sum(len(v) for v in m["V"])
        np.testing.assert_array_equal(api.stomsfem_ri_values(h2, n), api.stomsfem_ri_values(h, n))
        xi = torch.tensor(W.draw_xi(w["field"], 11, 5), device=DEV)
        r1, r2 = _run(g, h, xi), _run(g, h2, xi)
        for x, y in zip(r1, r2):
            np.testing.assert_array_equal(x, y)
    finally:
        api.stomsfem_ri_destroy(h2)
