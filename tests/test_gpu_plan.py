"""Plans on the GPU: the captured step (sample -> upscale -> coarse solve
-> moments) reproduces the direct calls bit for bit, replays and
re-captures, its timing events, the autotuner's choices, every
factorisation engine and unit order against the oracle, and the
default-stream path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1607_00693_gb300 import api
from paper_1607_00693_gb300 import workloads as W

DEV = "cuda:0"


@pytest.fixture(scope="module")
def case():
    from paper_1607_00693_gb300.build import build_library
    build_library()
    nf, nc, S = 128, 4, 6
    fld_d = dict(W.workload("upscale_1024")["field"], nbx=4, nby=4, width=0.125)
    g = api.grid(nf, nc, 1.0)
    fld = api.field_from_dict(fld_d)
    ov = np.random.default_rng(20).integers(0, 5, size=nc * nc).astype(np.int8)
    xt = torch.from_numpy(W.draw_xi(fld_d, S, 77)).to(DEV)
    return dict(g=g, fld=fld, ov=torch.from_numpy(ov).to(DEV), mo=int(ov.max()), xt=xt, S=S, nn=(nc + 1) ** 2)


def _direct(c, prec):
    g, S = c["g"], c["S"]
    a = torch.empty((S, g.nf, g.nf), dtype=torch.float64, device=DEV)
    api.stomsfem_sample_coef_precision(g, c["fld"], c["xt"], a, precision=api.FP32 if prec == api.FP32 else api.FP64)
    Ke = torch.empty((S, g.nc * g.nc, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((S, g.nc * g.nc, 4), dtype=torch.float64, device=DEV)
    api.stomsfem_upscale(g, a, Ke, be, oversample=c["ov"], max_oversample=c["mo"], precision=prec, refine_iters=2)
    u = torch.empty((S, c["nn"]), dtype=torch.float64, device=DEV)
    api.stomsfem_coarse_solve(g, Ke, be, u)
    torch.cuda.synchronize()
    return u.cpu().numpy()


@pytest.mark.parametrize("prec", [api.FP64, api.FP32_REFINED, api.FP32])
def test_plan_step_equals_direct_calls(case, prec):
    c = case
    u0 = _direct(c, prec)
    h = api.stomsfem_plan_create(c["g"], c["fld"], c["S"], prec, oversample=c["ov"], max_oversample=c["mo"])
    try:
        st = torch.cuda.Stream()
        u = torch.empty((c["S"], c["nn"]), dtype=torch.float64, device=DEV)
        with torch.cuda.stream(st):
            api.stomsfem_plan_step(h, c["xt"], u, use_graph=False, stream=st)
            st.synchronize()
            np.testing.assert_array_equal(u.cpu().numpy(), u0)
            u.fill_(0.0)
            api.stomsfem_plan_step(h, c["xt"], u, stream=st)       # capture + launch
            st.synchronize()
            np.testing.assert_array_equal(u.cpu().numpy(), u0)
            assert api.stomsfem_plan_info(h)[4] == 1
            t_up = api.stomsfem_plan_upscale_ms(h)     # events inside the graph
            assert 0.0 < t_up < 1e4
            u.fill_(0.0)
            api.stomsfem_plan_step(h, c["xt"], u, stream=st)       # replay
            st.synchronize()
            np.testing.assert_array_equal(u.cpu().numpy(), u0)
            # moments through the graph: the same batch twice
            mean = torch.zeros(c["nn"], dtype=torch.float64, device=DEV)
            m2 = torch.zeros_like(mean)
            cnt = torch.zeros(1, dtype=torch.float64, device=DEV)
            for _ in range(2):
                api.stomsfem_plan_step(h, c["xt"], u, mean, m2, cnt, stream=st)
            st.synchronize()
        assert cnt.item() == 2 * c["S"]
        np.testing.assert_allclose(mean.cpu().numpy(), u0.mean(axis=0), rtol=1e-12, atol=1e-18)
        np.testing.assert_allclose(m2.cpu().numpy() / (2 * c["S"]), u0.var(axis=0), rtol=1e-9, atol=1e-20)
    finally:
        api.stomsfem_plan_destroy(h)


def test_plan_tune_and_recapture(case):
    """FP32 with oversampling: launch choices (engine, unit order, split,
    blocks per SM) timed; the chosen one reproduces the direct result (bit
    for bit with the split launch and the default engine, whatever the
    order and blocks per SM; within the FP32 tolerance otherwise); a new
    output buffer re-captures."""
    c = case
    u0 = _direct(c, api.FP32)
    h = api.stomsfem_plan_create(c["g"], c["fld"], c["S"], api.FP32, oversample=c["ov"], max_oversample=c["mo"])
    try:
        st = torch.cuda.Stream()
        u = torch.empty((c["S"], c["nn"]), dtype=torch.float64, device=DEV)
        with torch.cuda.stream(st):
            bps, split, ms = api.stomsfem_plan_tune(h, c["xt"], u, stream=st)
            assert bps in (0, 1, 2) and split in (0, 1) and ms > 0
            info = api.stomsfem_plan_info(h)
            assert info[:2] == (bps, split)
            assert info[2] in (api.ENGINE_TC3, api.ENGINE_BLOCKED, api.ENGINE_WIDE)
            assert info[3] in (api.ORDER_CELL, api.ORDER_PATCH) and info[4] == 0
            api.stomsfem_plan_step(h, c["xt"], u, stream=st)
            u2 = torch.empty_like(u)
            api.stomsfem_plan_step(h, c["xt"], u2, stream=st)
            st.synchronize()
        for x in (u.cpu().numpy(), u2.cpu().numpy()):
            if split and info[2] == api.ENGINE_BLOCKED:
                np.testing.assert_array_equal(x, u0)
            else:
                assert np.max(np.linalg.norm(x - u0, axis=1) / np.linalg.norm(u0, axis=1)) <= 1e-5
    finally:
        api.stomsfem_plan_destroy(h)


@pytest.mark.parametrize("prec,engine,order", [
    (api.FP32, api.ENGINE_BLOCKED, api.ORDER_CELL), (api.FP32, api.ENGINE_TC3, api.ORDER_CELL),
    (api.FP32, api.ENGINE_WIDE, api.ORDER_CELL), (api.FP32, api.ENGINE_BLOCKED, api.ORDER_PATCH),
    (api.FP32, api.ENGINE_WIDE, api.ORDER_PATCH),
    (api.FP32_REFINED, api.ENGINE_BLOCKED, api.ORDER_CELL), (api.FP32_REFINED, api.ENGINE_TC3, api.ORDER_CELL),
    (api.FP32_REFINED, api.ENGINE_TC2, api.ORDER_CELL), (api.FP32_REFINED, api.ENGINE_WIDE, api.ORDER_CELL),
    (api.FP32_REFINED, api.ENGINE_WIDE, api.ORDER_PATCH),
    (api.FP64, api.ENGINE_BLOCKED, api.ORDER_PATCH)])
def test_plan_engines_match_oracle(case, orc, prec, engine, order):
    """Each factorisation engine and unit order a plan can be set to, with
    oversampled patches: the coarse solution against the FP64 oracle within
    the form's tolerance (FP32 1e-5, FP32 + two FP64 refinement sweeps
    1e-10, FP64 1e-9)."""
    c = case
    g, S = c["g"], c["S"]
    tol = {api.FP32: 1e-5, api.FP32_REFINED: 1e-10, api.FP64: 1e-9}[prec]
    h = api.stomsfem_plan_create(g, c["fld"], S, prec, oversample=c["ov"], max_oversample=c["mo"], refine_iters=2)
    try:
        api.stomsfem_plan_set_choice(h, 0, 1, engine, order)
        assert api.stomsfem_plan_info(h)[2:4] == (engine, order)
        st = torch.cuda.Stream()
        u = torch.empty((S, c["nn"]), dtype=torch.float64, device=DEV)
        with torch.cuda.stream(st):
            api.stomsfem_plan_step(h, c["xt"], u, use_graph=False, stream=st)
            st.synchronize()
    finally:
        api.stomsfem_plan_destroy(h)
    xi = c["xt"].cpu().numpy()
    fld_d = dict(W.workload("upscale_1024")["field"], nbx=4, nby=4, width=0.125)
    a = orc.sample_coef(g.nf, fld_d, xi)
    ov = c["ov"].cpu().numpy()
    Ko, bo = orc.upscale(g.nf, g.nc, 1.0, a, ov)
    uo = orc.coarse_solve(g.nc, Ko, bo)
    err = np.max(np.linalg.norm(u.cpu().numpy() - uo, axis=1) / np.linalg.norm(uo, axis=1))
    print("engine %d order %d precision %d: coarse error %.3e" % (engine, order, prec, err))
    assert err <= tol


@pytest.mark.parametrize("prec,engine,split", [(api.FP32, api.ENGINE_BLOCKED, 1), (api.FP32, api.ENGINE_BLOCKED, 0),
                                               (api.FP32, api.ENGINE_WIDE, 1), (api.FP32, api.ENGINE_TC3, 1),
                                               (api.FP32_REFINED, api.ENGINE_BLOCKED, 1),
                                               (api.FP64, api.ENGINE_BLOCKED, 1)])
def test_plan_order_and_blocks_do_not_change_results(case, prec, engine, split):
    """The unit order (cells fastest or by patch size) and the resident CTAs
    per SM only reorder independent units: the solutions agree bit for bit,
    with the flagged-cell handling included (an oversampling entry outside
    [0, max_oversample] gives NaN for its cell in either order)."""
    c = case
    g, S = c["g"], c["S"]
    ov_bad = c["ov"].clone()
    ov_bad[3] = c["mo"] + 1
    outs = []
    for order, bps in ((api.ORDER_CELL, 0), (api.ORDER_PATCH, 0), (api.ORDER_PATCH, 1)):
        h = api.stomsfem_plan_create(g, c["fld"], S, prec, oversample=c["ov"], max_oversample=c["mo"],
                                     refine_iters=2)
        try:
            api.stomsfem_plan_set_choice(h, bps, split, engine, order)
            st = torch.cuda.Stream()
            u = torch.empty((S, c["nn"]), dtype=torch.float64, device=DEV)
            with torch.cuda.stream(st):
                api.stomsfem_plan_step(h, c["xt"], u, stream=st)
                st.synchronize()
            outs.append(u.cpu().numpy())
        finally:
            api.stomsfem_plan_destroy(h)
        a = torch.empty((S, g.nf, g.nf), dtype=torch.float64, device=DEV)
        api.stomsfem_sample_coef(g, c["fld"], c["xt"], a)
        Ke = torch.empty((S, g.nc * g.nc, 10), dtype=torch.float64, device=DEV)
        be = torch.empty((S, g.nc * g.nc, 4), dtype=torch.float64, device=DEV)
        stt = torch.full((S, g.nc * g.nc), 7, dtype=torch.int32, device=DEV)
        api.stomsfem_upscale(g, a, Ke, be, oversample=ov_bad, max_oversample=c["mo"], precision=prec,
                             unit_status=stt, engine=engine, order=order)
        torch.cuda.synchronize()
        st_h = stt.cpu().numpy()
        assert np.all(st_h[:, 3] == -1) and np.all(np.delete(st_h, 3, axis=1) == 0)
        assert np.all(np.isnan(Ke.cpu().numpy()[:, 3])) and np.all(np.isfinite(np.delete(Ke.cpu().numpy(), 3, 1)))
    for x in outs[1:]:
        np.testing.assert_array_equal(x, outs[0])


def test_plan_rejects_ineligible_engine(case):
    c = case
    h = api.stomsfem_plan_create(c["g"], c["fld"], c["S"], api.FP64, oversample=c["ov"], max_oversample=c["mo"])
    try:
        for eng in (api.ENGINE_WIDE, api.ENGINE_TC3):
            with pytest.raises(Exception):
                api.stomsfem_plan_set_choice(h, 0, 1, eng)
        with pytest.raises(Exception):
            api.stomsfem_plan_set_choice(h, 0, 1, api.ENGINE_BLOCKED, 2)
    finally:
        api.stomsfem_plan_destroy(h)


def test_plan_default_stream_runs_directly(case):
    c = case
    u0 = _direct(c, api.FP64)
    h = api.stomsfem_plan_create(c["g"], c["fld"], c["S"], api.FP64, oversample=c["ov"], max_oversample=c["mo"])
    try:
        u = torch.empty((c["S"], c["nn"]), dtype=torch.float64, device=DEV)
        api.stomsfem_plan_step(h, c["xt"], u)      # the current (default) stream: no capture
        torch.cuda.synchronize()
        np.testing.assert_array_equal(u.cpu().numpy(), u0)
        assert api.stomsfem_plan_info(h)[4] == 0
    finally:
        api.stomsfem_plan_destroy(h)
