"""The allocation-free upscaling entry point, called through the C ABI.

stomsfem_upscale_noalloc serves callers that cannot allocate device memory
at the point where they upscale (its scratch is a fixed device array inside
the library).  Its results must match stomsfem_upscale, which uses a
caller-allocated workspace, within the parity tolerances of the other GPU
tests, on two calls in a row (the second call finds the first call's data
still in the shared array).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1607_00693_gb300 import _lib as L
from paper_1607_00693_gb300 import api

TOL = {api.FP64: 1e-11, api.FP32_REFINED: 1e-10, api.FP32: 1e-5}
DEV = "cuda:0"


@pytest.fixture(scope="module")
def lib():
    from paper_1607_00693_gb300.build import build_library
    build_library()
    h = L.lib()
    P, I = ctypes.c_void_p, ctypes.c_int32
    h.stomsfem_upscale_noalloc.restype = ctypes.c_int
    h.stomsfem_upscale_noalloc.argtypes = [ctypes.POINTER(L.Grid), P, P, I, I, I, I, P, P, P, P, P]
    h.stomsfem_upscale_static_scratch_bytes.restype = ctypes.c_size_t
    return h


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _inputs(seed, S, nf, nc):
    r = np.random.default_rng(seed)
    a = np.exp(r.uniform(-1.5, 1.5, size=(S, nf, nf)))
    ov = r.integers(0, 5, size=nc * nc).astype(np.int8)
    return torch.from_numpy(a).to(DEV), torch.from_numpy(ov).to(DEV), int(ov.max())


def _run_noalloc(lib, g, a, ov, mo, prec):
    """The entry point through ctypes (a, ov device tensors or ov None)."""
    S = a.shape[0]
    nc2 = g.nc * g.nc
    Ke = torch.full((S, nc2, 10), float("nan"), dtype=torch.float64, device=DEV)
    be = torch.full((S, nc2, 4), float("nan"), dtype=torch.float64, device=DEV)
    st = torch.full((S, nc2), 7, dtype=torch.int32, device=DEV)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.stomsfem_upscale_noalloc(ctypes.byref(g), _p(a), _p(ov), mo, S, prec, 2, _p(Ke), _p(be),
                                      None, _p(st), stream)
    assert rc == 0, lib.stomsfem_last_error()
    torch.cuda.synchronize()
    return Ke.cpu().numpy(), be.cpu().numpy(), st.cpu().numpy()


def _run_workspace(g, a, ov, mo, prec):
    S = a.shape[0]
    nc2 = g.nc * g.nc
    Ke = torch.empty((S, nc2, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((S, nc2, 4), dtype=torch.float64, device=DEV)
    api.stomsfem_upscale(g, a, Ke, be, oversample=ov, max_oversample=mo, precision=prec,
                         refine_iters=2)
    torch.cuda.synchronize()
    return Ke.cpu().numpy(), be.cpu().numpy()


def _rel(x, y):
    return float(np.max(np.linalg.norm(x - y, axis=-1) / np.linalg.norm(y, axis=-1)))


def test_noalloc_matches_workspace_path_twice(lib):
    """Three calls in a row (FP32, FP64, FP32 + refinement) on H/h = 32
    patches with oversampling 0..4: each matches the workspace path."""
    nf, nc = 128, 4     # H/h = 32, oversampling 0..4
    g = api.grid(nf, nc, 1.0)
    for call, (seed, S, prec) in enumerate([(11, 6, api.FP32), (12, 3, api.FP64), (13, 4, api.FP32_REFINED)]):
        a, ov, mo = _inputs(seed, S, nf, nc)
        Kn, bn, st = _run_noalloc(lib, g, a, ov, mo, prec)
        Kw, bw = _run_workspace(g, a, ov, mo, prec)
        assert np.all(st == 0), call
        assert _rel(Kn, Kw) <= TOL[prec], call
        assert _rel(bn, bw) <= TOL[prec], call


def test_noalloc_fewest_slots(lib):
    """The largest patch the upscaler accepts (half bandwidth 64: H/h = 64
    without oversampling) leaves the fewest slots in the fixed array (24 in
    FP64: six blocks of 4; 45 in FP32: five blocks of 8, the two-units-per-
    warp engine serving this bandwidth): the static path then runs the
    fewest units in flight and still matches the workspace path."""
    g = api.grid(128, 2, 1.0)
    for seed, prec, most in ((21, api.FP64, 32), (22, api.FP32, 64)):
        r = np.random.default_rng(seed)
        a = torch.from_numpy(np.exp(r.uniform(-1.0, 1.0, size=(3, 128, 128)))).to(DEV)
        slot, _ = api.stomsfem_upscale_workspace_size(g, 0, prec)
        assert (64 << 20) // slot < most
        Kn, bn, st = _run_noalloc(lib, g, a, None, 0, prec)
        Kw, bw = _run_workspace(g, a, None, 0, prec)
        assert np.all(st == 0)
        assert _rel(Kn, Kw) <= TOL[prec]
        assert _rel(bn, bw) <= TOL[prec]


def test_noalloc_rejects_oversized_patch(lib):
    """H/h = 128: the slots of one block (4 in FP64, 8 in the FP32 forms)
    exceed the fixed array; the call is refused on the host (real but small
    device buffers are passed, and nothing is launched)."""
    g = api.grid(256, 2, 1.0)
    assert lib.stomsfem_upscale_static_scratch_bytes() == 64 << 20
    a = torch.zeros((1, 256, 256), dtype=torch.float64, device=DEV)
    Ke = torch.zeros((1, 4, 10), dtype=torch.float64, device=DEV)
    be = torch.zeros((1, 4, 4), dtype=torch.float64, device=DEV)
    for prec in (api.FP64, api.FP32, api.FP32_REFINED):
        rc = lib.stomsfem_upscale_noalloc(ctypes.byref(g), _p(a), None, 0, 1, prec, 0, _p(Ke), _p(be), None,
                                          None, None)
        assert rc == L.EINVAL, prec
        assert b"static scratch" in lib.stomsfem_last_error()
    torch.cuda.synchronize()
    assert float(Ke.abs().sum()) == 0.0 and float(be.abs().sum()) == 0.0
    assert lib.stomsfem_upscale(ctypes.byref(g), None, None, 0, 0, 0, 0, None, None, None, None,
                                None, 0, None) == L.OK
    assert lib.stomsfem_upscale(ctypes.byref(g), None, None, 0, 1, 5, 0, None, None, None, None,
                                None, 0, None) == L.EINVAL
    assert lib.stomsfem_upscale(ctypes.byref(g), None, None, 0, 1, 0, 0, None, None, None, None,
                                None, 0, None) == L.EINVAL
    fld = L.Field(7, 4, 4, 0.1, 1.0, 0.0, 1.0)
    assert lib.stomsfem_sample_coef(ctypes.byref(g), ctypes.byref(fld), None, 1, None, None) == L.EINVAL
    cb = ctypes.c_size_t()
    assert lib.stomsfem_coarse_workspace_size(ctypes.byref(g), 64, ctypes.byref(cb)) == L.OK
    assert lib.stomsfem_coarse_solve(ctypes.byref(g), None, None, 3, None, None, None, None, None, 0,
                                     None) == L.EINVAL
