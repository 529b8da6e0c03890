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
    nf, nc = 128, 4     # H/h = 32, oversampling 0..4
    g = api.grid(nf, nc, 1.0)
    for call, (seed, S, prec) in enumerate([(11, 6, api.FP32), (12, 3, api.FP64)]):
        a, ov, mo = _inputs(seed, S, nf, nc)
        Kn, bn, st = _run_noalloc(lib, g, a, ov, mo, prec)
        Kw, bw = _run_workspace(g, a, ov, mo, prec)
        assert np.all(st == 0), call
        assert _rel(Kn, Kw) <= TOL[prec], call
        assert _rel(bn, bw) <= TOL[prec], call


def test_noalloc_rejects_oversized_patch(lib):
    # H/h = 128: four warp slots of this patch exceed the fixed array
    g = api.grid(256, 2, 1.0)
    assert lib.stomsfem_upscale_static_scratch_bytes() == 64 << 20
    rc = lib.stomsfem_upscale_noalloc(ctypes.byref(g), ctypes.c_void_p(256), None, 0, 1, api.FP64, 0,
                                      ctypes.c_void_p(256), ctypes.c_void_p(256), None, None, None)
    assert rc == L.EINVAL
    assert b"static scratch" in lib.stomsfem_last_error()
