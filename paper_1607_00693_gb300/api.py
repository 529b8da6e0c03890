"""Python binding of the C ABI, one function per entry point, same names.

Only argument marshalling happens here: shapes, dtypes and devices of the
torch tensors are checked, raw device pointers and the current CUDA
stream are passed to the library, and its status is turned into an
exception.  Every step of the method runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L
from ._lib import FP32, FP32_REFINED, FP64, FIELD_AFFINE, FIELD_EXP, FIELD_EXP_SIGMOID, Grid, Field  # noqa: F401


def _dev(t, dtype, shape=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def grid(nf, nc, f=1.0):
    return Grid(int(nf), int(nc), float(f))


def field(kind, nbx, nby, width, scale=1.0, contrast_log=0.0, gain=1.0):
    return Field(int(kind), int(nbx), int(nby), float(width), float(scale), float(contrast_log),
                 float(gain))


def field_from_dict(d):
    return field(d["kind"], d["nbx"], d["nby"], d["width"], d.get("scale", 1.0),
                 d.get("contrast_log", 0.0), d.get("gain", 1.0))


def stomsfem_version():
    return L.lib().stomsfem_version().decode()


def stomsfem_selftest_wait_timeout(iters=20000):
    """Run the bounded-wait self test; returns the device status word
    (STOMSFEM_ETIMEOUT when the wait ran out as it should)."""
    st = ctypes.c_int32(1)
    L.check(L.lib().stomsfem_selftest_wait_timeout(int(iters), ctypes.byref(st)))
    return st.value


def stomsfem_selftest_exp(t, out=None, stream=None):
    """exp of a float64 device tensor by the sampler's table-driven routine."""
    if out is None:
        out = torch.empty_like(t)
    L.check(L.lib().stomsfem_selftest_exp(_dev(t, torch.float64, None, "t"), t.numel(),
                                          _dev(out, torch.float64, tuple(t.shape), "out"), _stream(stream)))
    return out


def stomsfem_selftest_fma_rate(precision=FP32):
    """Measured FMA-pipe peak in TFLOP/s (FP32 or FP64)."""
    v = ctypes.c_float()
    L.check(L.lib().stomsfem_selftest_fma_rate(int(precision), ctypes.byref(v)))
    return v.value


def stomsfem_selftest_mma_rate(kind=0):
    """Measured mma.sync throughput in TFLOP/s (0: TF32 m16n8k8, 1: BF16 m16n8k16)."""
    v = ctypes.c_float()
    L.check(L.lib().stomsfem_selftest_mma_rate(int(kind), ctypes.byref(v)))
    return v.value


def stomsfem_sample_coef(g: Grid, fld: Field, xi, a, stream=None):
    S = xi.shape[0]
    L.check(L.lib().stomsfem_sample_coef(ctypes.byref(g), ctypes.byref(fld),
                                         _dev(xi, torch.float64, (S, fld.nbx * fld.nby), "xi"), S,
                                         _dev(a, torch.float64, (S, g.nf, g.nf), "a"), _stream(stream)))


def stomsfem_sample_coef_precision(g: Grid, fld: Field, xi, a, precision=FP64, stream=None):
    S = xi.shape[0]
    L.check(L.lib().stomsfem_sample_coef_precision(
        ctypes.byref(g), ctypes.byref(fld), _dev(xi, torch.float64, (S, fld.nbx * fld.nby), "xi"), S,
        int(precision), _dev(a, torch.float64, (S, g.nf, g.nf), "a"), _stream(stream)))


def stomsfem_upscale_workspace_size(g: Grid, max_oversample=0, precision=FP64):
    sb, rb = ctypes.c_size_t(), ctypes.c_size_t()
    L.check(L.lib().stomsfem_upscale_workspace_size(ctypes.byref(g), int(max_oversample),
                                                    int(precision), ctypes.byref(sb), ctypes.byref(rb)))
    return sb.value, rb.value


def stomsfem_upscale(g: Grid, a, Ke, be, oversample=None, max_oversample=0, precision=FP64,
                     refine_iters=2, phi=None, unit_status=None, workspace=None, stream=None, engine=None,
                     order=None):
    """engine and order None: stomsfem_upscale (the default engine, cell
    order); otherwise stomsfem_upscale_engine with those STOMSFEM_ENGINE_*
    and STOMSFEM_ORDER_* values (None: AUTO, CELL)."""
    S = a.shape[0]
    ncell = g.nc * g.nc
    rho = g.nf // g.nc
    if workspace is None:
        _, rb = stomsfem_upscale_workspace_size(g, max_oversample if oversample is not None else 0,
                                                precision)
        workspace = torch.empty(rb, dtype=torch.uint8, device=a.device)
    head = (ctypes.byref(g), _dev(a, torch.float64, (S, g.nf, g.nf), "a"),
            _dev(oversample, torch.int8, (ncell,), "oversample"), int(max_oversample), S, int(precision),
            int(refine_iters))
    tail = (_dev(Ke, torch.float64, (S, ncell, 10), "Ke"), _dev(be, torch.float64, (S, ncell, 4), "be"),
            _dev(phi, torch.float64, (S, ncell, 4, (rho + 1) ** 2), "phi"),
            _dev(unit_status, torch.int32, (S, ncell), "unit_status"),
            _dev(workspace, torch.uint8, None, "workspace"), workspace.numel(), _stream(stream))
    if engine is None and order is None:
        L.check(L.lib().stomsfem_upscale(*head, *tail))
    else:
        L.check(L.lib().stomsfem_upscale_engine(*head, int(engine or ENGINE_AUTO), int(order or ORDER_CELL),
                                                *tail))


def stomsfem_coarse_workspace_size(g: Grid, S):
    b = ctypes.c_size_t()
    L.check(L.lib().stomsfem_coarse_workspace_size(ctypes.byref(g), int(S), ctypes.byref(b)))
    return b.value


def stomsfem_coarse_solve(g: Grid, Ke, be, u, mean=None, m2=None, count=None, workspace=None,
                          stream=None):
    S = Ke.shape[0]
    ncell = g.nc * g.nc
    nn = (g.nc + 1) ** 2
    if workspace is None:
        workspace = torch.empty(stomsfem_coarse_workspace_size(g, S), dtype=torch.uint8,
                                device=Ke.device)
    L.check(L.lib().stomsfem_coarse_solve(
        ctypes.byref(g), _dev(Ke, torch.float64, (S, ncell, 10), "Ke"),
        _dev(be, torch.float64, (S, ncell, 4), "be"), S, _dev(u, torch.float64, (S, nn), "u"),
        _dev(mean, torch.float64, (nn,), "mean"), _dev(m2, torch.float64, (nn,), "m2"),
        _dev(count, torch.float64, (1,), "count"), _dev(workspace, torch.uint8, None, "workspace"),
        workspace.numel(), _stream(stream)))


def stomsfem_pod_build(g: Grid, phi_snap, a_train, tol=1e-6, max_rank=27, ranks=None, stream=None):
    """Returns (handle, ranks list)."""
    S = a_train.shape[0]
    ncell = g.nc * g.nc
    rho = g.nf // g.nc
    h = ctypes.c_void_p()
    rk = (ctypes.c_int32 * ncell)()
    rin = None
    if ranks is not None:
        rin = (ctypes.c_int32 * ncell)(*[int(x) for x in ranks])
    L.check(L.lib().stomsfem_pod_build(
        ctypes.byref(g), _dev(phi_snap, torch.float64, (S, ncell, 4, (rho + 1) ** 2), "phi_snap"),
        _dev(a_train, torch.float64, (S, g.nf, g.nf), "a_train"), S, float(tol), int(max_rank),
        ctypes.cast(rin, ctypes.c_void_p) if rin is not None else None, ctypes.byref(h),
        ctypes.cast(rk, ctypes.c_void_p), _stream(stream)))
    return h, list(rk)


def stomsfem_pod_build_per_l(g: Grid, phi_snap, a_train, tol=1e-6, max_rank_per_l=9, ranks=None, stream=None):
    """One basis per basis function: returns (handle, ranks [nc*nc][3] list)."""
    S = a_train.shape[0]
    ncell = g.nc * g.nc
    rho = g.nf // g.nc
    h = ctypes.c_void_p()
    rk = (ctypes.c_int32 * (3 * ncell))()
    rin = None
    if ranks is not None:
        flat = [int(x) for row in ranks for x in row]
        rin = (ctypes.c_int32 * (3 * ncell))(*flat)
    L.check(L.lib().stomsfem_pod_build_per_l(
        ctypes.byref(g), _dev(phi_snap, torch.float64, (S, ncell, 4, (rho + 1) ** 2), "phi_snap"),
        _dev(a_train, torch.float64, (S, g.nf, g.nf), "a_train"), S, float(tol), int(max_rank_per_l),
        ctypes.cast(rin, ctypes.c_void_p) if rin is not None else None, ctypes.byref(h),
        ctypes.cast(rk, ctypes.c_void_p), _stream(stream)))
    return h, [list(rk[3 * c:3 * c + 3]) for c in range(ncell)]


def stomsfem_build_pod(g: Grid, phi_snap, a_train, tol=1e-6, max_rank=27, ranks=None, stream=None):
    """The POD offline step under its method name: as stomsfem_pod_build."""
    return stomsfem_pod_build(g, phi_snap, a_train, tol, max_rank, ranks, stream)


def stomsfem_pod_destroy(h):
    L.check(L.lib().stomsfem_pod_destroy(h))


def stomsfem_pod_eigenvalues(h, g: Grid, per_l=False):
    """[nc*nc][n] (per-l handles: [nc*nc][3][n]) KL eigenvalues, descending."""
    import numpy as np
    rho = g.nf // g.nc
    lam = np.empty((g.nc * g.nc, 3, (rho - 1) ** 2) if per_l else (g.nc * g.nc, (rho - 1) ** 2))
    L.check(L.lib().stomsfem_pod_eigenvalues(h, lam.ctypes.data_as(ctypes.c_void_p)))
    return lam


def stomsfem_surrogate_set_partner(h, partner, tol):
    """partner None removes the ensemble partner."""
    L.check(L.lib().stomsfem_surrogate_set_partner(h, partner, float(tol)))


def stomsfem_pod_set_gemm_split(h, split=1):
    L.check(L.lib().stomsfem_pod_set_gemm_split(h, int(split)))


def stomsfem_pod_workspace_size(h, S):
    b = ctypes.c_size_t()
    L.check(L.lib().stomsfem_pod_workspace_size(h, int(S), ctypes.byref(b)))
    return b.value


def stomsfem_pod_upscale(h, g: Grid, a, Ke, be, refine_iters=0, unit_status=None, workspace=None,
                         stream=None):
    S = a.shape[0]
    ncell = g.nc * g.nc
    if workspace is None:
        workspace = torch.empty(stomsfem_pod_workspace_size(h, S), dtype=torch.uint8, device=a.device)
    L.check(L.lib().stomsfem_pod_upscale(
        h, _dev(a, torch.float64, (S, g.nf, g.nf), "a"), S, int(refine_iters),
        _dev(Ke, torch.float64, (S, ncell, 10), "Ke"), _dev(be, torch.float64, (S, ncell, 4), "be"),
        _dev(unit_status, torch.int32, (S, ncell), "unit_status"),
        _dev(workspace, torch.uint8, None, "workspace"), workspace.numel(), _stream(stream)))


# ---------------------------------------------------------------- surrogate

SURROGATE_PARAMS = 37264
SURROGATE_IN = 16


def stomsfem_local_vars(g: Grid, fld: Field, tau):
    """(k [ncell], var_ids [ncell][16], family [ncell], n_families) -- host."""
    import numpy as np
    ncell = g.nc * g.nc
    k = np.zeros(ncell, dtype=np.int32)
    ids = np.zeros((ncell, SURROGATE_IN), dtype=np.int32)
    fam = np.zeros(ncell, dtype=np.int32)
    nf = ctypes.c_int32()
    L.check(L.lib().stomsfem_local_vars(ctypes.byref(g), ctypes.byref(fld), float(tau),
                                        k.ctypes.data_as(ctypes.c_void_p),
                                        ids.ctypes.data_as(ctypes.c_void_p),
                                        fam.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nf)))
    return k, ids, fam, nf.value


def xavier_weights(n_families, seed):
    """Seeded Xavier-uniform initial weights in the flat [out][in] layout
    (biases zero), drawn by the library (stomsfem_surrogate_init_weights)."""
    import numpy as np
    out = np.empty((n_families, SURROGATE_PARAMS), dtype=np.float32)
    L.check(L.lib().stomsfem_surrogate_init_weights(int(n_families), int(seed) & ((1 << 64) - 1),
                                                    out.ctypes.data_as(ctypes.c_void_p)))
    return out


def _save(fn, h):
    n = ctypes.c_size_t()
    L.check(fn(h, None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    L.check(fn(h, buf, n.value, ctypes.byref(n)))
    return buf.raw[:n.value]


def stomsfem_pod_save(h):
    """Serialised offline stage as bytes."""
    return _save(L.lib().stomsfem_pod_save, h)


def stomsfem_pod_load(data: bytes):
    h = ctypes.c_void_p()
    L.check(L.lib().stomsfem_pod_load(data, len(data), ctypes.byref(h)))
    return h


def stomsfem_surrogate_save(h):
    """Serialised surrogate (weights, Adam state, step, input box) as bytes."""
    return _save(L.lib().stomsfem_surrogate_save, h)


def stomsfem_surrogate_load(data: bytes):
    h = ctypes.c_void_p()
    nfam = ctypes.c_int32()
    L.check(L.lib().stomsfem_surrogate_load(data, len(data), ctypes.byref(h), ctypes.byref(nfam)))
    return h, nfam.value


def stomsfem_surrogate_create(g: Grid, fld: Field, tau, init_weights):
    import numpy as np
    w = np.ascontiguousarray(init_weights, dtype=np.float32)
    h = ctypes.c_void_p()
    nfam = ctypes.c_int32()
    L.check(L.lib().stomsfem_surrogate_create(ctypes.byref(g), ctypes.byref(fld), float(tau),
                                              w.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h),
                                              ctypes.byref(nfam)))
    return h, nfam.value


def stomsfem_surrogate_destroy(h):
    L.check(L.lib().stomsfem_surrogate_destroy(h))


def stomsfem_surrogate_weights(h, n_families):
    import numpy as np
    w = np.empty((n_families, SURROGATE_PARAMS), dtype=np.float32)
    L.check(L.lib().stomsfem_surrogate_weights(h, w.ctypes.data_as(ctypes.c_void_p)))
    return w


def stomsfem_surrogate_train(h, xi, a, Ke, be, steps, lr=1e-3, lr_min=1e-5, seed=0, beta1=0.9,
                             beta2=0.999, eps=1e-8, fp32_products=False, stream=None):
    """Returns the per-step training loss (family mean) as a numpy array."""
    import numpy as np
    S = xi.shape[0]
    cfg = L.SurrogateCfg(int(steps), float(lr), float(lr_min), float(beta1), float(beta2), float(eps),
                         int(seed), int(bool(fp32_products)))
    loss = np.empty(int(steps), dtype=np.float32)
    L.check(L.lib().stomsfem_surrogate_train(
        h, ctypes.byref(cfg), _dev(xi, torch.float64, None, "xi"), _dev(a, torch.float64, None, "a"),
        _dev(Ke, torch.float64, None, "Ke"), _dev(be, torch.float64, None, "be"), S,
        loss.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return loss


def stomsfem_surrogate_grad(weights, X, T, grad, loss=None, fp32_products=False, stream=None):
    L.check(L.lib().stomsfem_surrogate_grad(
        _dev(weights, torch.float32, (SURROGATE_PARAMS,), "weights"),
        _dev(X, torch.float32, (64, 16), "X"), _dev(T, torch.float32, (64, 16), "T"),
        int(bool(fp32_products)),
        _dev(grad, torch.float32, (SURROGATE_PARAMS,), "grad"), _dev(loss, torch.float32, (1,), "loss"),
        _stream(stream)))


def stomsfem_surrogate_workspace_size(h, S):
    b = ctypes.c_size_t()
    L.check(L.lib().stomsfem_surrogate_workspace_size(h, int(S), ctypes.byref(b)))
    return b.value


def stomsfem_surrogate_infer(h, g: Grid, xi, a, Ke, be, fell_back, delta=0.02, workspace=None,
                             stream=None):
    S = xi.shape[0]
    ncell = g.nc * g.nc
    if workspace is None:
        workspace = torch.empty(stomsfem_surrogate_workspace_size(h, S), dtype=torch.uint8,
                                device=xi.device)
    L.check(L.lib().stomsfem_surrogate_infer(
        h, _dev(xi, torch.float64, None, "xi"), _dev(a, torch.float64, (S, g.nf, g.nf), "a"), S,
        float(delta), _dev(Ke, torch.float64, (S, ncell, 10), "Ke"),
        _dev(be, torch.float64, (S, ncell, 4), "be"), _dev(fell_back, torch.uint8, (S, ncell), "fell_back"),
        _dev(workspace, torch.uint8, None, "workspace"), workspace.numel(), _stream(stream)))


RI_CHEBYSHEV, RI_LEGENDRE = 0, 1
RI_MAX_DIM = 16


def stomsfem_ri_plan(g: Grid, fld: Field, eps, nu_max=8):
    """(family [ncell], var_ids [ncell][16], nu [ncell][16], n_families,
    n_points) -- host."""
    import numpy as np
    ncell = g.nc * g.nc
    fam = np.zeros(ncell, dtype=np.int32)
    ids = np.zeros((ncell, RI_MAX_DIM), dtype=np.int32)
    nu = np.zeros((ncell, RI_MAX_DIM), dtype=np.int32)
    nfam = ctypes.c_int32()
    npts = ctypes.c_int64()
    L.check(L.lib().stomsfem_ri_plan(ctypes.byref(g), ctypes.byref(fld), float(eps), int(nu_max),
                                     fam.ctypes.data_as(ctypes.c_void_p), ids.ctypes.data_as(ctypes.c_void_p),
                                     nu.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nfam),
                                     ctypes.byref(npts)))
    return fam, ids, nu, nfam.value, npts.value


def stomsfem_ri_build(g: Grid, fld: Field, eps, nu_max=8, nodes=RI_CHEBYSHEV, stream=None):
    h = ctypes.c_void_p()
    nfam = ctypes.c_int32()
    L.check(L.lib().stomsfem_ri_build(ctypes.byref(g), ctypes.byref(fld), float(eps), int(nu_max), int(nodes),
                                      ctypes.byref(h), ctypes.byref(nfam), _stream(stream)))
    return h, nfam.value


def stomsfem_ri_destroy(h):
    L.check(L.lib().stomsfem_ri_destroy(h))


def stomsfem_ri_values(h, n_points):
    import numpy as np
    V = np.zeros((int(n_points), 14))
    L.check(L.lib().stomsfem_ri_values(h, V.ctypes.data_as(ctypes.c_void_p), int(n_points)))
    return V


def stomsfem_ri_workspace_size(h, S):
    b = ctypes.c_size_t()
    L.check(L.lib().stomsfem_ri_workspace_size(h, int(S), ctypes.byref(b)))
    return b.value


def stomsfem_ri_upscale(h, g: Grid, xi, a, Ke, be, fell_back, workspace=None, stream=None):
    """a may be None (units outside the collocation box then get NaN and
    fell_back = 2)."""
    S = xi.shape[0]
    ncell = g.nc * g.nc
    if workspace is None:
        workspace = torch.empty(stomsfem_ri_workspace_size(h, S), dtype=torch.uint8, device=xi.device)
    L.check(L.lib().stomsfem_ri_upscale(
        h, _dev(xi, torch.float64, None, "xi"),
        _dev(a, torch.float64, (S, g.nf, g.nf), "a") if a is not None else None, S,
        _dev(Ke, torch.float64, (S, ncell, 10), "Ke"), _dev(be, torch.float64, (S, ncell, 4), "be"),
        _dev(fell_back, torch.uint8, (S, ncell), "fell_back"),
        _dev(workspace, torch.uint8, None, "workspace"), workspace.numel(), _stream(stream)))


def stomsfem_upscale_pg(g: Grid, a, Ke, be, oversample=None, max_oversample=0, precision=FP64,
                        refine_iters=2, phi=None, unit_status=None, workspace=None, stream=None):
    """Petrov-Galerkin form: Ke [S][ncell][16] (row trial, column test)."""
    S = a.shape[0]
    ncell = g.nc * g.nc
    rho = g.nf // g.nc
    if workspace is None:
        _, rb = stomsfem_upscale_workspace_size(g, max_oversample if oversample is not None else 0,
                                                precision)
        workspace = torch.empty(rb, dtype=torch.uint8, device=a.device)
    L.check(L.lib().stomsfem_upscale_pg(
        ctypes.byref(g), _dev(a, torch.float64, (S, g.nf, g.nf), "a"),
        _dev(oversample, torch.int8, (ncell,), "oversample"), int(max_oversample), S, int(precision),
        int(refine_iters), _dev(Ke, torch.float64, (S, ncell, 16), "Ke"),
        _dev(be, torch.float64, (S, ncell, 4), "be"),
        _dev(phi, torch.float64, (S, ncell, 4, (rho + 1) ** 2), "phi"),
        _dev(unit_status, torch.int32, (S, ncell), "unit_status"),
        _dev(workspace, torch.uint8, None, "workspace"), workspace.numel(), _stream(stream)))


BC_BILINEAR, BC_OSCILLATORY = 0, 1


def stomsfem_upscale_bc(g: Grid, pg, bc, a, Ke, be, oversample=None, max_oversample=0, precision=FP64,
                        refine_iters=2, phi=None, unit_status=None, workspace=None, stream=None):
    """Upscaling with the cell problems' boundary data ``bc`` (BC_BILINEAR or
    BC_OSCILLATORY), Galerkin (Ke [S][ncell][10]) or with ``pg``
    Petrov-Galerkin (Ke [S][ncell][16])."""
    S = a.shape[0]
    ncell = g.nc * g.nc
    rho = g.nf // g.nc
    if workspace is None:
        _, rb = stomsfem_upscale_workspace_size(g, max_oversample if oversample is not None else 0,
                                                precision)
        workspace = torch.empty(rb, dtype=torch.uint8, device=a.device)
    L.check(L.lib().stomsfem_upscale_bc(
        ctypes.byref(g), int(bool(pg)), int(bc), _dev(a, torch.float64, (S, g.nf, g.nf), "a"),
        _dev(oversample, torch.int8, (ncell,), "oversample"), int(max_oversample), S, int(precision),
        int(refine_iters), _dev(Ke, torch.float64, (S, ncell, 16 if pg else 10), "Ke"),
        _dev(be, torch.float64, (S, ncell, 4), "be"),
        _dev(phi, torch.float64, (S, ncell, 4, (rho + 1) ** 2), "phi"),
        _dev(unit_status, torch.int32, (S, ncell), "unit_status"),
        _dev(workspace, torch.uint8, None, "workspace"), workspace.numel(), _stream(stream)))


def stomsfem_coarse_pg_workspace_size(g: Grid, S):
    b = ctypes.c_size_t()
    L.check(L.lib().stomsfem_coarse_pg_workspace_size(ctypes.byref(g), int(S), ctypes.byref(b)))
    return b.value


def stomsfem_coarse_solve_pg(g: Grid, Ke, be, u, mean=None, m2=None, count=None, workspace=None,
                             stream=None):
    S = Ke.shape[0]
    ncell = g.nc * g.nc
    nn = (g.nc + 1) ** 2
    if workspace is None:
        workspace = torch.empty(stomsfem_coarse_pg_workspace_size(g, S), dtype=torch.uint8,
                                device=Ke.device)
    L.check(L.lib().stomsfem_coarse_solve_pg(
        ctypes.byref(g), _dev(Ke, torch.float64, (S, ncell, 16), "Ke"),
        _dev(be, torch.float64, (S, ncell, 4), "be"), S, _dev(u, torch.float64, (S, nn), "u"),
        _dev(mean, torch.float64, (nn,), "mean"), _dev(m2, torch.float64, (nn,), "m2"),
        _dev(count, torch.float64, (1,), "count"), _dev(workspace, torch.uint8, None, "workspace"),
        workspace.numel(), _stream(stream)))


def stomsfem_coarse_bc_workspace_size(g: Grid, pg, S):
    b = ctypes.c_size_t()
    L.check(L.lib().stomsfem_coarse_bc_workspace_size(ctypes.byref(g), int(bool(pg)), int(S), ctypes.byref(b)))
    return b.value


def stomsfem_coarse_solve_bc(g: Grid, pg, K, b, dirichlet, gval, u, mean=None, m2=None, count=None,
                             workspace=None, stream=None):
    """Mixed boundary data: u = gval where ``dirichlet`` (uint8
    [(nc+1)^2]) is nonzero, zero flux on the rest of the boundary; ``pg``
    selects the Petrov-Galerkin system (K [S][nc*nc][16])."""
    S = K.shape[0]
    ncell = g.nc * g.nc
    nn = (g.nc + 1) ** 2
    if workspace is None:
        workspace = torch.empty(stomsfem_coarse_bc_workspace_size(g, pg, S), dtype=torch.uint8, device=K.device)
    L.check(L.lib().stomsfem_coarse_solve_bc(
        ctypes.byref(g), int(bool(pg)), _dev(K, torch.float64, (S, ncell, 16 if pg else 10), "K"),
        _dev(b, torch.float64, (S, ncell, 4), "b"), _dev(dirichlet, torch.uint8, (nn,), "dirichlet"),
        _dev(gval, torch.float64, (nn,), "g"), S, _dev(u, torch.float64, (S, nn), "u"),
        _dev(mean, torch.float64, (nn,), "mean"), _dev(m2, torch.float64, (nn,), "m2"),
        _dev(count, torch.float64, (1,), "count"), _dev(workspace, torch.uint8, None, "workspace"),
        workspace.numel(), _stream(stream)))


def stomsfem_pod_set_affine(h, g: Grid, fld: Field, tau=1e-6, stream=None):
    L.check(L.lib().stomsfem_pod_set_affine(h, ctypes.byref(g), ctypes.byref(fld), float(tau), _stream(stream)))


def stomsfem_pod_upscale_affine(h, g: Grid, xi, Ke, be, a=None, refine_iters=0, unit_status=None, stream=None):
    S = xi.shape[0]
    ncell = g.nc * g.nc
    L.check(L.lib().stomsfem_pod_upscale_affine(
        h, _dev(xi, torch.float64, None, "xi"),
        _dev(a, torch.float64, (S, g.nf, g.nf), "a") if a is not None else None, S, int(refine_iters),
        _dev(Ke, torch.float64, (S, ncell, 10), "Ke"), _dev(be, torch.float64, (S, ncell, 4), "be"),
        _dev(unit_status, torch.int32, (S, ncell), "unit_status"), _stream(stream)))


def stomsfem_fine_fem_workspace_size(g: Grid, S):
    b = ctypes.c_size_t()
    L.check(L.lib().stomsfem_fine_fem_workspace_size(ctypes.byref(g), int(S), ctypes.byref(b)))
    return b.value


def stomsfem_fine_fem(g: Grid, a, u, workspace=None, stream=None):
    S = a.shape[0]
    if workspace is None:
        workspace = torch.empty(stomsfem_fine_fem_workspace_size(g, S), dtype=torch.uint8, device=a.device)
    L.check(L.lib().stomsfem_fine_fem(
        ctypes.byref(g), _dev(a, torch.float64, (S, g.nf, g.nf), "a"), S,
        _dev(u, torch.float64, (S, (g.nf + 1) ** 2), "u"), _dev(workspace, torch.uint8, None, "workspace"),
        workspace.numel(), _stream(stream)))


def stomsfem_restrict_to_coarse(g: Grid, u_fine, d, u_coarse=None, stream=None):
    S = u_fine.shape[0]
    nn = (g.nc + 1) ** 2
    L.check(L.lib().stomsfem_restrict_to_coarse(
        ctypes.byref(g), _dev(u_fine, torch.float64, (S, (g.nf + 1) ** 2), "u_fine"),
        _dev(u_coarse, torch.float64, (S, nn), "u_coarse") if u_coarse is not None else None, S,
        _dev(d, torch.float64, (S, nn), "d"), _stream(stream)))


def stomsfem_mc_moments(u, mean, m2, count, stream=None):
    S, n = u.shape
    L.check(L.lib().stomsfem_mc_moments(
        int(n), int(S), _dev(u, torch.float64, (S, n), "u"), _dev(mean, torch.float64, (n,), "mean"),
        _dev(m2, torch.float64, (n,), "m2"), _dev(count, torch.float64, (1,), "count"), _stream(stream)))


def stomsfem_mc_merge(mean, m2, count, mean_b, m2_b, count_b, stream=None):
    """Merges the moments (mean_b, m2_b, count_b) into (mean, m2, count) in place."""
    n = mean.shape[0]
    L.check(L.lib().stomsfem_mc_merge(
        int(n), _dev(mean, torch.float64, (n,), "mean"), _dev(m2, torch.float64, (n,), "m2"),
        _dev(count, torch.float64, (1,), "count"), _dev(mean_b, torch.float64, (n,), "mean_b"),
        _dev(m2_b, torch.float64, (n,), "m2_b"), _dev(count_b, torch.float64, (1,), "count_b"), _stream(stream)))


def stomsfem_plan_create(g: Grid, fld: Field, S, precision=FP64, oversample=None, max_oversample=0,
                         refine_iters=2):
    h = ctypes.c_void_p()
    ncell = g.nc * g.nc
    L.check(L.lib().stomsfem_plan_create(ctypes.byref(g), ctypes.byref(fld),
                                         _dev(oversample, torch.int8, (ncell,), "oversample"),
                                         int(max_oversample), int(S), int(precision), int(refine_iters),
                                         ctypes.byref(h)))
    return h


def stomsfem_plan_destroy(h):
    L.check(L.lib().stomsfem_plan_destroy(h))


def stomsfem_plan_tune(h, xi, u, stream=None):
    """-> (blocks_per_sm, split_fp32, ms per step)."""
    b, sp, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    L.check(L.lib().stomsfem_plan_tune(h, _dev(xi, torch.float64, None, "xi"), _dev(u, torch.float64, None, "u"),
                                       ctypes.byref(b), ctypes.byref(sp), ctypes.byref(ms), _stream(stream)))
    return b.value, sp.value, ms.value


def stomsfem_plan_step(h, xi, u, mean=None, m2=None, count=None, use_graph=True, stream=None):
    L.check(L.lib().stomsfem_plan_step(h, _dev(xi, torch.float64, None, "xi"), _dev(u, torch.float64, None, "u"),
                                       _dev(mean, torch.float64, None, "mean"), _dev(m2, torch.float64, None, "m2"),
                                       _dev(count, torch.float64, (1,), "count"), 1 if use_graph else 0,
                                       _stream(stream)))


ENGINE_AUTO, ENGINE_BLOCKED, ENGINE_TC3, ENGINE_TC2, ENGINE_WIDE = 0, 1, 2, 3, 4
ORDER_CELL, ORDER_PATCH = 0, 1


def stomsfem_plan_set_choice(h, blocks_per_sm=0, split_fp32=1, engine=ENGINE_AUTO, order=ORDER_CELL):
    L.check(L.lib().stomsfem_plan_set_choice(h, int(blocks_per_sm), int(split_fp32), int(engine), int(order)))


def stomsfem_plan_info(h):
    """-> (blocks_per_sm, split_fp32, engine, order, graph_ready, device_bytes)."""
    b, sp, en, od, gr = (ctypes.c_int32() for _ in range(5))
    nb = ctypes.c_size_t()
    L.check(L.lib().stomsfem_plan_info(h, ctypes.byref(b), ctypes.byref(sp), ctypes.byref(en), ctypes.byref(od),
                                       ctypes.byref(gr), ctypes.byref(nb)))
    return b.value, sp.value, en.value, od.value, gr.value, nb.value


def stomsfem_plan_upscale_ms(h):
    """Device time (ms) of the upscaling launches of the plan's last step."""
    v = ctypes.c_float()
    L.check(L.lib().stomsfem_plan_upscale_ms(h, ctypes.byref(v)))
    return v.value


def stomsfem_ri_save(h):
    return _save(L.lib().stomsfem_ri_save, h)


def stomsfem_ri_load(data: bytes):
    buf = ctypes.create_string_buffer(data, len(data))
    h = ctypes.c_void_p()
    nfam = ctypes.c_int32()
    L.check(L.lib().stomsfem_ri_load(buf, len(data), ctypes.byref(h), ctypes.byref(nfam)))
    return h, nfam.value


# ---------------------------------------------------------------- local KL

KL_BUMPS, KL_GAUSSIAN, KL_MAX_N = 0, 1, 112


def stomsfem_local_kl_build(g: Grid, oversample, cov_kind, fld: Field = None, var=1.0 / 3.0, beta=0.1,
                            sigma=1.0, kmax=16, energy=0.0, stream=None):
    """Returns (handle, K per cell list)."""
    h = ctypes.c_void_p()
    ncell = g.nc * g.nc
    k = (ctypes.c_int32 * ncell)()
    L.check(L.lib().stomsfem_local_kl_build(ctypes.byref(g), int(oversample), int(cov_kind),
                                            ctypes.byref(fld) if fld is not None else None, float(var),
                                            float(beta), float(sigma), int(kmax), float(energy), ctypes.byref(h),
                                            ctypes.cast(k, ctypes.c_void_p), _stream(stream)))
    return h, list(k)


def stomsfem_local_kl_destroy(h):
    L.check(L.lib().stomsfem_local_kl_destroy(h))


def stomsfem_local_kl_modes(h, g: Grid, kmax):
    """(lam [ncell][kmax], w [ncell][kmax][112]) host arrays."""
    import numpy as np
    ncell = g.nc * g.nc
    lam = np.empty((ncell, kmax))
    w = np.empty((ncell, kmax, KL_MAX_N))
    L.check(L.lib().stomsfem_local_kl_modes(h, lam.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p)))
    return lam, w


def stomsfem_local_kl_project(h, kappa, xi, kappa_bar=None, stream=None):
    S = kappa.shape[0]
    L.check(L.lib().stomsfem_local_kl_project(h, _dev(kappa, torch.float64, None, "kappa"),
                                              _dev(kappa_bar, torch.float64, None, "kappa_bar"), S,
                                              _dev(xi, torch.float64, None, "xi"), _stream(stream)))
