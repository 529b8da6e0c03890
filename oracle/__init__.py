"""Plain FP64 CPU oracle for the StoMsFEM local-upscaling hot path.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` use it; the product library never
imports, links or calls anything here, and this package imports nothing
from the product package.

Parts (each follows the paper's definitions, Hou-Li-Zhang, arXiv 1607.00693):

* ``sample_coef``   -- coefficient a(x, xi) at fine-element centroids
                        (nonlinear transform, Sec. 2.1.3; C code).
* ``upscale``       -- per-sample MsFEM: cell problems (Eq. MsFEB) on the
                        fine mesh, oversampling recombination (Remark in
                        Sec. 2.2), K_e and b_e (Eq. stiffness_local); C code.
                        ``bc=BC_OSCILLATORY`` gives the cell problems the
                        oscillatory boundary data of Sec. 5.3 (harmonic
                        coordinate along each patch edge) instead of the
                        bilinear data; ``cell``, ``cell_pg`` and
                        ``upscale_pg`` take it too.
* ``coarse_solve``  -- coarse assembly and solve (Eq. upscaleSUF); C code.
* ``upscale_pg``, ``coarse_solve_pg`` -- the Petrov-Galerkin form (Eq.
                        stiffness_local_petrov: bilinear test functions,
                        deterministic load; non-symmetric coarse system by
                        banded LU); C code.
* ``coarse_solve_bc`` -- the coarse system with prescribed values on chosen
                        nodes and zero flux elsewhere (Sec. 5.2, Eqs.
                        xsquarewave / ysquarewave), Galerkin or
                        Petrov-Galerkin; C code.
* ``fine_fem``      -- standard Q1 FEM on the fine grid; C code.
* ``mc_moments``    -- Monte Carlo mean and variance (Eq. MCestimate),
                        two-pass.
* ``two_level_mean`` -- the two-level estimator of Eq. MCmean2level with
                        ``restrict_to_coarse`` (fine solution at the coarse
                        nodes).
* ``pod``           -- reduced basis by KL of the basis functions in the
                        energy inner product (Eq. KLphi) and the Galerkin
                        reduced system (Eqs. localRB, localRBsystem).
* ``mlp``           -- FP64 MLP forward/backward/Adam for the surrogate.
* ``ri``            -- random interpolation of K_e and b_e in the local
                        parameters (Sec. 3.1, Algorithms 1-2).
* ``local_kl``      -- the local KL expansion of a random field on a patch
                        (Sec. 2.1.1): restricted covariance, eigenpairs,
                        local parameters, truncation.

The C part is compiled on first use (gcc, -O2, OpenMP) into
``oracle/_build/liborc.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stomsfem_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (plain gcc, no GPU)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        lib.orc_sample_coef.argtypes = [i, i, i, i, d, d, d, d, p, i, p, i]
        lib.orc_sample_coef_window.argtypes = [i, i, i, i, d, d, d, d, p, i, i, i, i, p]
        lib.orc_cell.argtypes = [i, i, d, p, i, i, i, p, p, p, p]
        lib.orc_upscale.argtypes = [i, i, d, p, p, i, p, p, p, p, i]
        lib.orc_coarse_solve.argtypes = [i, p, p, i, p]
        lib.orc_fine_fem.argtypes = [i, d, p, p]
        lib.orc_band_solve_dense.argtypes = [i, i, p, p]
        lib.orc_cell_pg.argtypes = [i, i, d, p, i, i, i, p, p]
        lib.orc_cell_bc.argtypes = [i, i, d, p, i, i, i, i, p, p, p, p]
        lib.orc_upscale_bc.argtypes = [i, i, d, p, p, i, i, p, p, p, p, i]
        lib.orc_cell_pg_bc.argtypes = [i, i, d, p, i, i, i, i, p, p]
        lib.orc_upscale_pg_bc.argtypes = [i, i, d, p, p, i, i, p, p, p, i]
        lib.orc_upscale_pg.argtypes = [i, i, d, p, p, i, p, p, p, i]
        lib.orc_coarse_solve_pg.argtypes = [i, p, p, i, p]
        lib.orc_coarse_solve_bc.argtypes = [i, i, p, p, p, p, i, p]
        lib.orc_patch_bounds.argtypes = [i, i, i, i, i, p, p, p, p]
        _lib = lib
    return _lib


def _ptr(x):
    return None if x is None else x.ctypes.data_as(ctypes.c_void_p)


def ncores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


FIELD_EXP = 0
FIELD_EXP_SIGMOID = 1


def sample_coef(nf, field, xi, nthreads=0):
    """a[S][nf][nf] at element centroids; ``field`` is a dict with keys
    kind, nbx, nby, width, scale, contrast_log, gain."""
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    S = xi.shape[0]
    a = np.empty((S, nf, nf), dtype=np.float64)
    rc = _L().orc_sample_coef(nf, int(field["kind"]), int(field["nbx"]), int(field["nby"]),
                              float(field["width"]), float(field.get("scale", 1.0)),
                              float(field.get("contrast_log", 0.0)),
                              float(field.get("gain", 1.0)), _ptr(xi), S, _ptr(a), nthreads)
    if rc != 0:
        raise ValueError("orc_sample_coef failed: %d" % rc)
    return a


def sample_coef_window(nf, field, xi_row, ex0, ex1, ey0, ey1, out=None):
    """The coefficient of one sample on the element window [ex0,ex1)x[ey0,ey1)
    of an nf x nf array (other entries: ``out``'s, default NaN)."""
    xi_row = np.ascontiguousarray(xi_row, dtype=np.float64)
    a = np.full((nf, nf), np.nan) if out is None else out
    rc = _L().orc_sample_coef_window(nf, int(field["kind"]), int(field["nbx"]), int(field["nby"]),
                                     float(field["width"]), float(field.get("scale", 1.0)),
                                     float(field.get("contrast_log", 0.0)),
                                     float(field.get("gain", 1.0)), _ptr(xi_row), ex0, ex1, ey0,
                                     ey1, _ptr(a))
    if rc != 0:
        raise ValueError("orc_sample_coef_window failed")
    return a


def patch_bounds(nf, nc, cx, cy, o):
    v = [ctypes.c_int() for _ in range(4)]
    _L().orc_patch_bounds(nf, nc, cx, cy, o, *[ctypes.byref(x) for x in v])
    return tuple(x.value for x in v)  # x0, x1, y0, y1


BC_BILINEAR = 0      # Eq. MsFEB: bilinear nodal functions on the patch boundary
BC_OSCILLATORY = 1   # harmonic coordinate along each patch edge (Sec. 5.3)


def cell(nf, nc, f, a2d, cx, cy, o=0, bc=BC_BILINEAR):
    """One unit.  Returns (Ke[10], be[4], phi[4][rho+1][rho+1],
    psi[4][Ny+1][Nx+1]); ``bc`` selects the cell problems' boundary data."""
    a2d = np.ascontiguousarray(a2d, dtype=np.float64)
    rho = nf // nc
    x0, x1, y0, y1 = patch_bounds(nf, nc, cx, cy, o)
    Ke = np.empty(10)
    be = np.empty(4)
    phi = np.empty((4, rho + 1, rho + 1))
    psi = np.empty((4, y1 - y0 + 1, x1 - x0 + 1))
    rc = _L().orc_cell_bc(nf, nc, f, _ptr(a2d), cx, cy, o, bc, _ptr(Ke), _ptr(be), _ptr(phi), _ptr(psi))
    if rc != 0:
        raise ValueError("orc_cell failed: %d" % rc)
    return Ke, be, phi, psi


def upscale(nf, nc, f, a, oversample=None, want_phi=False, nthreads=0, bc=BC_BILINEAR):
    """Ke[S][nc*nc][10], be[S][nc*nc][4] (and phi[S][nc*nc][4][(rho+1)^2])."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    S = a.shape[0]
    rho = nf // nc
    Ke = np.empty((S, nc * nc, 10))
    be = np.empty((S, nc * nc, 4))
    phi = np.empty((S, nc * nc, 4, (rho + 1) ** 2)) if want_phi else None
    st = np.zeros(S * nc * nc, dtype=np.int32)
    ov = None
    if oversample is not None:
        ov = np.ascontiguousarray(oversample, dtype=np.int8)
    rc = _L().orc_upscale_bc(nf, nc, f, _ptr(a), _ptr(ov), bc, S, _ptr(Ke), _ptr(be), _ptr(phi),
                             _ptr(st), nthreads)
    if rc != 0:
        raise ValueError("orc_upscale failed: %d (first bad unit %d)" % (rc, int(np.argmax(st != 0))))
    return (Ke, be, phi) if want_phi else (Ke, be)


def cell_pg(nf, nc, f, a2d, cx, cy, o=0, bc=BC_BILINEAR):
    """One unit in the Petrov-Galerkin form: (Kpg[4][4] (row trial l,
    column test l'), bpg[4])."""
    a2d = np.ascontiguousarray(a2d, dtype=np.float64)
    K = np.empty(16)
    b = np.empty(4)
    rc = _L().orc_cell_pg_bc(nf, nc, f, _ptr(a2d), cx, cy, o, bc, _ptr(K), _ptr(b))
    if rc != 0:
        raise ValueError("orc_cell_pg failed: %d" % rc)
    return K.reshape(4, 4), b


def upscale_pg(nf, nc, f, a, oversample=None, nthreads=0, bc=BC_BILINEAR):
    """Kpg[S][nc*nc][16] (row-major 4x4, row trial, column test), bpg[S][nc*nc][4]."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    S = a.shape[0]
    K = np.empty((S, nc * nc, 16))
    b = np.empty((S, nc * nc, 4))
    st = np.zeros(S * nc * nc, dtype=np.int32)
    ov = None if oversample is None else np.ascontiguousarray(oversample, dtype=np.int8)
    rc = _L().orc_upscale_pg_bc(nf, nc, f, _ptr(a), _ptr(ov), bc, S, _ptr(K), _ptr(b), _ptr(st), nthreads)
    if rc != 0:
        raise ValueError("orc_upscale_pg failed: %d" % rc)
    return K, b


def coarse_solve_pg(nc, Kpg, bpg):
    Kpg = np.ascontiguousarray(Kpg, dtype=np.float64)
    bpg = np.ascontiguousarray(bpg, dtype=np.float64)
    S = Kpg.shape[0]
    u = np.empty((S, (nc + 1) ** 2))
    rc = _L().orc_coarse_solve_pg(nc, _ptr(Kpg), _ptr(bpg), S, _ptr(u))
    if rc != 0:
        raise ValueError("orc_coarse_solve_pg failed: %d" % rc)
    return u


def coarse_solve_bc(nc, K, b, dirichlet, g, pg=False):
    """Coarse solve with mixed boundary data (Sec. 5.2, Eqs. xsquarewave /
    ysquarewave): u = g where ``dirichlet`` [(nc+1)^2] is nonzero, zero flux
    on the rest of the boundary; every coarse node is an unknown.  ``K`` is
    the packed Galerkin K_e [S][nc*nc][10], or with ``pg`` the
    Petrov-Galerkin S_e [S][nc*nc][16].  Returns u [S][(nc+1)^2]; raises on
    a zero pivot (e.g. no Dirichlet node)."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    dm = np.ascontiguousarray(dirichlet, dtype=np.uint8).reshape(-1)
    g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
    assert dm.size == (nc + 1) ** 2 and g.size == dm.size
    S = K.shape[0]
    u = np.empty((S, (nc + 1) ** 2))
    rc = _L().orc_coarse_solve_bc(nc, 1 if pg else 0, _ptr(K), _ptr(b), _ptr(dm), _ptr(g), S, _ptr(u))
    if rc != 0:
        raise ValueError("orc_coarse_solve_bc failed: %d" % rc)
    return u


def coarse_solve(nc, Ke, be):
    Ke = np.ascontiguousarray(Ke, dtype=np.float64)
    be = np.ascontiguousarray(be, dtype=np.float64)
    S = Ke.shape[0]
    u = np.empty((S, (nc + 1) ** 2))
    rc = _L().orc_coarse_solve(nc, _ptr(Ke), _ptr(be), S, _ptr(u))
    if rc != 0:
        raise ValueError("orc_coarse_solve failed: %d" % rc)
    return u


def fine_fem(nf, f, a2d):
    a2d = np.ascontiguousarray(a2d, dtype=np.float64)
    u = np.empty((nf + 1) ** 2)
    rc = _L().orc_fine_fem(nf, f, _ptr(a2d), _ptr(u))
    if rc != 0:
        raise ValueError("orc_fine_fem failed: %d" % rc)
    return u


def band_solve_dense(A, bw, b):
    """The oracle's own banded Cholesky applied to a full SPD matrix."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    x = np.array(b, dtype=np.float64, copy=True)
    rc = _L().orc_band_solve_dense(A.shape[0], bw, _ptr(A), _ptr(x))
    if rc != 0:
        raise ValueError("orc_band_solve_dense failed: %d" % rc)
    return x


def restrict_to_coarse(u_fine, nf, nc):
    """u_fine [S][(nf+1)^2] at the coarse nodes -> [S][(nc+1)^2]."""
    rho = nf // nc
    S = u_fine.shape[0]
    return u_fine.reshape(S, nf + 1, nf + 1)[:, ::rho, ::rho].reshape(S, -1)


def two_level_mean(uH_0, uh_1, uH_1):
    """Eq. MCmean2level: mean of u_H over the level-0 samples plus the mean
    of (u_h - u_H) over the level-1 samples (u_h at the coarse nodes); also
    the sampling variance estimate var_0/N_0 + var_1/N_1 per node."""
    d = uh_1 - uH_1
    est = uH_0.mean(axis=0) + d.mean(axis=0)
    var = uH_0.var(axis=0) / uH_0.shape[0] + d.var(axis=0) / d.shape[0]
    return est, var


def mc_moments(u):
    """Eq. MCestimate: sample mean and the population variance
    M[u^2] - M[u]^2, evaluated two-pass as M[(u - M[u])^2]."""
    u = np.asarray(u, dtype=np.float64)
    mean = u.sum(axis=0) / u.shape[0]
    var = ((u - mean) ** 2).sum(axis=0) / u.shape[0]
    return mean, var


def pack_upper(M):
    """4x4 symmetric -> 10 packed upper-triangle entries (row-major)."""
    return np.array([M[l, lp] for l in range(4) for lp in range(l, 4)])


def unpack_upper(k):
    M = np.empty((4, 4))
    q = 0
    for l in range(4):
        for lp in range(l, 4):
            M[l, lp] = M[lp, l] = k[q]
            q += 1
    return M
