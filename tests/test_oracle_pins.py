"""Pins of the FP64 oracle against what the paper and the mathematics fix
(closed forms, invariants, library solves, brute force on tiny grids).
Each test is chosen so that a plausible slip in the oracle (a dropped
term, a wrong sign or index, a transposed operand) fails at least one."""
import math

import numpy as np
import pytest

from tests import fem_ref
from paper_1607_00693_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

KREF_PACKED = np.array([4, -1, -2, -1, 4, -1, -2, 4, -1, 4]) / 6.0


def rng_a(nf, seed, lo=0.2, hi=5.0):
    r = np.random.default_rng(seed)
    return np.exp(r.uniform(np.log(lo), np.log(hi), size=(nf, nf)))


# ---------------------------------------------------------------- field

def test_field_one_hot_location_and_symmetry(orc):
    # a non-square lattice catches an x/y transpose of the bump index
    field = dict(kind=0, nbx=4, nby=2, width=0.15, scale=1.0)
    nf = 32
    for (bx, by) in [(0, 0), (3, 1), (1, 0)]:
        xi = np.zeros((1, 8))
        xi[0, by * 4 + bx] = 1.0
        la = np.log(orc.sample_coef(nf, field, xi)[0])
        ey, ex = np.unravel_index(np.argmax(la), la.shape)
        cx, cy = (bx + 0.5) / 4, (by + 0.5) / 2
        assert abs((ex + 0.5) / nf - cx) <= 0.5 / nf + 1e-12
        assert abs((ey + 0.5) / nf - cy) <= 0.5 / nf + 1e-12
        # centres of a 4x2 lattice on a 32 grid sit on element edges:
        # log a is mirror symmetric about them (within the grid)
        ic, jc = int(round(cx * nf)), int(round(cy * nf))
        w = min(ic, nf - ic, jc, nf - jc)
        blk = la[jc - w:jc + w, ic - w:ic + w]
        np.testing.assert_allclose(blk, blk[::-1, :], rtol=0, atol=1e-14)
        np.testing.assert_allclose(blk, blk[:, ::-1], rtol=0, atol=1e-14)


def test_field_superposition_and_scale(orc):
    field = dict(kind=0, nbx=3, nby=3, width=0.2, scale=0.7)
    r = np.random.default_rng(0)
    x1, x2 = r.uniform(-1, 1, (1, 9)), r.uniform(-1, 1, (1, 9))
    l1 = np.log(orc.sample_coef(16, field, x1))
    l2 = np.log(orc.sample_coef(16, field, x2))
    l12 = np.log(orc.sample_coef(16, field, x1 + x2))
    np.testing.assert_allclose(l12, l1 + l2, rtol=1e-13, atol=1e-13)
    f2 = dict(field, scale=1.4)
    np.testing.assert_allclose(np.log(orc.sample_coef(16, f2, x1)), 2 * l1, rtol=1e-13, atol=1e-13)


def test_field_gaussian_width(orc):
    # a lone bump of width w falls to exp(-d^2/w^2) of its peak: compare two
    # centroids at known distances d1, d2 from the centre (ratio of logs)
    field = dict(kind=0, nbx=1, nby=1, width=0.25, scale=1.0)
    nf = 64
    la = np.log(orc.sample_coef(nf, field, np.ones((1, 1)))[0])
    e1, e2 = (32, 32), (32, 44)      # (ey, ex)
    d1 = math.hypot((32.5 / nf - 0.5), (32.5 / nf - 0.5))
    d2 = math.hypot((44.5 / nf - 0.5), (32.5 / nf - 0.5))
    assert la[e2] / la[e1] == pytest.approx(math.exp(-(d2 ** 2 - d1 ** 2) / 0.25 ** 2), rel=1e-13)


def test_field_sigmoid_kind(orc):
    field = dict(kind=1, nbx=2, nby=2, width=0.2, contrast_log=math.log(1e4), gain=8.0)
    # z = 0 gives sigma = 1/2, a = exp(ln(1e4)/2) = 100 exactly
    a0 = orc.sample_coef(8, field, np.zeros((1, 4)))
    np.testing.assert_allclose(a0, 100.0, rtol=1e-14)
    a = orc.sample_coef(16, field, np.random.default_rng(1).standard_normal((3, 4)) * 3)
    assert np.all(a > 1.0) and np.all(a < 1e4)


# ------------------------------------------------------- banded Cholesky

@pytest.mark.parametrize("n,bw", [(1, 1), (7, 2), (30, 6), (49, 8)])
def test_band_solver_matches_library(orc, n, bw):
    r = np.random.default_rng(n)
    B = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - bw), i + 1):
            B[i, j] = r.uniform(-1, 1)
    A = B @ B.T + n * np.eye(n)
    A[np.abs(np.subtract.outer(np.arange(n), np.arange(n))) > bw] = 0.0
    A += 2 * n * np.eye(n)
    b = r.uniform(-1, 1, n)
    np.testing.assert_allclose(orc.band_solve_dense(A, bw, b), np.linalg.solve(A, b),
                               rtol=1e-12, atol=1e-13)


# ------------------------------------------------------------ cell problem

@pytest.mark.parametrize("nf,nc,o", [(8, 4, 0), (16, 4, 0), (16, 4, 1), (24, 3, 2), (32, 4, 3)])
def test_P1_constant_coefficient(orc, nf, nc, o):
    """a == c: the bilinear nodal functions are discrete-harmonic, so the
    basis is bilinear and K_e = c K_ref, b_l = f H^2 / 4 (every cell,
    clipped and unclipped patches)."""
    c, f = 3.7, 1.3
    a = np.full((1, nf, nf), c)
    ov = np.full(nc * nc, o, dtype=np.int8)
    Ke, be = orc.upscale(nf, nc, f, a, ov)
    H = 1.0 / nc
    np.testing.assert_allclose(Ke[0], np.tile(c * KREF_PACKED, (nc * nc, 1)), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(be[0], f * H * H / 4.0, rtol=1e-13)


@pytest.mark.parametrize("o", [0, 2])
def test_P2_layered_along_layers_is_arithmetic_mean(orc, o):
    """a = a(x): the y-linear function solves the cell problem exactly, so
    for v = (0,0,1,1) (value 1 on the top corners) v^T K_e v is the
    arithmetic mean of a over the cell; across the layers (v = (0,1,1,0))
    the energy lies between the harmonic and arithmetic means."""
    nf, nc = 32, 4
    rho = nf // nc
    prof = np.exp(np.random.default_rng(3).uniform(-2, 2, nf))
    a = np.tile(prof[None, :], (nf, 1))[None]
    Ke, _ = orc.upscale(nf, nc, 1.0, a, np.full(nc * nc, o, dtype=np.int8))
    vy = np.array([0, 0, 1, 1.0])
    vx = np.array([0, 1, 1, 0.0])
    for cell in range(nc * nc):
        cx = cell % nc
        seg = prof[cx * rho:(cx + 1) * rho]
        K = orc.unpack_upper(Ke[0, cell])
        assert vy @ K @ vy == pytest.approx(seg.mean(), rel=1e-13)
        if o == 0:
            e = vx @ K @ vx
            assert 1.0 / np.mean(1.0 / seg) * (1 - 1e-13) <= e <= seg.mean() * (1 + 1e-13)
    # the transposed layering pins the other axis
    aT = np.transpose(a, (0, 2, 1)).copy()
    KeT, _ = orc.upscale(nf, nc, 1.0, aT, np.full(nc * nc, o, dtype=np.int8))
    for cell in range(nc * nc):
        cy = cell // nc
        seg = prof[cy * rho:(cy + 1) * rho]
        K = orc.unpack_upper(KeT[0, cell])
        assert vx @ K @ vx == pytest.approx(seg.mean(), rel=1e-13)


@pytest.mark.parametrize("nf,nc,o", [(16, 4, 0), (24, 3, 2), (40, 5, 4)])
def test_P3_invariants(orc, nf, nc, o):
    """Symmetric PSD K_e with kernel span{1}; partition of unity of the
    basis; loads summing to f H^2 (each of the four cell problems is
    solved separately by the oracle, so these are genuine checks)."""
    a = rng_a(nf, nf + o)[None]
    f = 2.0
    rho = nf // nc
    H = 1.0 / nc
    for cell in range(nc * nc):
        cx, cy = cell % nc, cell // nc
        Ke, be, phi, psi = orc.cell(nf, nc, f, a[0], cx, cy, o)
        K = orc.unpack_upper(Ke)
        scale = np.abs(K).max()
        np.testing.assert_allclose(K.sum(axis=1), 0.0, atol=1e-13 * scale)
        ev = np.linalg.eigvalsh(K)
        assert ev[0] > -1e-13 * scale and ev[1] > 1e-6 * scale
        np.testing.assert_allclose(phi.sum(axis=0), 1.0, atol=1e-13)
        np.testing.assert_allclose(psi.sum(axis=0), 1.0, atol=1e-13)
        assert be.sum() == pytest.approx(f * H * H, rel=1e-13)
        # nodal at the cell corners
        corners = [(0, 0), (0, rho), (rho, rho), (rho, 0)]   # (j, i)
        for l in range(4):
            for k, (j, i) in enumerate(corners):
                assert phi[l, j, i] == pytest.approx(1.0 if l == k else 0.0, abs=1e-13)
        # symmetric: recompute S from phi with the test's own assembly
        A = fem_ref.stiffness(a[0, cy * rho:(cy + 1) * rho, cx * rho:(cx + 1) * rho])
        P = phi.reshape(4, -1)
        np.testing.assert_allclose(P @ A @ P.T, K, rtol=1e-12, atol=1e-13 * scale)


def test_P6_brute_force_small_patches(orc):
    """rho = 2: one interior node, psi_c = -(sum of off-diagonal row
    entries times boundary values) / diagonal.  rho = 4 and oversampled
    patches: the harmonic extension by a dense library solve."""
    nf, nc = 8, 4
    a = rng_a(nf, 7)
    for cell in range(16):
        cx, cy = cell % nc, cell // nc
        _, _, _, psi = orc.cell(nf, nc, 1.0, a, cx, cy, 0)
        blk = a[cy * 2:cy * 2 + 2, cx * 2:cx * 2 + 2]
        # diagonal (2/3) sum a; edge neighbours -(1/6)(a_1 + a_2); corners -(1/3) a
        aSW, aSE, aNE, aNW = blk[0, 0], blk[0, 1], blk[1, 1], blk[1, 0]
        diag = (2.0 / 3.0) * (aSW + aSE + aNE + aNW)
        for l in range(4):
            p = fem_ref.bilinear(2, 2)[l].reshape(3, 3)
            s = (-(aSW + aSE) / 6 * p[0, 1] - (aNE + aNW) / 6 * p[2, 1]
                 - (aSW + aNW) / 6 * p[1, 0] - (aSE + aNE) / 6 * p[1, 2]
                 - aSW / 3 * p[0, 0] - aSE / 3 * p[0, 2] - aNE / 3 * p[2, 2] - aNW / 3 * p[2, 0])
            assert psi[l, 1, 1] == pytest.approx(-s / diag, rel=1e-13)
    nf, nc = 24, 3
    a = rng_a(nf, 8)
    for (cx, cy, o) in [(1, 1, 0), (0, 0, 2), (1, 2, 3), (2, 1, 1)]:
        _, _, _, psi = orc.cell(nf, nc, 1.0, a, cx, cy, o)
        x0, x1, y0, y1 = orc.patch_bounds(nf, nc, cx, cy, o)
        blk = a[y0:y1, x0:x1]
        g = fem_ref.bilinear(x1 - x0, y1 - y0)
        for l in range(4):
            ref = fem_ref.harmonic_extension(blk, g[l])
            np.testing.assert_allclose(psi[l].reshape(-1), ref, rtol=1e-12, atol=1e-13)


def test_energy_minimality(orc):
    """The cell-problem solution minimises the energy among functions with
    the same boundary data: random interior perturbations never lower it."""
    nf, nc = 24, 3
    a = rng_a(nf, 9)
    _, _, _, psi = orc.cell(nf, nc, 1.0, a, 1, 1, 0)
    A = fem_ref.stiffness(a[8:16, 8:16])
    it = ~fem_ref.boundary_mask(8, 8)
    r = np.random.default_rng(0)
    for l in range(4):
        u = psi[l].reshape(-1)
        e0 = u @ A @ u
        for _ in range(5):
            d = np.zeros_like(u)
            d[it] = r.standard_normal(it.sum()) * 1e-3
            assert (u + d) @ A @ (u + d) > e0


@pytest.mark.parametrize("nf", [6, 12])
def test_P4_H_equals_h(orc, nf):
    """rho = 1: no interior nodes; K_e = a_e K_ref and the coarse system is
    the fine FEM system, so the MsFEM solution equals the fine solution."""
    a = rng_a(nf, nf)[None]
    Ke, be = orc.upscale(nf, nf, 1.0, a)
    np.testing.assert_allclose(Ke[0], a[0].reshape(-1, 1) * KREF_PACKED[None], rtol=1e-14)
    u = orc.coarse_solve(nf, Ke, be)[0]
    uf = orc.fine_fem(nf, 1.0, a[0])
    np.testing.assert_allclose(u, uf, rtol=1e-12, atol=1e-15)


def test_fine_fem_library_solve(orc):
    nf = 10
    a = rng_a(nf, 11)
    A = fem_ref.stiffness(a)
    bd = fem_ref.boundary_mask(nf, nf)
    it = ~bd
    F = np.zeros((nf + 1) ** 2)
    h = 1.0 / nf
    for ey in range(nf):
        for ex in range(nf):
            for (j, i) in [(ey, ex), (ey, ex + 1), (ey + 1, ex + 1), (ey + 1, ex)]:
                F[j * (nf + 1) + i] += 0.7 * h * h / 4
    ref = np.zeros_like(F)
    ref[it] = np.linalg.solve(A[np.ix_(it, it)], F[it])
    np.testing.assert_allclose(orc.fine_fem(nf, 0.7, a), ref, rtol=1e-12, atol=1e-16)


def test_coarse_solve_constant_is_coarse_Q1(orc):
    """a == 1: the multiscale space is the coarse bilinear space, so the
    MsFEM solution equals standard Q1 FEM on the coarse grid."""
    nf, nc = 32, 8
    Ke, be = orc.upscale(nf, nc, 1.0, np.ones((1, nf, nf)))
    u = orc.coarse_solve(nc, Ke, be)[0]
    np.testing.assert_allclose(u, orc.fine_fem(nc, 1.0, np.ones((nc, nc))), rtol=1e-12, atol=1e-16)


def _global_basis(orc, nf, nc, a):
    """Fine-grid representation of every coarse nodal basis function."""
    rho = nf // nc
    N = nf + 1
    Phi = np.zeros(((nc + 1) ** 2, N * N))
    Ke, be, phi = orc.upscale(nf, nc, 1.0, a[None], want_phi=True)
    for cell in range(nc * nc):
        cx, cy = cell % nc, cell // nc
        corners = [(cx, cy), (cx + 1, cy), (cx + 1, cy + 1), (cx, cy + 1)]
        for l, (I, J) in enumerate(corners):
            loc = phi[0, cell, l].reshape(rho + 1, rho + 1)
            for j in range(rho + 1):
                for i in range(rho + 1):
                    Phi[J * (nc + 1) + I, (cy * rho + j) * N + cx * rho + i] = loc[j, i]
    return Phi, Ke, be


def test_P5_galerkin_orthogonality(orc):
    """No oversampling: the multiscale space is a conforming subspace of the
    fine Q1 space, so S_IJ = a_h(Phi_I, Phi_J), b_J = (f, Phi_J), and the
    fine solution minus the MsFEM solution is a_h-orthogonal to every
    coarse basis function; its energy never exceeds the fine energy."""
    nf, nc = 24, 4
    a = rng_a(nf, 12)
    Phi, Ke, be = _global_basis(orc, nf, nc, a)
    A = fem_ref.stiffness(a)
    h = 1.0 / nf
    F = np.zeros((nf + 1) ** 2)
    for ey in range(nf):
        for ex in range(nf):
            for (j, i) in [(ey, ex), (ey, ex + 1), (ey + 1, ex + 1), (ey + 1, ex)]:
                F[j * (nf + 1) + i] += h * h / 4
    uh = orc.fine_fem(nf, 1.0, a)
    U = orc.coarse_solve(nc, Ke, be)[0]
    uH = U @ Phi
    inner = [J for J in range((nc + 1) ** 2) if 0 < J % (nc + 1) < nc and 0 < J // (nc + 1) < nc]
    PhiI = Phi[inner]
    # coarse matrix from K_e equals the Galerkin matrix of the fine operator
    S = PhiI @ A @ PhiI.T
    Sref = np.zeros_like(S)
    pos = {J: q for q, J in enumerate(inner)}
    for cell in range(nc * nc):
        cx, cy = cell % nc, cell // nc
        K = orc.unpack_upper(Ke[0, cell])
        nodes = [cy * (nc + 1) + cx, cy * (nc + 1) + cx + 1, (cy + 1) * (nc + 1) + cx + 1,
                 (cy + 1) * (nc + 1) + cx]
        for r in range(4):
            for c in range(4):
                if nodes[r] in pos and nodes[c] in pos:
                    Sref[pos[nodes[r]], pos[nodes[c]]] += K[r, c]
    np.testing.assert_allclose(S, Sref, rtol=1e-11, atol=1e-12 * np.abs(S).max())
    # b_J equals (f, Phi_J)
    bref = np.zeros(len(inner))
    for cell in range(nc * nc):
        cx, cy = cell % nc, cell // nc
        nodes = [cy * (nc + 1) + cx, cy * (nc + 1) + cx + 1, (cy + 1) * (nc + 1) + cx + 1,
                 (cy + 1) * (nc + 1) + cx]
        for r in range(4):
            if nodes[r] in pos:
                bref[pos[nodes[r]]] += be[0, cell, r]
    np.testing.assert_allclose(PhiI @ F, bref, rtol=1e-12)
    # Galerkin orthogonality
    res = PhiI @ (A @ (uh - uH))
    assert np.abs(res).max() <= 1e-11 * np.abs(PhiI @ F).max()
    assert uH @ A @ uH <= uh @ A @ uh * (1 + 1e-12)


def test_P9_mc_moments(orc):
    u = np.random.default_rng(5).standard_normal((37, 11)) * 3 + 1
    m, v = orc.mc_moments(u)
    np.testing.assert_allclose(m, np.mean(u, axis=0), rtol=1e-14)
    np.testing.assert_allclose(v, np.var(u, axis=0), rtol=1e-13)


def test_workload_msfem_64_smoke(orc):
    """The msfem_64 workload end to end on a few samples: invariants hold and
    the MsFEM solution is close to the fine solution."""
    w = W.workload("msfem_64")
    xi = W.draw_xi(w["field"], 3, w["seed"])
    a = orc.sample_coef(w["nf"], w["field"], xi)
    Ke, be = orc.upscale(w["nf"], w["nc"], w["f"], a)
    assert np.abs(be.sum(axis=(1, 2)) - 1.0).max() < 1e-13
    u = orc.coarse_solve(w["nc"], Ke, be)
    uf = orc.fine_fem(w["nf"], 1.0, a[0])
    r = w["nf"] // w["nc"]
    uf_c = uf.reshape(w["nf"] + 1, -1)[::r, ::r].reshape(-1)
    assert np.linalg.norm(u[0] - uf_c) / np.linalg.norm(uf_c) < 0.1


def test_field_window_matches_full_field(orc):
    field = dict(kind=1, nbx=3, nby=2, width=0.2, contrast_log=math.log(1e4), gain=8.0)
    xi = np.random.default_rng(4).standard_normal((1, 6))
    full = orc.sample_coef(24, field, xi)[0]
    win = orc.sample_coef_window(24, field, xi[0], 5, 17, 3, 11)
    np.testing.assert_array_equal(win[3:11, 5:17], full[3:11, 5:17])
    assert np.isnan(win[0, 0])


def test_two_level_estimator_telescopes():
    """Eq. MCmean2level with the same samples on both levels is the plain
    fine-grid mean; the coarse-node restriction picks every rho-th node."""
    import oracle
    oracle.build()
    nf, nc = 32, 4
    fld = dict(kind=0, nbx=4, nby=4, width=0.1, scale=1.0)
    a = oracle.sample_coef(nf, fld, W.draw_xi(fld, 6, 41))
    Ke, be = oracle.upscale(nf, nc, 1.0, a)
    uH = oracle.coarse_solve(nc, Ke, be)
    uh = np.stack([oracle.fine_fem(nf, 1.0, a[s]) for s in range(6)])
    uhc = oracle.restrict_to_coarse(uh, nf, nc)
    assert uhc.shape == uH.shape
    np.testing.assert_array_equal(uhc.reshape(6, nc + 1, nc + 1)[:, 1, 2],
                                  uh.reshape(6, nf + 1, nf + 1)[:, 8, 16])
    est, var = oracle.two_level_mean(uH, uhc, uH)
    np.testing.assert_allclose(est, uhc.mean(axis=0), rtol=1e-13, atol=1e-16)
    # independent halves: the estimate is the coarse mean plus the mean correction
    est2, var2 = oracle.two_level_mean(uH[:3], uhc[3:], uH[3:])
    np.testing.assert_allclose(est2, uH[:3].mean(0) + (uhc[3:] - uH[3:]).mean(0), rtol=1e-13, atol=1e-16)
    assert np.all(var2 >= 0)
