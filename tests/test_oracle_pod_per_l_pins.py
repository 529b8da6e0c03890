"""Pins of the oracle's per-l reduced bases (the patch study of Sec. 5.1:
one KL basis for each of phi^1, phi^2, phi^3, phi^4 from the partition of
unity), no GPU.  Full rank reproduces the MsFEM; each basis is Abar-
orthonormal and its training tail energy is the sum of its dropped
eigenvalues (Eckart-Young); the partition of unity holds by construction;
the energy error of every phi_l is non-increasing in its own rank (nested
Galerkin spaces); a per-l basis is no worse than the shared basis of the
same rank for the function it was built for, on the training samples."""
import numpy as np
import pytest

from paper_1607_00693_gb300 import workloads as W

NF, NC = 32, 4
FIELD = dict(kind=0, nbx=4, nby=4, width=0.1, scale=1.0)


@pytest.fixture(scope="module")
def setup():
    import oracle
    from oracle import pod
    oracle.build()
    xi = W.draw_xi(FIELD, 40, 3)
    a = oracle.sample_coef(NF, FIELD, xi)
    _, _, phi = oracle.upscale(NF, NC, 1.0, a, want_phi=True)
    return oracle, pod, a, phi


def _unpack(k):
    M = np.zeros((4, 4))
    q = 0
    for l in range(4):
        for lp in range(l, 4):
            M[l, lp] = M[lp, l] = k[q]
            q += 1
    return M


def test_full_rank_reproduces_msfem(setup):
    orc, pod, a, phi = setup
    n_int = (NF // NC - 1) ** 2
    models = [pod.build_cell_per_l(phi[:, c], pod.cell_coef(a, NC, c % NC, c // NC), ranks=[n_int] * 3)
              for c in range(NC * NC)]
    at = orc.sample_coef(NF, FIELD, W.draw_xi(FIELD, 3, 99))
    Ke, be = pod.upscale_per_l(models, NF, NC, 1.0, at)
    Ke0, be0 = orc.upscale(NF, NC, 1.0, at)
    assert np.linalg.norm(Ke - Ke0) / np.linalg.norm(Ke0) < 1e-10
    assert np.linalg.norm(be - be0) / np.linalg.norm(be0) < 1e-10


def test_bases_orthonormal_with_eckart_young_tails(setup):
    orc, pod, a, phi = setup
    cell = 6
    ac = pod.cell_coef(a, NC, cell % NC, cell // NC)
    m = pod.build_cell_per_l(phi[:, cell], ac, tol=1e-4)
    Abar = pod.cell_stiffness(ac.mean(axis=0))
    assert len(m["V"]) == 3 and len(m["rank"]) == 3
    for l in range(3):
        V, lam, r = m["V"][l], m["lam"][l], m["rank"][l]
        np.testing.assert_allclose(V.T @ Abar @ V, np.eye(r), atol=1e-10)
        X = phi[:, cell, l] - m["phibar"][l][None]               # Ns x N2
        Rm = X.T - V @ (V.T @ Abar @ X.T)
        tail = np.einsum("ik,ij,jk->", Rm, Abar, Rm) / X.shape[0]
        assert tail == pytest.approx(lam[r:].sum(), rel=1e-6, abs=1e-14 * lam[0])
        assert np.sqrt(lam[r - 1] / lam[0]) >= 1e-4 > np.sqrt(max(lam[r], 0.0) / lam[0])


def test_partition_of_unity_and_structure(setup):
    """phi^4 = 1 - sum: K_e symmetric with zero row sums, sum b = f H^2,
    for truncated bases too."""
    orc, pod, a, phi = setup
    models = pod.build_per_l(NF, NC, phi, a, tol=1e-3)
    at = orc.sample_coef(NF, FIELD, W.draw_xi(FIELD, 2, 98))
    Ke, be = pod.upscale_per_l(models, NF, NC, 1.3, at)
    for k, b in zip(Ke.reshape(-1, 10), be.reshape(-1, 4)):
        M = _unpack(k)
        np.testing.assert_allclose(M.sum(axis=1), 0.0, atol=1e-12 * np.abs(M).max())
        assert b.sum() == pytest.approx(1.3 / NC ** 2, rel=1e-12)


def test_energy_error_non_increasing_in_rank(setup):
    """The Galerkin reduced phi_l is the A(omega)-orthogonal projection of
    the MsFEM phi_l onto phi_bar_l + span(V_l); the spans are nested in the
    rank, so its energy error cannot grow."""
    orc, pod, a, phi = setup
    cell = 9
    cx, cy = cell % NC, cell // NC
    ac = pod.cell_coef(a, NC, cx, cy)
    at = orc.sample_coef(NF, FIELD, W.draw_xi(FIELD, 1, 97))
    a_cell = pod.cell_coef(at[0], NC, cx, cy)
    _, _, phi_true, _ = orc.cell(NF, NC, 1.0, at[0], cx, cy, 0)
    A = pod.cell_stiffness(a_cell)
    for l in range(3):
        errs = []
        for r in (1, 2, 4, 8, 16):
            m = pod.build_cell_per_l(phi[:, cell], ac, ranks=[r] * 3)
            V = m["V"][l]
            c = np.linalg.solve(V.T @ A @ V, -(V.T @ A @ m["phibar"][l]))
            e = m["phibar"][l] + V @ c - phi_true[l].reshape(-1)
            errs.append(e @ A @ e)
        assert all(errs[i + 1] <= errs[i] * (1 + 1e-9) + 1e-18 for i in range(len(errs) - 1)), errs


def test_per_l_basis_fits_its_own_function_better_on_training(setup):
    """On the training snapshots, the Abar-projection tail of phi_l's
    centred snapshots is the smallest possible for its rank (its own KL),
    so the shared basis of the same rank leaves at least as much."""
    orc, pod, a, phi = setup
    cell = 3
    ac = pod.cell_coef(a, NC, cell % NC, cell // NC)
    Abar = pod.cell_stiffness(ac.mean(axis=0))
    r = 4
    per_l = pod.build_cell_per_l(phi[:, cell], ac, ranks=[r] * 3)
    shared = pod.build_cell(phi[:, cell], ac, rank=r)

    def tail(V, l):
        X = (phi[:, cell, l] - per_l["phibar"][l][None]).T
        Rm = X - V @ (V.T @ Abar @ X)
        return np.einsum("ik,ij,jk->", Rm, Abar, Rm)

    for l in range(3):
        assert tail(per_l["V"][l], l) <= tail(shared["V"], l) * (1 + 1e-10)
