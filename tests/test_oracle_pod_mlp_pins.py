"""Pins of the POD and MLP oracles (no GPU)."""
import math

import numpy as np
import pytest

from paper_1607_00693_gb300 import workloads as W


def _training(orc, nf=32, nc=4, Ns=40, seed=3):
    field = dict(kind=0, nbx=4, nby=4, width=0.1, scale=1.0)
    xi = W.draw_xi(field, Ns, seed)
    a = orc.sample_coef(nf, field, xi)
    _, _, phi = orc.upscale(nf, nc, 1.0, a, want_phi=True)
    return field, a, phi


@pytest.fixture(scope="module")
def pod_setup():
    import oracle
    from oracle import pod
    oracle.build()
    field, a, phi = _training(oracle)
    return oracle, pod, field, a, phi


def test_pod_full_rank_reproduces_msfem(pod_setup):
    """With the full interior space as reduced basis the Galerkin reduced
    system is the cell problem itself: K_e and b_e equal plain MsFEM."""
    orc, pod, field, a, phi = pod_setup
    nf, nc = 32, 4
    n_int = (nf // nc - 1) ** 2
    models = pod.build(nf, nc, phi, a, ranks=[n_int] * (nc * nc))
    xi = W.draw_xi(field, 3, 99)
    at = orc.sample_coef(nf, field, xi)
    Ke, be = pod.upscale(models, nf, nc, 1.0, at)
    Ke0, be0 = orc.upscale(nf, nc, 1.0, at)
    assert np.linalg.norm(Ke - Ke0) / np.linalg.norm(Ke0) < 1e-10
    assert np.linalg.norm(be - be0) / np.linalg.norm(be0) < 1e-10


def test_pod_basis_properties(pod_setup):
    """V is orthonormal in the training-mean energy inner product; the
    eigenvalues are non-negative and non-increasing; the snapshot energy
    outside span(V) equals the sum of the dropped eigenvalues
    (Eckart-Young for the KL expansion); the truncation rule is monotone
    in the tolerance."""
    orc, pod, field, a, phi = pod_setup
    nf, nc = 32, 4
    rho = nf // nc
    inner = pod.interior_mask(rho)
    cell = 5
    cx, cy = cell % nc, cell // nc
    ac = pod.cell_coef(a, nc, cx, cy)
    m = pod.build_cell(phi[:, cell], ac, tol=1e-4)
    Abar = pod.cell_stiffness(ac.mean(axis=0))
    V = m["V"]
    G = V.T @ Abar @ V
    np.testing.assert_allclose(G, np.eye(m["rank"]), atol=1e-10)
    lam = m["lam"]
    assert np.all(np.diff(lam) <= 1e-14 * lam[0]) and lam[-1] > -1e-12 * lam[0]
    # energy of the centred snapshots left outside span(V)
    X = (phi[:, cell] - m["phibar"][None]).reshape(-1, phi.shape[-1])
    Pr = V @ (V.T @ Abar @ X.T)
    Rm = X.T - Pr
    tail = np.einsum("ik,ij,jk->", Rm, Abar, Rm) / X.shape[0]
    assert tail == pytest.approx(lam[m["rank"]:].sum(), rel=1e-6, abs=1e-14 * lam[0])
    r2 = pod.build_cell(phi[:, cell], ac, tol=1e-6)["rank"]
    r1 = pod.build_cell(phi[:, cell], ac, tol=1e-2)["rank"]
    assert r1 <= m["rank"] <= r2
    assert np.sqrt(lam[m["rank"] - 1] / lam[0]) >= 1e-4 > np.sqrt(max(lam[m["rank"]], 0) / lam[0])
    # phi_bar is the training mean: it keeps the partition of unity
    np.testing.assert_allclose(m["phibar"].sum(axis=0), 1.0, atol=1e-13)
    del inner


def test_pod_invariance_and_structure(pod_setup):
    """The reduced K_e depends on span(V) only (V -> V Q), keeps symmetric
    zero row sums, and its error falls as the rank grows."""
    orc, pod, field, a, phi = pod_setup
    nf, nc = 32, 4
    cell = 6
    cx, cy = cell % nc, cell // nc
    ac = pod.cell_coef(a, nc, cx, cy)
    at = orc.sample_coef(nf, field, W.draw_xi(field, 1, 123))
    ref, _, _, _ = orc.cell(nf, nc, 1.0, at[0], cx, cy, 0)
    errs = []
    for r in (2, 4, 8):
        m = pod.build_cell(phi[:, cell], ac, rank=r)
        Ke, _ = pod.online_cell(m, pod.cell_coef(at[0], nc, cx, cy), 1.0, 1.0 / nf)
        Q, _ = np.linalg.qr(np.random.default_rng(r).standard_normal((r, r)))
        m2 = dict(m, V=m["V"] @ Q)
        Ke2, _ = pod.online_cell(m2, pod.cell_coef(at[0], nc, cx, cy), 1.0, 1.0 / nf)
        np.testing.assert_allclose(Ke2, Ke, rtol=1e-11, atol=1e-12)
        K = orc.unpack_upper(Ke)
        np.testing.assert_allclose(K.sum(axis=1), 0.0, atol=1e-12 * np.abs(K).max())
        errs.append(np.linalg.norm(Ke - ref) / np.linalg.norm(ref))
    assert errs[2] <= errs[1] <= errs[0]
    # energy minimisation: the reduced diagonal entries bound the exact ones from above
    m = pod.build_cell(phi[:, cell], ac, rank=2)
    Ke, _ = pod.online_cell(m, pod.cell_coef(at[0], nc, cx, cy), 1.0, 1.0 / nf)
    for q in (0, 4, 7, 9):
        assert Ke[q] >= ref[q] * (1 - 1e-12)


# ---------------------------------------------------------------- MLP

def _params(k=5, width=7, out=4, seed=0):
    r = np.random.default_rng(seed)
    dims = [k, width, width, width, out]
    return [(r.standard_normal((dims[i], dims[i + 1])) / math.sqrt(dims[i]),
             r.standard_normal(dims[i + 1]) * 0.1) for i in range(4)]


def test_gelu_known_values():
    from oracle import mlp
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    # Phi(1) = 0.8413447460685429 (standard normal CDF)
    assert mlp.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-15)
    assert mlp.gelu(np.array([-1.0]))[0] == pytest.approx(-1 + 0.8413447460685429, rel=1e-14)
    t = np.linspace(-3, 3, 13)
    fd = (mlp.gelu(t + 1e-6) - mlp.gelu(t - 1e-6)) / 2e-6
    np.testing.assert_allclose(mlp.gelu_grad(t), fd, rtol=1e-8, atol=1e-9)


def test_mlp_backward_central_differences():
    from oracle import mlp
    P = _params()
    r = np.random.default_rng(1)
    x = r.standard_normal((6, 5))
    t = r.standard_normal((6, 4))
    y, cache = mlp.forward(P, x)
    grads = mlp.backward(P, cache, y, t)
    eps = 1e-6
    for li in range(4):
        for j in range(2):
            arr = P[li][j]
            flat = arr.reshape(-1)
            for idx in r.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + eps
                lp = mlp.loss(mlp.forward(P, x)[0], t)
                flat[idx] = old - eps
                lm = mlp.loss(mlp.forward(P, x)[0], t)
                flat[idx] = old
                g = grads[li][j].reshape(-1)[idx]
                assert g == pytest.approx((lp - lm) / (2 * eps), rel=1e-6, abs=1e-9)


def test_adam_first_step_is_signed_lr():
    """With bias correction, Adam's first step moves every parameter by
    -lr * g / (|g| + eps'), i.e. by lr against the sign of its gradient."""
    from oracle import mlp
    P = _params()
    G = [(np.full_like(W, 0.3) * np.sign(np.random.default_rng(2).standard_normal(W.shape)),
          np.full_like(b, -2.0)) for W, b in P]
    P0 = [(W.copy(), b.copy()) for W, b in P]
    st = mlp.adam_init(P)
    mlp.adam_step(P, G, st, lr=1e-3, eps=1e-12)
    for (W, b), (W0, b0), (gW, gb) in zip(P, P0, G):
        np.testing.assert_allclose(W - W0, -1e-3 * np.sign(gW), rtol=1e-9)
        np.testing.assert_allclose(b - b0, -1e-3 * np.sign(gb), rtol=1e-9)


def test_zero_row_sum_projector():
    from oracle import mlp, unpack_upper, pack_upper
    Pm = mlp.zero_row_sum_projector()
    np.testing.assert_allclose(Pm @ Pm, Pm, atol=1e-14)
    np.testing.assert_allclose(Pm, Pm.T, atol=1e-14)
    assert np.linalg.matrix_rank(Pm) == 6
    r = np.random.default_rng(3)
    O = r.standard_normal((4, 4))
    O = O + O.T
    np.fill_diagonal(O, 0)
    np.fill_diagonal(O, -O.sum(axis=1))
    k = pack_upper(O)
    np.testing.assert_allclose(Pm @ k, k, atol=1e-14)
    y = r.standard_normal(10)
    np.testing.assert_allclose(unpack_upper(Pm @ y).sum(axis=1), 0.0, atol=1e-13)


def test_surrogate_flat_layout_gradient():
    """The surrogate oracle's flat-layout loss gradient (13 used outputs)
    against central differences."""
    from oracle import surrogate as S
    r = np.random.default_rng(0)
    w = r.standard_normal(S.N_PARAMS) * 0.05
    X = r.standard_normal((8, 16))
    T = r.standard_normal((8, 16))
    L, g = S.loss_and_grad(w, X, T)

    def lossf(wv):
        return float(np.mean((S.forward(wv, X) - T)[:, :13] ** 2))

    assert L == pytest.approx(lossf(w), rel=1e-14)
    for idx in [0, 2047, 2100, 5000, 20000, 35000, 37250, 37260]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += 1e-6
        wm[idx] -= 1e-6
        assert g[idx] == pytest.approx((lossf(wp) - lossf(wm)) / 2e-6, rel=1e-6, abs=1e-10)
    # outputs 13..15 carry no loss: their last-layer rows have zero gradient
    o = S.N_PARAMS - 16 - 16 * 128
    assert np.all(g[o + 13 * 128:o + 16 * 128] == 0) and np.all(g[-3:] == 0)


def test_surrogate_predict_structure():
    from oracle import surrogate as S, unpack_upper
    r = np.random.default_rng(1)
    K, b = S.predict(r.standard_normal(16) * 0.1, 2.5, 1.3, 0.125)
    np.testing.assert_allclose(unpack_upper(K).sum(axis=1), 0.0, atol=1e-14)
    assert b.sum() == pytest.approx(1.3 * 0.125 ** 2, rel=1e-14)
    K0, b0 = S.predict(np.zeros(16), 2.5, 1.0, 0.125)
    np.testing.assert_allclose(K0, 2.5 * S.KREF_PACKED, rtol=1e-15)
