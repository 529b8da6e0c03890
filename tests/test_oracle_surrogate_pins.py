"""Pins of the surrogate oracle's local parameters, error indicator and
training loop (no GPU).

The indicator is fixed by closed forms: a constant coefficient gives
K_e = c K_ref with both energy bounds attained; a medium layered across x
attains the arithmetic mean along the layers (the y-linear function solves
the cell problem exactly) and lies between the harmonic and arithmetic
means across them; subtracting beta v_h v_h^T (v_h the hourglass corner
vector, an eigenvector of K_ref with eigenvalue 2/3 and norm^2 4) leaves
both energies unchanged and makes K indefinite exactly when beta > 1/6.
The minibatch draw is SplitMix64, checked against the generator's published
output for seed 1234567; Adam's first step moves every weight by -lr sign(g)
and the cosine schedule starts at lr and ends at lr_min."""
import math
import os

import numpy as np
import pytest

from oracle import surrogate as S
from paper_1607_00693_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KREF = S.KREF_PACKED


def _golden_local_vars():
    rows = []
    for line in open(os.path.join(GOLDEN, "local_vars_cell_1_2.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        p = line.split()
        rows.append((float(p[0]), int(p[1]), [int(v) for v in p[2:]]))
    return rows


def test_local_vars_hand_worked_cell():
    """Cell (1, 2) of the 64^2 / 8^2 grid with 4 x 4 bumps of width 0.1:
    the local bumps and their order at three thresholds, worked by hand
    (tests/golden/local_vars_cell_1_2.txt)."""
    field = dict(kind=0, nbx=4, nby=4, width=0.1, scale=1.0)
    cell = 2 * 8 + 1
    rows = _golden_local_vars()
    assert len(rows) == 3
    for tau, k, ids in rows:
        kk, idd, _, _ = S.local_vars(64, 8, field, tau)
        assert kk[cell] == k
        assert list(idd[cell, :k]) == ids
        assert np.all(idd[cell, k:] == -1)


def _box(lo=-1.0, hi=1.0):
    b = np.zeros((16, 2))
    b[:, 0], b[:, 1] = lo, hi
    return b


def test_indicator_constant_coefficient(orc):
    """a = c: K_e = c K_ref (the bilinears are discrete-harmonic), both
    corner energies equal c = abar = ahar; accepted with any slack, and a
    scaling by 1 +- 2 delta crosses the upper / lower bound."""
    c = 3.5
    a = np.full((1, 64, 64), c)
    Ke, _ = orc.upscale(64, 8, 1.0, a)
    Kp = Ke[0, 9]
    ex, ey = S.energy_values(Kp)
    assert ex == pytest.approx(c, rel=1e-13) and ey == pytest.approx(c, rel=1e-13)
    x, box = np.zeros(16), _box()
    d = 0.01
    assert S.indicator(x, box, 0.01, Kp, c, c, d) == {"range": False, "energy": False, "pd": False}
    assert S.indicator(x, box, 0.01, Kp * (1 + 2 * d), c, c, d)["energy"]
    assert S.indicator(x, box, 0.01, Kp * (1 - 2 * d), c, c, d)["energy"]
    assert not S.indicator(x, box, 0.01, Kp * (1 + 0.5 * d), c, c, d)["energy"]
    assert not S.indicator(x, box, 0.01, Kp * (1 - 0.5 * d), c, c, d)["energy"]


def test_indicator_layered_medium(orc):
    """a = a(x) layered across x: the y-linear energy equals the cell's
    arithmetic mean exactly; the x-linear energy lies between the harmonic
    and arithmetic means; the rule accepts the exact K_e at a tiny slack.
    The same values with the two means swapped are rejected (a swapped
    bound would not pass this pin)."""
    rng = np.random.default_rng(11)
    prof = np.exp(rng.uniform(-1.5, 1.5, 64))
    a = np.broadcast_to(prof[None, None, :], (1, 64, 64)).copy()
    Ke, _ = orc.upscale(64, 8, 1.0, a)
    for cell in (0, 13, 42):
        cx = cell % 8
        seg = prof[cx * 8:(cx + 1) * 8]
        abar, ahar = seg.mean(), 1.0 / np.mean(1.0 / seg)
        assert abar > 1.05 * ahar
        ex, ey = S.energy_values(Ke[0, cell])
        assert ey == pytest.approx(abar, rel=1e-12)
        assert ahar < ex < abar
        r = S.indicator(np.zeros(16), _box(), 0.01, Ke[0, cell], abar, ahar, 1e-9)
        assert not r["energy"] and not r["pd"]
        assert S.indicator(np.zeros(16), _box(), 0.01, Ke[0, cell], ahar, abar, 1e-9)["energy"]


def test_indicator_accepts_exact_msfem(orc):
    """Exact MsFEM matrices of the surrogate workload (o = 0) pass the rule
    at the default slack of 2%."""
    w = W.workload("surrogate_64")
    xi = W.draw_xi(w["field"], 6, 123)
    a = orc.sample_coef(w["nf"], w["field"], xi)
    Ke, _ = orc.upscale(w["nf"], w["nc"], w["f"], a)
    rho = w["nf"] // w["nc"]
    for s in range(6):
        for cell in range(w["nc"] ** 2):
            cx, cy = cell % w["nc"], cell // w["nc"]
            blk = a[s, cy * rho:(cy + 1) * rho, cx * rho:(cx + 1) * rho]
            r = S.indicator(np.zeros(16), _box(), 0.01, Ke[s, cell], blk.mean(), 1.0 / np.mean(1.0 / blk), 0.02)
            assert not any(r.values()), (s, cell, r)


def test_indicator_pd_closed_form():
    """K_ref - beta v_h v_h^T with v_h = (1, -1, 1, -1): corner energies stay
    1 (v_h is orthogonal to both affine corner vectors) and the matrix is
    indefinite on the complement of the constants iff beta > 1/6; the full
    4 x 4 spectrum (numpy) agrees."""
    vh = np.array([1.0, -1.0, 1.0, -1.0])
    Pvh = S.pack_upper_sym(np.outer(vh, vh))
    for beta, bad in ((0.10, False), (0.16, False), (0.17, True), (0.30, True)):
        Kp = KREF - beta * Pvh
        ex, ey = S.energy_values(Kp)
        assert ex == pytest.approx(1.0, abs=1e-14) and ey == pytest.approx(1.0, abs=1e-14)
        r = S.indicator(np.zeros(16), _box(), 0.01, Kp, 1.0, 1.0, 0.02)
        assert r == {"range": False, "energy": False, "pd": bad}
        lam = np.linalg.eigvalsh(S._sym4(Kp))
        assert (np.sum(lam < -1e-12) > 0) == bad
        assert min(abs(lam)) < 1e-12  # the constants stay in the kernel


def test_indicator_range_margin():
    """Inputs just inside / outside lo - m and hi + m, m = margin (hi - lo)."""
    box = _box(-0.5, 1.5)  # width 2, margin 1% -> 0.02
    Kp = KREF.copy()
    for j in (0, 7, 15):
        for v, bad in ((1.519, False), (1.521, True), (-0.519, False), (-0.521, True), (0.3, False)):
            x = np.zeros(16)
            x[j] = v
            assert S.indicator(x, box, 0.01, Kp, 1.0, 1.0, 0.02)["range"] == bad


def test_splitmix64_reference_values():
    """SplitMix64 with state 1234567: the generator's published first five
    outputs."""
    gamma = 0x9E3779B97F4A7C15
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    got = [S.splitmix64((1234567 + k * gamma) % (1 << 64)) for k in range(5)]
    assert got == want


def test_minibatch_rows_hold_out_every_tenth():
    for nrows in (7, 64, 1000):
        for step in range(20):
            r = S.minibatch_rows(5, 3, step, nrows)
            assert len(r) == 64 and all(0 <= v < nrows for v in r)
            assert all(v % 10 != 9 for v in r)


def test_train_first_step_and_schedule():
    """Adam's first bias-corrected step is -lr g / (|g| + eps): every weight
    with a non-negligible gradient moves by lr against its sign; the cosine
    rate equals lr at the first step and lr_min after the last."""
    rng = np.random.default_rng(3)
    w0 = rng.standard_normal(S.N_PARAMS) * 0.05
    X = rng.uniform(-1, 1, (200, 16))
    T = rng.standard_normal((200, 16)) * 0.3
    lr = 1e-3
    w1, _, _, _ = S.train(w0, X, T, 1, lr=lr, lr_min=1e-5, seed=9)
    rows = S.minibatch_rows(9, 0, 0, 200)
    _, g = S.loss_and_grad(w0, X[rows], T[rows])
    big = np.abs(g) > 1e-4
    np.testing.assert_allclose((w1 - w0)[big], -lr * np.sign(g[big]), rtol=1e-3)
    # the rate of the last step of a 4-step call: lr_min + (lr - lr_min)(1 + cos(3 pi / 4)) / 2
    r3 = 1e-5 + 0.5 * (lr - 1e-5) * (1 + math.cos(math.pi * 3 / 4))
    assert 1e-5 < r3 < lr


def test_train_reduces_loss():
    rng = np.random.default_rng(4)
    w0 = rng.standard_normal(S.N_PARAMS) * 0.05
    X = rng.uniform(-1, 1, (300, 16))
    T = np.tanh(X[:, :16] @ rng.standard_normal((16, 16)) * 0.3)
    _, _, _, loss = S.train(w0, X, T, 60, lr=3e-3, lr_min=1e-4, seed=1)
    assert loss[-10:].mean() < 0.5 * loss[:3].mean()


def test_ensemble_disagreement_rule():
    """Identical predictions never disagree; a scaled copy (1 + eps) K
    disagrees exactly when |eps| > tol; the norm is the first network's
    (K2 = 2 K1 differs by ||K1||: flagged at tol 0.9 from K1's side, not
    from K2's, where the difference is half of ||K2||)."""
    from oracle import surrogate as S
    K1 = S.KREF_PACKED * 1.7
    for tol in (0.0, 0.01, 0.5):
        assert not S.ensemble_disagrees(K1, K1.copy(), tol)
    for eps, tol, want in ((0.049, 0.05, False), (0.051, 0.05, True), (-0.051, 0.05, True), (0.2, 0.25, False)):
        assert S.ensemble_disagrees(K1, (1 + eps) * K1, tol) == want, (eps, tol)
    assert S.ensemble_disagrees(K1, 2 * K1, 0.9)
    assert not S.ensemble_disagrees(2 * K1, K1, 0.9)
