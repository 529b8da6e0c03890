"""Learned surrogate on the GPU: gradients of the fused training kernel
(BF16 products, FP32 accumulation) against the FP64 oracle, training that
reduces the loss, and (once trained) inference with fallback."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1607_00693_gb300 import api
from paper_1607_00693_gb300 import workloads as W

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1607_00693_gb300.build import build_library
    build_library()


def test_gradients_match_oracle():
    from oracle import surrogate as S
    r = np.random.default_rng(7)
    w = api.xavier_weights(1, 3)[0].astype(np.float64)
    w[2048:2176] = r.standard_normal(128) * 0.1           # nonzero biases
    X = r.uniform(-1, 1, (64, 16))
    X[:, 9:] = 0.0
    T = r.standard_normal((64, 16)) * 0.3
    L_o, g_o = S.loss_and_grad(w, X, T)
    wt = torch.tensor(w, dtype=torch.float32, device=DEV)
    grad = torch.empty(api.SURROGATE_PARAMS, dtype=torch.float32, device=DEV)
    loss = torch.empty(1, dtype=torch.float32, device=DEV)
    api.stomsfem_surrogate_grad(wt, torch.tensor(X, dtype=torch.float32, device=DEV),
                                torch.tensor(T, dtype=torch.float32, device=DEV), grad, loss)
    g = grad.cpu().numpy().astype(np.float64)
    assert loss.item() == pytest.approx(L_o, rel=2e-2)
    # per parameter tensor, relative error in the norm (BF16 products)
    off = 0
    for shp in S.SHAPES:
        n = int(np.prod(shp))
        go, gg = g_o[off:off + n], g[off:off + n]
        if np.linalg.norm(go) > 0:
            assert np.linalg.norm(gg - go) / np.linalg.norm(go) <= 2e-2, (shp, off)
        off += n


def _training_set(S, seed):
    import oracle
    w = W.workload("surrogate_64")
    xi = W.draw_xi(w["field"], S, seed)
    g = api.grid(w["nf"], w["nc"], w["f"])
    xt = torch.from_numpy(xi).to(DEV)
    a = torch.empty((S, w["nf"], w["nf"]), dtype=torch.float64, device=DEV)
    api.stomsfem_sample_coef(g, api.field_from_dict(w["field"]), xt, a)
    Ke = torch.empty((S, w["nc"] ** 2, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((S, w["nc"] ** 2, 4), dtype=torch.float64, device=DEV)
    api.stomsfem_upscale(g, a, Ke, be)
    return w, g, xt, a, Ke, be


def test_training_reduces_loss():
    w, g, xt, a, Ke, be = _training_set(256, 4)
    fld = api.field_from_dict(w["field"])
    _, _, _, nfam = api.stomsfem_local_vars(g, fld, 1e-6)
    h, nf2 = api.stomsfem_surrogate_create(g, fld, 1e-6, api.xavier_weights(nfam, 0))
    assert nf2 == nfam == 36
    try:
        loss = api.stomsfem_surrogate_train(h, xt, a, Ke, be, steps=400, lr=2e-3, seed=1)
        assert np.all(np.isfinite(loss))
        assert loss[-20:].mean() < 0.05 * loss[:5].mean()
    finally:
        api.stomsfem_surrogate_destroy(h)
